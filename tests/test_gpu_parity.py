"""GPU parity: every hot-path step, called through the C ABI, against the FP64
CPU oracle on the same seeded inputs.

Thresholds (FP64 form): relative max-norm difference <= 1e-12 for A x and the
box-space steps, <= 1e-11 for local solves and M r; solves at rtol 1e-11
reach a true relative residual <= 1e-10 and a relative solution difference
<= 1e-9; iteration counts at rtol 1e-8 differ by at most one.  Integer and
index results (Dirichlet set, subdomain index sets, active box vertices) are
bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


WORKLOADS = {
    "cube8": lambda: meshes.workload_cube8(),
    "cube32": lambda: meshes.workload_cube32(),
    "ragged": lambda: (meshes.cube((5, 3, 7), perturb=0.15, seed=3, boxes=(3, 2, 3), name="ragged"),
                       meshes.rhs(6 * 4 * 8, 9)),
    "mixed": lambda: (meshes.cube(11, perturb=0.15, seed=[2, 7], part_mode="mixed", name="mixed"),
                      meshes.rhs(12 ** 3, 10)),
    "cyl": lambda: meshes.workload_cylinder(scale=8),
}


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


_cache = {}


def problem(name):
    if name not in _cache:
        m, b = WORKLOADS[name]()
        _cache[name] = (m, b, O.Problem(m.xyz, m.conn, m.part, m.boxes))
    return _cache[name]


@pytest.fixture
def mesh_of(ctx):
    made = []

    def make(name, prec="fp64", form="hybrid"):
        m, b, P = problem(name)
        h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form)
        made.append(h)
        return m, b, P, h

    yield make
    for h in made:
        h.free()


NAMES = list(WORKLOADS)


@pytest.mark.parametrize("name", NAMES)
def test_setup_index_sets_bit_exact(mesh_of, name):
    m, b, P, h = mesh_of(name)
    ex = cgs.cgs_mesh_export(h.handle)
    np.testing.assert_array_equal(ex["dirichlet"].astype(bool), P.dir)
    np.testing.assert_array_equal(ex["box_active"], P.box_active)
    assert h.info["n_free"] == P.free.size and h.info["n_r"] == P.nr
    assert h.info["n_sub"] == len(P.sub_idx)
    for p, idx in enumerate(P.sub_idx):
        np.testing.assert_array_equal(ex["sub_idx"][ex["sub_ptr"][p]:ex["sub_ptr"][p + 1]], idx)


@pytest.mark.parametrize("name", NAMES)
def test_apply_A(mesh_of, name):
    m, b, P, h = mesh_of(name)
    x = np.random.default_rng(1).standard_normal(m.nv)
    y = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    cgs.cgs_apply_A(h.handle, dev(x), y)
    ref = P.apply_A(np.where(P.dir, 0.0, x))
    got = host(y)
    assert rel_inf(got, ref) <= 1e-12
    assert np.all(got[P.dir] == 0)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("weighted", [True, False])
def test_apply_local(mesh_of, name, weighted):
    m, b, P, h = mesh_of(name)
    r = np.where(P.dir, 0.0, np.random.default_rng(2).standard_normal(m.nv))
    out = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    cgs.cgs_apply_local(h.handle, dev(r), out, weighted)
    assert rel_inf(host(out), P.local_solves(r, weighted)) <= 1e-11


@pytest.mark.parametrize("weighted", [True, False])
def test_fp64_lane_packs_against_oracle(ctx, weighted):
    """The FP64 form's lane packs (one lane per subdomain, the triangle walked
    by diagonals), used from 9,472 subdomains on: the halved cylinder (16,384
    subdomains of 2^3 elements, classes 18 to 27) entry by entry against the
    oracle's local solves (Sec. 3, Eq. (4)) at 1e-11."""
    m, _ = meshes.workload_cylinder(scale=2)
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    r = np.where(P.dir, 0.0, np.random.default_rng(5).standard_normal(m.nv))
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64") as h:
        assert h.info["n_sub"] == 16384 and h.info["n_lane_packs"] == 16384 // 32
        out = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_local(h.handle, dev(r), out, weighted)
        assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
        assert rel_inf(host(out), P.local_solves(r, weighted)) <= 1e-11


@pytest.mark.parametrize("name", NAMES)
def test_box_steps(mesh_of, name):
    m, b, P, h = mesh_of(name)
    rng = np.random.default_rng(3)
    s = np.where(P.dir, 0.0, rng.standard_normal(m.nv))
    rr = torch.empty(max(P.nr, 1), dtype=torch.float64, device="cuda")
    cgs.cgs_restrict(h.handle, dev(s), rr)
    assert rel_inf(host(rr)[:P.nr], P.restrict(s)) <= 1e-12
    u = rng.standard_normal(P.nr)
    ur = torch.empty(max(P.nr, 1), dtype=torch.float64, device="cuda")
    cgs.cgs_coarse_solve(h.handle, dev(u), ur)
    assert rel_inf(host(ur)[:P.nr], P.coarse_solve(u)) <= 1e-12
    z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    cgs.cgs_interp(h.handle, dev(u), z)
    assert rel_inf(host(z), P.interp(u)) <= 1e-12


@pytest.mark.parametrize("name", ["cube8", "cube32", "cyl"])
def test_coarse_solve_float_pair(mesh_of, name):
    """Mixed forms keep A_r^{-1} and r_r as hi/lo float pairs (~48 bits) and
    multiply on the FP32 pipes.  Against the oracle (a Cholesky solve) the
    max-norm difference stays below 1e-11; against the float64 product with
    the same explicit inverse (FP64 form) every entry is within the pair
    rounding bound 2^-45 sum_j |a_ij u_j| (entry and input rounding 2^-48
    each, pair sums over at most a few thousand terms)."""
    m, b, P, h = mesh_of(name, prec="fp32")
    m64, _, _, h64 = mesh_of(name, prec="fp64")
    u = np.random.default_rng(8).standard_normal(P.nr)
    ur = torch.empty(max(P.nr, 1), dtype=torch.float64, device="cuda")
    cgs.cgs_coarse_solve(h.handle, dev(u), ur)
    got = host(ur)[:P.nr]
    assert rel_inf(got, P.coarse_solve(u)) <= 1e-11
    cgs.cgs_coarse_solve(h64.handle, dev(u), ur)
    got64 = host(ur)[:P.nr]
    bound = 2.0 ** -45 * (np.abs(np.linalg.inv(P.Ar)) @ np.abs(u)) + 1e-300
    assert np.all(np.abs(got - got64) <= bound)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_preconditioner(mesh_of, name, form):
    m, b, P, h = mesh_of(name, form=form)
    r = np.random.default_rng(4).standard_normal(m.nv)
    z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
    assert rel_inf(host(z), P.apply_M(r, form)) <= 1e-11


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_preconditioner_reduced_precision(mesh_of, prec, form):
    """M r in the FP32-bulk and FP16-local forms against the FP64 oracle:
    relative max-norm difference <= 1e-5 (float rounding of the local
    inverses, the inner apply and the interpolation weights)."""
    m, b, P, h = mesh_of("cube32", prec=prec, form=form)
    r = np.random.default_rng(4).standard_normal(m.nv)
    z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
    tol = 1e-5 if prec == "fp32" else 2e-3
    assert rel_inf(host(z), P.apply_M(r, form)) <= tol


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_solve_fp64(mesh_of, name, form):
    m, b, P, h = mesh_of(name, form=form)
    x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    st, its, relres = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-11, maxit=500)
    assert st == cgs.OK
    xo, its_o, relres_o, ok = P.solve(b, rtol=1e-11, maxit=500, form=form)
    assert ok and relres[0] <= 1e-10
    xg = host(x)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-9
    # independent check of the GPU's reported residual with the oracle's operator
    bb = np.where(P.dir, 0.0, b)
    assert np.linalg.norm(bb - P.apply_A(xg)) / np.linalg.norm(bb) <= 1e-10
    st, its8, _ = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8, maxit=500)
    _, its8_o, _, _ = P.solve(b, rtol=1e-8, maxit=500, form=form)
    assert abs(int(its8[0]) - its8_o) <= 1


def test_multiple_rhs_and_host_entry(mesh_of):
    m, b, P, h = mesh_of("cube8")
    B3 = np.stack([b, 2.0 * b + 1.0, np.random.default_rng(7).standard_normal(m.nv)])
    X = torch.empty(3 * m.nv, dtype=torch.float64, device="cuda")
    st, its, rel = cgs.cgs_solve(h.handle, dev(B3.ravel()), X, nrhs=3, rtol=1e-10)
    assert st == cgs.OK and np.all(rel <= 1e-10)
    Xh = np.empty(3 * m.nv)
    st2, its2, rel2 = cgs.cgs_solve_host(h.handle, np.ascontiguousarray(B3.ravel()), Xh, nrhs=3, rtol=1e-10)
    assert st2 == cgs.OK and list(its2) == list(its)
    np.testing.assert_allclose(Xh, host(X), rtol=0, atol=1e-12 * np.abs(Xh).max())
    for k in range(3):
        xo, _, _, _ = P.solve(B3[k], rtol=1e-12)
        assert np.linalg.norm(Xh[k * m.nv:(k + 1) * m.nv] - xo) / np.linalg.norm(xo) <= 1e-8


# ---------------------------------------------------------------------------
# reduced-precision forms: error bounds and iteration counts
# ---------------------------------------------------------------------------

U32, U16 = 2.0 ** -24, 2.0 ** -11


def _abs_local_bound(P, r, weighted):
    """sum_p R_p^T |A_p^{-1}| |R_p r| (then W_ov), the magnitude the local-solve
    rounding errors scale with."""
    out = np.zeros(P.nv)
    for mm, (ps, I, Ap, L) in P.groups.items():
        inv = np.abs(np.linalg.inv(Ap))
        np.add.at(out, I.ravel(), (inv @ np.abs(r[I])[..., None])[..., 0].ravel())
    if weighted:
        nz = P.mult > 0
        out[nz] /= P.mult[nz]
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("name", ["cube32", "mixed", "cyl"])
def test_local_solve_error_within_bound(mesh_of, name, prec):
    """FP32: |dl| <= gamma_{m+12} W sum_p |A_p^-1||R_p r| (inverse and input
    rounded once, m-term dot, <= 8 atomic additions); FP16 adds 2 u16 for the
    scaled half-precision inverse entries and u32 * scale for subnormals."""
    m, b, P, h = mesh_of(name, prec=prec)
    r = np.where(P.dir, 0.0, np.random.default_rng(5).standard_normal(m.nv))
    out = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    cgs.cgs_apply_local(h.handle, dev(r), out, True)
    err = np.abs(host(out) - P.local_solves(r, True))
    mmax = h.info["max_sub_dofs"]
    g = (mmax + 12) * U32 / (1 - (mmax + 12) * U32)
    mag = _abs_local_bound(P, r, True)
    bound = (g + (2 * U16 if prec == "fp16" else 0.0)) * mag + 1e-300
    if prec == "fp16":
        # entries below the half-precision normal range lose relative accuracy
        bound += 2.0 ** -24 * max(abs(np.linalg.inv(Ap)).max() for (_, _, Ap, _) in P.groups.values()) \
            * mmax * np.abs(r).max()
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("name", ["cube32", "cyl"])
def test_mixed_precision_solve(mesh_of, name, prec):
    """FP64 outer PCG around reduced-precision preconditioners: the true
    residual still reaches the tolerance and the iteration count stays within
    one of the FP64 plain form."""
    m, b, P, h = mesh_of(name, prec=prec)
    m64, _, _, h64 = mesh_of(name, prec="fp64")
    x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8)
    st64, its64, rel64 = cgs.cgs_solve(h64.handle, dev(b), x, rtol=1e-8)
    assert st == cgs.OK and st64 == cgs.OK
    assert rel[0] <= 1.5e-8
    assert abs(int(its[0]) - int(its64[0])) <= 1
    st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-11)
    xo, _, _, _ = P.solve(b, rtol=1e-12)
    assert rel[0] <= 1e-10
    assert np.linalg.norm(host(x) - xo) / np.linalg.norm(xo) <= 1e-9


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_zero_rhs(mesh_of):
    m, b, P, h = mesh_of("cube8")
    x = dev(np.full(m.nv, 7.0))
    st, its, rel = cgs.cgs_solve(h.handle, dev(np.zeros(m.nv)), x)
    assert st == cgs.OK and its[0] == 0 and rel[0] == 0.0
    assert not host(x).any()


def test_maxit_reports_no_convergence(mesh_of):
    m, b, P, h = mesh_of("cube32")
    x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
    st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-14, maxit=3)
    assert st == cgs.ERR_NO_CONVERGENCE and its[0] == 3 and rel[0] > 1e-14


def test_single_element_all_dirichlet(ctx):
    m = meshes.cube(1)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=(1, 1, 1)) as h:
        assert h.info["n_free"] == 0 and h.info["n_r"] == 0
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, its, rel = cgs.cgs_solve(h.handle, dev(np.ones(m.nv)), x)
        assert st == cgs.OK and its[0] == 0 and not host(x).any()


def test_rank_deficient_coarse_space_reported(ctx):
    """One free vertex against eight box corners: J has rank 1, A_r is
    singular, and setup reports NOT_SPD (the oracle refuses it too)."""
    m = meshes.cube(2, perturb=0.1, seed=1)
    with pytest.raises(ValueError):
        O.Problem(m.xyz, m.conn, m.part, (1, 1, 1))
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, None, m.part, (1, 1, 1))
    assert ei.value.status == cgs.ERR_NOT_SPD


def test_one_box_small_mesh(ctx):
    m = meshes.cube(3, perturb=0.1, seed=1)
    P = O.Problem(m.xyz, m.conn, m.part, (1, 1, 1))
    b = meshes.rhs(m.nv, 3)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=(1, 1, 1)) as h:
        assert h.info["n_free"] == 8 and h.info["n_r"] == P.nr == 8
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-12)
        xo, its_o, _, _ = P.solve(b, rtol=1e-12)
        assert st == cgs.OK and abs(int(its[0]) - its_o) <= 1
        np.testing.assert_allclose(host(x), xo, rtol=1e-10, atol=1e-14)


def test_single_subdomain_is_exact(ctx):
    m = meshes.cube(4, perturb=0.15, seed=0, boxes=(2, 2, 2))
    b = meshes.rhs(m.nv, 1)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=np.zeros(m.ne, np.int32), boxes=m.boxes) as h:
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-12)
        assert st == cgs.OK and its[0] == 1 and rel[0] < 1e-12


def test_invalid_meshes_rejected(ctx):
    m = meshes.cube(3, perturb=0.1, seed=0)
    bad = m.conn.copy()
    bad[5, 3] = m.nv
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, bad, None, m.part, (2, 2, 2))
    assert ei.value.status == cgs.ERR_INVALID_MESH
    inv = m.conn.copy()
    inv[4] = inv[4][[1, 0, 3, 2, 5, 4, 7, 6]]      # mirrored element: negative Jacobian
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, inv, None, m.part, (2, 2, 2))
    assert ei.value.status == cgs.ERR_INVALID_MESH
    part = m.part.copy()
    part[0] = -1
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, None, part, (2, 2, 2))
    assert ei.value.status == cgs.ERR_INVALID_ARG
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, None, m.part, (0, 2, 2))
    assert ei.value.status == cgs.ERR_INVALID_ARG


def test_admission_budget():
    m, b = meshes.workload_cube8()
    c = cgs.cgs_create(0, 1 << 16)
    try:
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_mesh_setup(c, m.xyz, m.conn, None, m.part, m.boxes)
        assert ei.value.status == cgs.ERR_ADMISSION
        assert cgs.cgs_ctx_bytes_in_use(c) == 0
    finally:
        cgs.cgs_destroy(c)


# ---------------------------------------------------------------------------
# the full-size hollow cylinder (1,073,280 vertices): sampled outputs and
# properties that hold at any size
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_full_cylinder_sampled(ctx):
    m, b = meshes.workload_cylinder()
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        assert h.info["nv"] == 1073280 and h.info["n_sub"] == 131072
        dirm = O.dirichlet_mask(m.conn, m.nv)
        ex = cgs.cgs_mesh_export(h.handle)
        np.testing.assert_array_equal(ex["dirichlet"].astype(bool), dirm)
        rng = np.random.default_rng(12)
        xv = rng.standard_normal(m.nv)
        y = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_A(h.handle, dev(xv), y)
        got = host(y)
        rows = rng.choice(m.nv, 2000, replace=False)
        sel = np.flatnonzero(np.isin(m.conn, rows).any(axis=1))
        Ae, _ = O.element_matrices(m.xyz, m.conn[sel])
        xm = np.where(dirm, 0.0, xv)
        ref = np.zeros(m.nv)
        contrib = np.einsum("ekl,el->ek", Ae, xm[m.conn[sel]])
        np.add.at(ref, m.conn[sel].ravel(), contrib.ravel())
        ref[dirm] = 0.0
        scale = np.abs(ref[rows]).max()
        assert np.abs(got[rows] - ref[rows]).max() <= 1e-12 * scale
        # the solve: true residual checked with the oracle's assembled operator
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8)
        assert st == cgs.OK and rel[0] <= 1.5e-8
        Aeall, _ = O.element_matrices(m.xyz, m.conn)
        A = O.assemble(m.conn.astype(np.int64), Aeall, m.nv)
        bb = np.where(dirm, 0.0, b)
        xg = np.where(dirm, 0.0, host(x))
        res = bb - np.where(dirm, 0.0, A @ xg)
        assert np.linalg.norm(res) / np.linalg.norm(bb) <= 1.5e-8


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_cylinder_against_stored_oracle_results(ctx, prec):
    """The full-size cylinder in the launch configuration the benchmark times,
    against FP64 oracle results stored by tests/golden/make_cylinder_golden.py
    at 256 sampled free vertices: A b, the weighted local solves, M b (hybrid
    and additive), and the PCG solve to rtol 1e-8 (the oracle needs 300
    iterations).  FP64: 1e-12 for A b, 1e-11 for the preconditioner terms
    (relative to the largest sampled value); FP32 bulk: 1e-5.  Solves: the
    iteration count within one of the oracle's and the sampled solution within
    1e-6 relative (both stop at relres 1e-8 along the same iteration)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cylinder_oracle.json")))
    idx = np.array(g["idx"])
    m, b = meshes.workload_cylinder()
    dirm = O.dirichlet_mask(m.conn, m.nv)
    b = np.where(dirm, 0.0, b)
    tol = 1e-11 if prec == "fp64" else 1e-5
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) as h:
        cgs.cgs_mesh_tune(h.handle)
        bd = dev(b)
        out = torch.empty(m.nv, dtype=torch.float64, device="cuda")

        def check(got, key, t):
            ref = np.array(g[key])
            assert np.abs(got[idx] - ref).max() <= t * np.abs(ref).max(), key

        cgs.cgs_apply_A(h.handle, bd, out)
        check(host(out), "apply_A", 1e-12)
        cgs.cgs_apply_local(h.handle, bd, out, True)
        check(host(out), "local_w", tol)
        cgs.cgs_apply_preconditioner(h.handle, bd, out)
        check(host(out), "m_hybrid", tol)
        cgs.cgs_mesh_set_form(h.handle, "additive")
        cgs.cgs_apply_preconditioner(h.handle, bd, out)
        check(host(out), "m_additive", tol)
        cgs.cgs_mesh_set_form(h.handle, "hybrid")
        assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
        st, its, rel = cgs.cgs_solve(h.handle, bd, out, rtol=1e-8, maxit=1000)
        assert st == cgs.OK and rel[0] <= 1.5e-8
        assert abs(int(its[0]) - g["solve"]["iters"]) <= 1
        xs, xo = host(out)[idx], np.array(g["solve"]["x"])
        assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
