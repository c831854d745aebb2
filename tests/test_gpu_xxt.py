"""The XX^T reduced solver (Sec. 2: A_r^{-1} = X X^T, X sparse with
A_r-conjugate columns in a nested-dissection order of the box lattice) on the
GPU: t = X^T r_r by column segments, u_r = X t by rows, against the FP64
oracle and against the dense explicit inverse.

Thresholds: u_r against the oracle's Cholesky solve and its own XX^T solve,
relative max norm <= 1e-12 (FP64 form) and <= 1e-11 (float-pair X in the
mixed forms, ~2^-48 per entry and per operation); M r as in the per-step
parity tests; solves at rtol 1e-10 take the dense form's iteration count
within one and agree to 1e-8 in the relative 2-norm.
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


CASES = {
    "cube8": lambda: meshes.workload_cube8(),
    "ragged": lambda: (meshes.cube((5, 3, 7), perturb=0.15, seed=3, boxes=(3, 2, 3), name="ragged"),
                       meshes.rhs(6 * 4 * 8, 9)),
    "mixed": lambda: (meshes.cube(11, perturb=0.15, seed=[2, 7], part_mode="mixed", name="mixed"),
                      meshes.rhs(12 ** 3, 10)),
    "cyl": lambda: meshes.workload_cylinder(scale=8),
    "cube32": lambda: meshes.workload_cube32(),
}
_cache = {}


def problem(name):
    if name not in _cache:
        m, b = CASES[name]()
        _cache[name] = (m, b, O.Problem(m.xyz, m.conn, m.part, m.boxes))
    return _cache[name]


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


def mesh(ctx, name, prec="fp64", form="hybrid", coarse="xxt"):
    m, b, P = problem(name)
    return m, b, P, cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form, coarse=coarse)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coarse_solve_xxt_against_oracle(ctx, name, prec):
    m, b, P, h = mesh(ctx, name, prec)
    with h:
        info = cgs.cgs_mesh_info(h.handle)
        assert info["coarse_solver"] == cgs.COARSE["xxt"] and info["n_r"] == P.nr
        assert 0 < info["xxt_nnz"] <= P.nr * (P.nr + 1) // 2
        rng = np.random.default_rng(11)
        tol = 1e-12 if prec == "fp64" else 1e-11
        for _ in range(2):   # t is cleared between calls
            u = rng.standard_normal(P.nr)
            ur = torch.empty(max(P.nr, 1), dtype=torch.float64, device="cuda")
            cgs.cgs_coarse_solve(h.handle, dev(u), ur)
            got = host(ur)[:P.nr]
            assert rel_inf(got, P.coarse_solve(u)) <= tol
            assert rel_inf(got, P.coarse_solve_xxt(u)) <= tol


@pytest.mark.parametrize("form", ["hybrid", "additive"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_preconditioner_xxt(ctx, form, prec):
    m, b, P, h = mesh(ctx, "mixed", prec, form)
    with h:
        r = np.random.default_rng(4).standard_normal(m.nv)
        z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        for _ in range(2):
            cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
            assert rel_inf(host(z), P.apply_M(r, form)) <= (1e-11 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("name", ["cube8", "mixed", "cyl"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_solve_xxt_matches_dense(ctx, name, prec, form):
    m, b, _ = problem(name)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form, coarse="dense") as hd, \
            cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form, coarse="xxt") as hx:
        assert cgs.cgs_mesh_info(hd.handle)["coarse_solver"] == cgs.COARSE["dense"]
        x0 = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        x1 = torch.empty_like(x0)
        st0, it0, _ = cgs.cgs_solve(hd.handle, dev(b), x0, rtol=1e-10)
        st1, it1, rel1 = cgs.cgs_solve(hx.handle, dev(b), x1, rtol=1e-10)
        assert st0 == cgs.OK and st1 == cgs.OK
        assert abs(int(it0[0]) - int(it1[0])) <= 1 and rel1[0] <= 1e-10
        a, c = host(x0), host(x1)
        assert np.linalg.norm(a - c) / np.linalg.norm(a) <= 1e-8


def test_batch_and_server_mix_dense_and_xxt(ctx):
    """One batch (and one server) holding dense and XX^T meshes: every slot
    matches its own single-mesh solve."""
    names = ["cube8", "mixed", "ragged"]
    hs, bs, xs, ref = [], [], [], []
    try:
        for i, name in enumerate(names):
            m, b, _ = problem(name)
            h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32",
                         coarse="xxt" if i % 2 == 0 else "dense")
            hs.append(h)
            bs.append(dev(b))
            xs.append(torch.empty(m.nv, dtype=torch.float64, device="cuda"))
            x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
            st, it, _ = cgs.cgs_solve(h.handle, bs[-1], x, rtol=1e-10)
            assert st == cgs.OK
            ref.append((host(x), int(it[0])))
        batch = cgs.cgs_batch_create(ctx, hs, 1)
        try:
            st, its, rel, sts = cgs.cgs_batch_solve(batch, bs, xs, rtol=1e-10)
            assert st == cgs.OK
            for k, (x, it) in enumerate(ref):
                assert abs(int(its[k]) - it) <= 1
                assert np.linalg.norm(host(xs[k]) - x) <= 1e-8 * np.linalg.norm(x)
        finally:
            cgs.cgs_batch_free(batch)
        max_nr = max(h.info["n_r"] for h in hs)
        server = cgs.cgs_server_create(ctx, 4, 1 << 16, 4 * max_nr, prec="fp32", rtol=1e-10)
        try:
            tickets = [cgs.cgs_submit(server, h, b, x) for h, b, x in zip(hs, bs, xs)]
            done = {}
            for _ in range(200):
                cgs.cgs_server_step(server, iterations=8)
                for tk, it, r, s in cgs.cgs_server_drain(server):
                    done[tk] = (it, r, s)
                if len(done) == len(tickets):
                    break
            assert len(done) == len(tickets)
            for tk, (x, it) in zip(tickets, ref):
                assert done[tk][2] == cgs.OK
            for k, (x, it) in enumerate(ref):
                assert np.linalg.norm(host(xs[k]) - x) <= 1e-8 * np.linalg.norm(x)
        finally:
            cgs.cgs_server_free(server)
    finally:
        for h in hs:
            h.free()


def test_xxt_footprint_and_persistent_fallback(ctx):
    m, b, P, hx = mesh(ctx, "cube32", "fp32")
    with hx, cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32", coarse="dense") as hd:
        ix, id_ = cgs.cgs_mesh_info(hx.handle), cgs.cgs_mesh_info(hd.handle)
        # X by columns and by rows (10 bytes an entry each) instead of n_r^2 pairs
        assert ix["footprint_bytes"] < id_["footprint_bytes"]
        # the persistent loop runs the dense product only: XX^T meshes stay on the graph loop
        cgs.cgs_mesh_set_schedule(hx.handle, persistent=1)
        assert cgs.cgs_mesh_info(hx.handle)["loop"] == 1
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, it, rel = cgs.cgs_solve(hx.handle, dev(b), x, rtol=1e-8)
        assert st == cgs.OK and rel[0] <= 1e-8


def test_auto_picks_by_size_and_bad_value_rejected(ctx):
    m, b, P, h = mesh(ctx, "cube8", "fp64", coarse="auto")
    with h:
        assert cgs.cgs_mesh_info(h.handle)["coarse_solver"] == cgs.COARSE["dense"]   # n_r = 125 <= 1500
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, None, m.part, m.boxes, 0.0, 1, "fp64", "hybrid", 7)
    assert ei.value.status == cgs.ERR_INVALID_ARG
