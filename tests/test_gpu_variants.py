"""The paper's variants of the method on the GPU, against the FP64 oracle.

* Neumann boundaries everywhere except an outflow cap (Sec. 5, the boundary
  conditions of the production runs): the set-up takes the Dirichlet mask;
  the operator, both preconditioner forms and the solve follow the oracle
  with the same mask.
* Restricted additive Schwarz (Sec. 3): local solutions keep only the nodes
  of the original subdomain, averaged where several store one.
* Inexact local solves (Sec. 6): k CG steps on each A_p from zero.
* Outer iterations other than the PCG: Schwarz-Richardson and flexible GMRES.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


_outflow = {}


def outflow_case():
    if not _outflow:
        m, b = meshes.workload_cylinder(scale=8)
        d = meshes.outflow_dirichlet(m)
        P = O.Problem(m.xyz, m.conn, m.part, m.boxes, dirichlet=d.astype(bool))
        _outflow.update(m=m, b=b, d=d, P=P, its={})
    return _outflow


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_outflow_boundary(ctx, prec, form):
    c = outflow_case()
    m, b, d, P = c["m"], c["b"], c["d"], c["P"]
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, dirichlet=d, prec=prec, form=form) as h:
        ex = cgs.cgs_mesh_export(h.handle)
        np.testing.assert_array_equal(ex["dirichlet"], d)
        np.testing.assert_array_equal(ex["box_active"], P.box_active)
        r = np.random.default_rng(51).standard_normal(m.nv)
        y = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_A(h.handle, dev(r), y)
        assert rel_inf(host(y), P.apply_A(np.where(P.dir, 0.0, r))) <= 1e-12
        cgs.cgs_apply_preconditioner(h.handle, dev(r), y)
        assert rel_inf(host(y), P.apply_M(r, form)) <= (1e-11 if prec == "fp64" else 1e-5)
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), y, rtol=1e-8, maxit=4000)
        assert st == cgs.OK and rel[0] <= 1.5e-8
        if form not in c["its"]:
            _, c["its"][form], _, ok = P.solve(b, rtol=1e-8, maxit=4000, form=form)
            assert ok
        # FP64 within one iteration of the oracle; the float32 bulk over the
        # ~200 iterations this Neumann-dominated problem needs within 2%
        assert abs(int(its[0]) - c["its"][form]) <= (1 if prec == "fp64" else max(1, c["its"][form] // 50))
        bb = np.where(P.dir, 0.0, b)
        assert np.linalg.norm(bb - P.apply_A(host(y))) <= 1.5e-8 * np.linalg.norm(bb)


# ---------------------------------------------------------------------------
# restricted additive Schwarz (Sec. 3, R~_p without the grown part)
# ---------------------------------------------------------------------------

_problems = {}


def problem(name):
    if name not in _problems:
        m, b = {"cube32": meshes.workload_cube32, "cyl2": lambda: meshes.workload_cylinder(scale=2),
                "cube8": meshes.workload_cube8}[name]()
        _problems[name] = (m, b, O.Problem(m.xyz, m.conn, m.part, m.boxes), {})
    return _problems[name]


TOL_M = {"fp64": 1e-11, "fp32": 1e-5, "fp16": 2e-3}


@pytest.mark.parametrize("name", ["cube32", "cyl2"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_ras_preconditioner_and_solve(ctx, name, prec):
    """M r with the restricted prolongation against the oracle; cube32 uses
    warp kernels (FP64) or row packs, the halved cylinder lane packs in every
    precision.  The flexible PCG with the (nonsymmetric) RAS M follows the
    oracle's iteration count within one."""
    m, b, P, its_cache = problem(name)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form="ras") as h:
        r = np.random.default_rng(61).standard_normal(m.nv)
        z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
        assert rel_inf(host(z), P.apply_M(r, "ras")) <= TOL_M[prec]
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), z, rtol=1e-8, maxit=2000)
        assert st == cgs.OK and rel[0] <= 1.5e-8
        if "ras" not in its_cache:
            _, its_cache["ras"], _, ok = P.solve(b, rtol=1e-8, maxit=2000, form="ras")
            assert ok
        assert abs(int(its[0]) - its_cache["ras"]) <= 1


def test_ras_form_switch(ctx):
    """A mesh set up hybrid switches to RAS (the weights are always set up)."""
    m, b, P, _ = problem("cube8")
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes) as h:
        cgs.cgs_mesh_set_form(h.handle, "ras")
        r = np.random.default_rng(62).standard_normal(m.nv)
        z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
        assert rel_inf(host(z), P.apply_M(r, "ras")) <= 1e-11


# ---------------------------------------------------------------------------
# inexact local solves (Sec. 6): k CG steps on each A_p
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,prec,tol", [("cube32", "fp64", 1e-11), ("cyl2", "fp64", 1e-10),
                                           ("cube32", "fp32", 1e-4)])
@pytest.mark.parametrize("k", [2, 6])
def test_inexact_local_solves(ctx, name, prec, tol, k):
    """cgs_apply_local and M r (hybrid) with k inner CG steps against the
    oracle's batched CG from zero; the flexible PCG around the nonlinear M
    follows the oracle's iteration count within one (FP64, cube32)."""
    m, b, P, its_cache = problem(name)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, local_cg_steps=k) as h:
        r = np.where(P.dir, 0.0, np.random.default_rng(63).standard_normal(m.nv))
        out = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_local(h.handle, dev(r), out, True)
        assert rel_inf(host(out), P.local_solves(r, True, inner=k)) <= tol
        cgs.cgs_apply_preconditioner(h.handle, dev(r), out)
        assert rel_inf(host(out), P.apply_M(r, "hybrid", inner=k)) <= tol
        if prec == "fp64" and name == "cube32":
            st, its, rel = cgs.cgs_solve(h.handle, dev(b), out, rtol=1e-8, maxit=3000)
            assert st == cgs.OK and rel[0] <= 1.5e-8
            key = ("inexact", k)
            if key not in its_cache:
                _, its_cache[key], _, ok = P.solve(b, rtol=1e-8, maxit=3000, inner=k)
                assert ok
            assert abs(int(its[0]) - its_cache[key]) <= 1


def test_inexact_rejects_fp16_and_large_subdomains(ctx):
    m, b, P, _ = problem("cube8")
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, None, m.part, m.boxes, prec="fp16", local_cg_steps=2)
    assert ei.value.status == cgs.ERR_INVALID_ARG
    # one subdomain of 343 dofs: CG needs m_p <= 64
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, None, np.zeros(m.ne, np.int32), m.boxes, local_cg_steps=2)
    assert ei.value.status == cgs.ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# outer iterations around the preconditioner: Schwarz-Richardson and
# flexible GMRES (the paper's wrappers)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["richardson", "fgmres"])
@pytest.mark.parametrize("name,prec,form,inner", [("cube8", "fp64", "hybrid", 0), ("cube32", "fp64", "hybrid", 0),
                                                  ("cube32", "fp32", "hybrid", 0), ("cube32", "fp64", "ras", 0),
                                                  ("cube32", "fp64", "hybrid", 3)])
def test_wrapped_solvers_follow_the_oracle(ctx, method, name, prec, form, inner):
    """cgs_solve_wrapped against the oracle's richardson / fgmres with the same
    preconditioner: iterations within one, the true residual at the tolerance,
    and the solutions close (both stop at relres 1e-8)."""
    if method == "richardson" and (inner or form != "hybrid"):
        # undamped Richardson needs rho(I - M A) < 1, which the hybrid step
        # gives (pinned densely in the oracle tests); the additive-type RAS
        # sum does not, and a nonlinear M is no fixed-point iteration
        pytest.skip("Richardson is run with the hybrid, exact preconditioner")
    m, b, P, its_cache = problem(name)
    bb = np.where(P.dir, 0.0, b)
    key = (method, form, inner)
    if key not in its_cache:
        Mo = lambda r: P.apply_M(r, form, inner)
        if method == "richardson":
            its_cache[key] = O.richardson(P.apply_A, Mo, bb, 1e-8, 2000)
        else:
            its_cache[key] = O.fgmres(P.apply_A, Mo, bb, 1e-8, 2000, restart=30)
    xo, its_o, rel_o, ok = its_cache[key]
    assert ok
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form,
                  local_cg_steps=inner) as h:
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, its, rel = cgs.cgs_solve_wrapped(h.handle, dev(b), x, method, rtol=1e-8, maxit=2000, restart=30)
        assert st == cgs.OK and rel <= 1e-8
        assert abs(its - its_o) <= 1
        xg = host(x)
        assert np.linalg.norm(bb - P.apply_A(xg)) <= 1.5e-8 * np.linalg.norm(bb)
        assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


def test_wrapped_solver_arguments(ctx):
    m, b, P, _ = problem("cube8")
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes) as h:
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_solve_wrapped(h.handle, dev(b), x, "fgmres", restart=0)
        assert ei.value.status == cgs.ERR_INVALID_ARG
        st, its, rel = cgs.cgs_solve_wrapped(h.handle, dev(b), x, "fgmres", rtol=1e-14, maxit=3)
        assert st == cgs.ERR_NO_CONVERGENCE and its == 3
        st, its, rel = cgs.cgs_solve_wrapped(h.handle, dev(np.zeros(m.nv)), x, "richardson")
        assert st == cgs.OK and its == 0 and not host(x).any()
        st, its, rel = cgs.cgs_solve_wrapped(h.handle, dev(b), x, "pcg", rtol=1e-10)
        _, its_o, _, _ = P.solve(b, rtol=1e-10)
        assert st == cgs.OK and abs(its - its_o) <= 1
