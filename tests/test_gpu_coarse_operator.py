"""The full-support coarse operators (Sec. 4) on the GPU: the Galerkin
A_r = J~^T A J~ with the averaged interpolant, and the vertex-based J (each
node interpolated in the box cell holding it) with A_r = J^T A J, against
the FP64 oracle built with the same operator.

Thresholds as in the per-step parity tests: r_r, u_r and z = J u_r to 1e-12
(relative max norm, FP64 form), M r to 1e-11 (1e-5 for FP32 bulk); solves at
rtol 1e-8 take the oracle's iteration count within one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402

ORACLE_OP = {"galerkin": "galerkin", "vertex": "vertex"}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


_cache = {}


def problem(name, op):
    key = (name, op)
    if key not in _cache:
        if name == "cube8":
            m, b = meshes.workload_cube8()
        else:
            m, b = meshes.cube(11, perturb=0.15, seed=[2, 7], part_mode="mixed", name="mixed"), meshes.rhs(12 ** 3, 10)
        _cache[key] = (m, b, O.Problem(m.xyz, m.conn, m.part, m.boxes, coarse_operator=ORACLE_OP[op]))
    return _cache[key]


@pytest.mark.parametrize("op", ["galerkin", "vertex"])
@pytest.mark.parametrize("name", ["cube8", "mixed"])
def test_box_steps_and_preconditioner(ctx, op, name):
    m, b, P = problem(name, op)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64", coarse_operator=op) as h:
        info = cgs.cgs_mesh_info(h.handle)
        assert info["n_r"] == P.nr and info["coarse_operator"] == cgs.COARSE_OP[op]
        assert info["ar_nnz"] == int(np.count_nonzero(P.Ar))
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
        r = rng.standard_normal(m.nv)
        cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
        assert rel_inf(host(z), P.apply_M(r, "hybrid")) <= 1e-11


@pytest.mark.parametrize("op", ["galerkin", "vertex"])
@pytest.mark.parametrize("prec,coarse", [("fp64", "dense"), ("fp32", "xxt"), ("fp32", "dense")])
def test_solve_matches_oracle_iterations(ctx, op, prec, coarse):
    m, b, P = problem("mixed", op)
    _, it_ref, _, _ = P.solve(b, rtol=1e-8)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, coarse=coarse,
                  coarse_operator=op) as h:
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, it, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8)
        assert st == cgs.OK and rel[0] <= 1e-8 and abs(int(it[0]) - it_ref) <= 1
        if prec == "fp32":
            r = np.random.default_rng(4).standard_normal(m.nv)
            z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
            cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
            assert rel_inf(host(z), P.apply_M(r, "hybrid")) <= 1e-5


def test_bad_operator_rejected(ctx):
    m, _ = meshes.workload_cube8()
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, None, m.part, m.boxes, 0.0, 1, "fp64", "hybrid", "auto", 5)
    assert ei.value.status == cgs.ERR_INVALID_ARG
