"""The interpolation over cell-sorted (vertex, cell, weight) entries (one warp
per cell range, atomic adds into z, the PCG dots in their own kernel) against
the FP64 oracle and against the per-vertex interpolation with fused dots.

The entries are the per-vertex box lists of W Q^T J_L regrouped by cell, so
the sum is the same; only the order in which the cells of a vertex on a cell
boundary add into z differs (one rounding per add).  Thresholds: the box
steps and M r as in the per-vertex parity tests (1e-12 and 1e-11 relative
max norm, FP64 form; 1e-5 for FP32 bulk); solves at rtol 1e-10 take the same
iteration count within one and agree to 1e-8 in the relative 2-norm.
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


def by_cells(h, on):
    cgs.cgs_mesh_set_schedule(h.handle, interp_cells=1 if on else 0)
    assert cgs.cgs_mesh_get_schedule(h.handle)["interp_cells"] == (1 if on else 0)


@pytest.mark.parametrize("name", list(CASES))
def test_interp_by_cells_against_oracle(ctx, name):
    m, b, P = problem(name)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64") as h:
        by_cells(h, True)
        u = np.random.default_rng(5).standard_normal(P.nr)
        z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_interp(h.handle, dev(u), z)
        assert rel_inf(host(z), P.interp(u)) <= 1e-12
        r = np.random.default_rng(6).standard_normal(m.nv)
        cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
        assert rel_inf(host(z), P.apply_M(r, "hybrid")) <= 1e-11


@pytest.mark.parametrize("form", ["hybrid", "additive"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_preconditioner_by_cells(ctx, form, prec):
    m, b, P = problem("mixed")
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form) as h:
        by_cells(h, True)
        r = np.random.default_rng(4).standard_normal(m.nv)
        z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_preconditioner(h.handle, dev(r), z)
        assert rel_inf(host(z), P.apply_M(r, form)) <= (1e-11 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_solve_by_cells_matches_by_vertex(ctx, name, prec, form):
    m, b, _ = problem(name)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form) as h:
        x0 = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        x1 = torch.empty_like(x0)
        by_cells(h, False)
        st0, it0, rel0 = cgs.cgs_solve(h.handle, dev(b), x0, rtol=1e-10)
        by_cells(h, True)
        st1, it1, rel1 = cgs.cgs_solve(h.handle, dev(b), x1, rtol=1e-10)
        assert st0 == cgs.OK and st1 == cgs.OK
        assert abs(int(it0[0]) - int(it1[0])) <= 1 and rel1[0] <= 1e-10
        a, c = host(x0), host(x1)
        assert np.linalg.norm(a - c) / np.linalg.norm(a) <= 1e-8
        # maxit is honoured by the loop condition the dots kernel now sets
        st2, it2, _ = cgs.cgs_solve(h.handle, dev(b), x1, rtol=1e-14, maxit=3)
        assert st2 == cgs.ERR_NO_CONVERGENCE and int(it2[0]) == 3
