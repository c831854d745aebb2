"""Projection onto prior solutions for repeated right-hand sides (Sec. 5:
solve for the change from the A-orthogonal best fit onto l prior
solutions), through cgs_mesh_set_projection and cgs_solve, against the FP64
oracle's projected sequence (oracle.cgs_oracle.solve_projected) and exact
solutions.

Thresholds: every solution within 1e-8 (relative max norm) of the dense
direct solution at rtol 1e-10; iteration counts within one of the oracle's
projected sequence and never above the plain solve's; a right-hand side that
is a combination of earlier ones needs no iteration.
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


CASES = {
    "cube8": lambda: meshes.workload_cube8()[0],
    "mixed": lambda: meshes.cube(11, perturb=0.15, seed=[2, 7], part_mode="mixed", name="mixed"),
}
_cache = {}


def problem(name):
    if name not in _cache:
        m = CASES[name]()
        _cache[name] = (m, O.Problem(m.xyz, m.conn, m.part, m.boxes))
    return _cache[name]


def direct(P, b):
    x = np.zeros(P.nv)
    x[P.free] = np.linalg.solve(P.A.toarray(), np.where(P.dir, 0.0, b)[P.free])
    return x


def sequence(nv, n, seed=3):
    rng = np.random.default_rng(seed)
    b0, b1 = rng.standard_normal(nv), rng.standard_normal(nv)
    return [b0 + 0.05 * k * b1 for k in range(n)]


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_projected_sequence_against_oracle(ctx, name, prec):
    m, P = problem(name)
    bs = sequence(m.nv, 6)
    ref = O.solve_projected(P, bs, 3, rtol=1e-10)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) as h:
        plain = []
        for b in bs:
            x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
            st, it, _ = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-10)
            plain.append(int(it[0]))
        cgs.cgs_mesh_set_projection(h.handle, 3)
        its, sizes = [], []
        for b, (xr, itr, _, _, _) in zip(bs, ref):
            x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
            st, it, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-10)
            assert st == cgs.OK and rel[0] <= 5e-10
            exact = direct(P, b)
            assert np.abs(host(x) - exact).max() <= 1e-8 * np.abs(exact).max()
            assert abs(int(it[0]) - itr) <= 1
            its.append(int(it[0]))
            sizes.append(cgs.cgs_mesh_projection_size(h.handle))
        assert sizes == [r[4] for r in ref]           # restarts and skipped directions as in the oracle
        assert its[0] == plain[0] and all(a <= p for a, p in zip(its, plain)) and sum(its) < sum(plain)


def test_combination_of_prior_right_hand_sides_needs_no_iteration(ctx):
    m, P = problem("cube8")
    rng = np.random.default_rng(5)
    b1, b2 = rng.standard_normal(m.nv), rng.standard_normal(m.nv)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64") as h:
        cgs.cgs_mesh_set_projection(h.handle, 4)
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        for b in (b1, b2):
            cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-13)
        b = 0.3 * b1 - 1.7 * b2
        st, it, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8)
        assert st == cgs.OK and int(it[0]) == 0 and rel[0] <= 1e-8
        exact = direct(P, b)
        assert np.abs(host(x) - exact).max() <= 1e-9 * np.abs(exact).max()


def test_several_right_hand_sides_in_one_call_and_switching_off(ctx):
    m, P = problem("cube8")
    bs = sequence(m.nv, 4, seed=8)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        cgs.cgs_mesh_set_projection(h.handle, 8)
        B = dev(np.stack(bs))
        X = torch.empty_like(B)
        st, its, rel = cgs.cgs_solve(h.handle, B, X, nrhs=4, rtol=1e-10)
        # b_2, b_3 lie in the span of b_0, b_1: their solutions add no direction
        assert st == cgs.OK and np.all(rel <= 5e-10) and cgs.cgs_mesh_projection_size(h.handle) == 2
        assert its[2] < its[0] and its[3] < its[0]
        for k in range(4):
            exact = direct(P, bs[k])
            assert np.abs(host(X[k]) - exact).max() <= 1e-8 * np.abs(exact).max()
        cgs.cgs_mesh_set_projection(h.handle, 0)
        assert cgs.cgs_mesh_projection_size(h.handle) == 0
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, it, _ = cgs.cgs_solve(h.handle, dev(bs[3]), x, rtol=1e-10)
        assert int(it[0]) == int(its[0]) or int(it[0]) >= int(its[3])
        for bad in (-1, cgs.PROJECTION_MAX + 1):
            with pytest.raises(cgs.CGSError) as ei:
                cgs.cgs_mesh_set_projection(h.handle, bad)
            assert ei.value.status == cgs.ERR_INVALID_ARG
