"""Batches: many meshes and right-hand sides solved by the same launches.

Each slot of a batch must give what the single-mesh solve gives for the same
mesh and right-hand side (same iteration count within one, solutions within
the solve tolerance), stop on its own (a zero right-hand side takes no
iteration while the others run), and report its own status.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


def _meshes(n=6, seed=2):
    sizes = np.random.default_rng(seed).integers(4, 10, n)
    return [meshes.cube(int(k), perturb=0.15, seed=[seed, i], part_mode="mixed") for i, k in enumerate(sizes)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_batch_matches_single_solves(ctx, prec, nrhs):
    ms = _meshes()
    hs = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) for m in ms]
    try:
        bs, xs = [], []
        for i, m in enumerate(ms):
            B = meshes.rhs(m.nv, [7, i], count=nrhs)
            for r in range(nrhs):
                bs.append(dev(B[r]))
                xs.append(torch.empty(m.nv, dtype=torch.float64, device="cuda"))
        batch = cgs.cgs_batch_create(ctx, hs, nrhs)
        try:
            st, its, rel, sts = cgs.cgs_batch_solve(batch, bs, xs, rtol=1e-10)
            assert st == cgs.OK and np.all(sts == cgs.OK)
            assert np.all(rel <= 1e-10)
            for s in range(len(bs)):
                h = hs[s // nrhs]
                x1 = torch.empty_like(xs[s])
                st1, its1, rel1 = cgs.cgs_solve(h.handle, bs[s], x1, rtol=1e-10)
                assert abs(int(its1[0]) - int(its[s])) <= 1
                xb, xa = xs[s].cpu().numpy(), x1.cpu().numpy()
                assert np.linalg.norm(xb - xa) / np.linalg.norm(xa) <= 1e-8
            # and against the oracle for the first slot of each mesh
            for i, m in enumerate(ms[:3]):
                P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
                xo, _, _, _ = P.solve(bs[i * nrhs].cpu().numpy(), rtol=1e-12)
                xb = xs[i * nrhs].cpu().numpy()
                assert np.linalg.norm(xb - xo) / np.linalg.norm(xo) <= 1e-8
            # a second solve on the same batch reuses its plan and graph
            st2, its2, rel2, _ = cgs.cgs_batch_solve(batch, bs, xs, rtol=1e-10)
            assert st2 == cgs.OK and list(its2) == list(its)
        finally:
            cgs.cgs_batch_free(batch)
    finally:
        for h in hs:
            h.free()


def test_batch_slots_stop_independently(ctx):
    ms = _meshes(3, seed=5)
    hs = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") for m in ms]
    try:
        bs = [dev(meshes.rhs(ms[0].nv, 1)), dev(np.zeros(ms[1].nv)), dev(meshes.rhs(ms[2].nv, 3))]
        xs = [torch.full((m.nv,), 5.0, dtype=torch.float64, device="cuda") for m in ms]
        batch = cgs.cgs_batch_create(ctx, hs, 1)
        try:
            st, its, rel, sts = cgs.cgs_batch_solve(batch, bs, xs, rtol=1e-9)
            assert st == cgs.OK and its[1] == 0 and its[0] > 0 and its[2] > 0
            assert not xs[1].cpu().numpy().any()
            st, its, rel, sts = cgs.cgs_batch_solve(batch, bs, xs, rtol=1e-14, maxit=2)
            assert st == cgs.ERR_NO_CONVERGENCE
            assert list(sts) == [cgs.ERR_NO_CONVERGENCE, cgs.OK, cgs.ERR_NO_CONVERGENCE]
            assert list(its) == [2, 0, 2]
        finally:
            cgs.cgs_batch_free(batch)
    finally:
        for h in hs:
            h.free()


def test_solve_batched_convenience(ctx):
    ms = _meshes(2, seed=9)
    hs = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp16") for m in ms]
    try:
        bs = [dev(meshes.rhs(m.nv, [3, i], count=2)[r]) for i, m in enumerate(ms) for r in range(2)]
        xs = [torch.empty_like(b) for b in bs]
        st, its, rel = cgs.cgs_solve_batched(hs, bs, xs, nrhs=2, rtol=1e-9)
        assert st == cgs.OK and np.all(rel <= 1e-9) and np.all(its > 0)
    finally:
        for h in hs:
            h.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotuner_keeps_results(ctx, prec):
    """The tuner only changes block sizes: the solve gives the same answer."""
    m, b = meshes.workload_cube32()
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) as h:
        x0 = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, its0, _ = cgs.cgs_solve(h.handle, dev(b), x0, rtol=1e-10)
        cgs.cgs_mesh_tune(h.handle)
        sch = cgs.cgs_mesh_get_schedule(h.handle)
        assert sch["vert_chunk"] in (256, 512, 1024, 2048) and sch["sub_chunk"] in (8, 16, 32, 64)
        assert sch["box_chunk"] in (256, 512, 1024) and sch["tile_tma"] in (0, 1)
        x1 = torch.empty_like(x0)
        st, its1, rel = cgs.cgs_solve(h.handle, dev(b), x1, rtol=1e-10)
        assert st == cgs.OK and abs(int(its1[0]) - int(its0[0])) <= 1
        a, c = x0.cpu().numpy(), x1.cpu().numpy()
        assert np.linalg.norm(a - c) / np.linalg.norm(a) <= 1e-8
