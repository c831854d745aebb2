"""The persistent PCG loop (one cooperative launch for all iterations, grid
barriers between the phases) against the one-launch-per-step path: same
iteration counts, same solutions to the solve tolerance, for single meshes,
batches and the server."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_20496_b300 import cgs, meshes  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


CASES = {
    "cube8": lambda: meshes.workload_cube8(),
    "mixed": lambda: (meshes.cube(11, perturb=0.15, seed=[2, 7], part_mode="mixed", name="mixed"),
                      meshes.rhs(12 ** 3, 10)),
    "cyl": lambda: meshes.workload_cylinder(scale=8),
    "nobox": lambda: (meshes.cube(6, perturb=0.1, seed=4, boxes=(1, 1, 1)), meshes.rhs(7 ** 3, 3)),
}


def set_persistent(h, on):
    cgs.cgs_mesh_set_schedule(h.handle, persistent=1 if on else 0)
    assert cgs.cgs_mesh_info(h.handle)["loop"] == (2 if on else 1)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_persistent_matches_stepwise(ctx, name, prec, form):
    m, b = CASES[name]()
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form) as h:
        x0 = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        x1 = torch.empty_like(x0)
        set_persistent(h, False)
        st0, it0, rel0 = cgs.cgs_solve(h.handle, dev(b), x0, rtol=1e-10)
        set_persistent(h, True)
        st1, it1, rel1 = cgs.cgs_solve(h.handle, dev(b), x1, rtol=1e-10)
        assert st0 == cgs.OK and st1 == cgs.OK
        assert abs(int(it0[0]) - int(it1[0])) <= 1 and rel1[0] <= 1e-10
        a, c = x0.cpu().numpy(), x1.cpu().numpy()
        assert np.linalg.norm(a - c) / np.linalg.norm(a) <= 1e-8
        # maxit is honoured inside the loop
        st2, it2, _ = cgs.cgs_solve(h.handle, dev(b), x1, rtol=1e-14, maxit=3)
        assert st2 == cgs.ERR_NO_CONVERGENCE and int(it2[0]) == 3


def test_persistent_batch_and_server(ctx):
    work = meshes.workload_batch(12, seed=5)
    hs = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") for m, _ in work]
    try:
        bs = [dev(B[0]) for _, B in work]
        xs = [torch.empty_like(bb) for bb in bs]
        batch = cgs.cgs_batch_create(ctx, hs, 1)
        try:
            st, its, rel, sts = cgs.cgs_batch_solve(batch, bs, xs, rtol=1e-9)
            assert st == cgs.OK and np.all(rel <= 1e-9 * 1.01)
        finally:
            cgs.cgs_batch_free(batch)
        for h, bb, xx, k in zip(hs, bs, xs, its):
            x1 = torch.empty_like(bb)
            st1, it1, _ = cgs.cgs_solve(h.handle, bb, x1, rtol=1e-9)
            assert abs(int(it1[0]) - int(k)) <= 1
            a, c = x1.cpu().numpy(), xx.cpu().numpy()
            assert np.linalg.norm(a - c) / np.linalg.norm(a) <= 1e-7
        server = cgs.cgs_server_create(ctx, 4, 4 * max(m.nv for m, _ in work), 4 * max(h.info["n_r"] for h in hs),
                                       prec="fp32", rtol=1e-9)
        try:
            tickets = [cgs.cgs_submit(server, h, bb, xx) for h, bb, xx in zip(hs, bs, xs)]
            res = {}
            for _ in range(500):
                cgs.cgs_server_step(server, iterations=3)
                for t in tickets:
                    if t not in res:
                        r = cgs.cgs_poll(server, t)
                        if r is not None:
                            res[t] = r
                if len(res) == len(tickets):
                    break
            assert len(res) == len(tickets)
            assert all(r[2] == cgs.OK and r[1] <= 1e-9 * 1.01 for r in res.values())
        finally:
            cgs.cgs_server_free(server)
    finally:
        for h in hs:
            h.free()


def test_schedule_round_trip_and_pdl_off(ctx):
    """Every schedule field is settable, invalid values are refused, and
    ordinary launches (pdl = 0) give the same solve as programmatic ones."""
    m, b = meshes.workload_cube8()
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        x0 = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        x1 = torch.empty_like(x0)
        st0, it0, _ = cgs.cgs_solve(h.handle, dev(b), x0, rtol=1e-10)
        cgs.cgs_mesh_set_schedule(h.handle, vert_chunk=512, sub_chunk=16, pack_chunk=16, box_chunk=512, pdl=0)
        sch = cgs.cgs_mesh_get_schedule(h.handle)
        assert (sch["vert_chunk"], sch["sub_chunk"], sch["pack_chunk"], sch["box_chunk"], sch["pdl"]) == \
            (512, 16, 16, 512, 0)
        st1, it1, _ = cgs.cgs_solve(h.handle, dev(b), x1, rtol=1e-10)
        assert st0 == st1 == cgs.OK and int(it0[0]) == int(it1[0])
        assert np.array_equal(x0.cpu().numpy(), x1.cpu().numpy()) or \
            np.linalg.norm(x0.cpu().numpy() - x1.cpu().numpy()) <= 1e-8 * np.linalg.norm(x0.cpu().numpy())
        for bad in ({"vert_chunk": 300}, {"sub_chunk": 4}, {"pack_chunk": 7}, {"box_chunk": 100},
                    {"tile_tma": 2}, {"persistent": 5}, {"pdl": -1}, {"row_packs": 3}, {"interp_cells": 2}):
            with pytest.raises(cgs.CGSError) as ei:
                cgs.cgs_mesh_set_schedule(h.handle, **bad)
            assert ei.value.status == cgs.ERR_INVALID_ARG
        assert cgs.cgs_mesh_get_schedule(h.handle)["pdl"] == 0
