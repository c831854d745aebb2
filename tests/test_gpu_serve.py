"""Serving by continuous batching: requests that arrive while others run join
free slots and share their launches; each result must equal the solo solve
of the same mesh and right-hand side within the solve tolerance, and the FP64
oracle's solve (iterations within one, relative solution difference <= 1e-8
at rtol 1e-10)."""
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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_results_same_alone_and_in_the_mix(ctx, prec):
    mesh_defs = [meshes.cube(10, perturb=0.15, seed=1), meshes.cube(16, deform=True, permute_seed=3),
                 meshes.cylinder(6, 24, 8, grading=1.1, aspect=5.0, boxes=(3, 3, 3)),
                 meshes.cube((7, 9, 5), perturb=0.1, seed=4, part_mode="mixed")]
    hs = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) for m in mesh_defs]
    oracles = [O.Problem(m.xyz, m.conn, m.part, m.boxes) for m in mesh_defs]
    rtol = 1e-10
    server = cgs.cgs_server_create(ctx, max_slots=3, pool_nv=3 * max(m.nv for m in mesh_defs),
                                   pool_nr=3 * max(h.info["n_r"] for h in hs), prec=prec, rtol=rtol)
    try:
        rng = np.random.default_rng(0)
        reqs = []   # (mesh index, b, x, ticket)
        pending = []
        # arrivals over several steps: 3 slots for 10 requests, so some queue
        schedule = [2, 0, 3, 1, 0, 4, 0, 0]
        k = 0
        for step, n_new in enumerate(schedule + [0] * 60):
            for _ in range(n_new):
                mi = k % len(hs)
                b = dev(rng.standard_normal(mesh_defs[mi].nv))
                x = torch.zeros_like(b)
                t = cgs.cgs_submit(server, hs[mi], b, x)
                reqs.append([mi, b, x, t, None])
                pending.append(len(reqs) - 1)
                k += 1
            active, queued, finished = cgs.cgs_server_step(server, iterations=3)
            assert active <= 3
            for i in list(pending):
                r = cgs.cgs_poll(server, reqs[i][3])
                if r is not None:
                    reqs[i][4] = r
                    pending.remove(i)
            if not pending and step >= len(schedule):
                break
        assert not pending and len(reqs) == 10
        for mi, b, x, t, (its, rel, st) in reqs:
            assert st == cgs.OK and rel <= rtol * 1.01
            x1 = torch.empty_like(x)
            st1, its1, rel1 = cgs.cgs_solve(hs[mi].handle, b, x1, rtol=rtol)
            assert abs(int(its1[0]) - its) <= 1
            xa, xb = x1.cpu().numpy(), x.cpu().numpy()
            assert np.linalg.norm(xb - xa) / np.linalg.norm(xa) <= 1e-8
            # against the oracle's solve of the same request
            xo, its_o, _, ok = oracles[mi].solve(b.cpu().numpy(), rtol=rtol)
            assert ok and abs(its_o - its) <= 1
            assert np.linalg.norm(xb - xo) / np.linalg.norm(xo) <= 1e-8
    finally:
        cgs.cgs_server_free(server)
        for h in hs:
            h.free()


def test_request_larger_than_the_arena_is_refused(ctx):
    small = meshes.cube(6, perturb=0.1, seed=2)
    big = meshes.cube(12, perturb=0.1, seed=3)
    hs, hb = (cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") for m in (small, big))
    server = cgs.cgs_server_create(ctx, max_slots=2, pool_nv=small.nv, pool_nr=hs.info["n_r"], prec="fp32")
    try:
        b = dev(np.ones(big.nv))
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_submit(server, hb, b, torch.zeros_like(b))
        assert ei.value.status == cgs.ERR_ADMISSION
        b = dev(np.zeros(small.nv))
        t = cgs.cgs_submit(server, hs, b, torch.zeros_like(b))
        cgs.cgs_server_step(server, iterations=1)
        assert cgs.cgs_poll(server, t) == (0, 0.0, cgs.OK)
    finally:
        cgs.cgs_server_free(server)
        hs.free()
        hb.free()


def test_admission_by_footprint(ctx):
    """Four free slots but an arena for two requests: two run, two wait for
    arena space, in arrival order; every result still equals its solo solve."""
    m = meshes.cube(12, perturb=0.1, seed=5)
    small = meshes.cube(5, perturb=0.1, seed=6)
    h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32")
    hsm = cgs.Mesh(ctx, small.xyz, small.conn, part=small.part, boxes=small.boxes, prec="fp32")
    oracle_of = {id(h): O.Problem(m.xyz, m.conn, m.part, m.boxes),
                 id(hsm): O.Problem(small.xyz, small.conn, small.part, small.boxes)}
    pool_nv = 2 * ((m.nv + 31) // 32 * 32)
    server = cgs.cgs_server_create(ctx, max_slots=4, pool_nv=pool_nv, pool_nr=2 * h.info["n_r"], prec="fp32",
                                   rtol=1e-10)
    try:
        fp = cgs.cgs_server_footprint(server, h)
        st0 = cgs.cgs_server_stats(server)
        assert fp >= 48 * m.nv and st0["bytes_in_use"] == 0 and st0["arena_bytes"] >= 2 * fp
        rng = np.random.default_rng(7)
        reqs = []
        for i in range(4):
            mm, hh = (m, h) if i < 3 else (small, hsm)
            b = dev(rng.standard_normal(mm.nv))
            x = torch.zeros_like(b)
            reqs.append((hh, b, x, cgs.cgs_submit(server, hh, b, x)))
        active, queued, finished = cgs.cgs_server_step(server, iterations=1)
        st1 = cgs.cgs_server_stats(server)
        # the small request fits beside the two but may not overtake the third
        assert (active, queued, finished) == (2, 2, 0)
        assert st1["bytes_in_use"] == 2 * fp and st1["active"] == 2 and st1["queued"] == 2
        results = {}
        for _ in range(400):
            cgs.cgs_server_step(server, iterations=4)
            for hh, b, x, t in reqs:
                if t not in results:
                    r = cgs.cgs_poll(server, t)
                    if r is not None:
                        results[t] = r
            if len(results) == 4:
                break
        assert len(results) == 4
        assert cgs.cgs_server_stats(server)["bytes_in_use"] == 0
        for hh, b, x, t in reqs:
            its, rel, st = results[t]
            assert st == cgs.OK and rel <= 1e-10 * 1.01
            x1 = torch.empty_like(x)
            cgs.cgs_solve(hh.handle, b, x1, rtol=1e-10)
            xa, xb = x1.cpu().numpy(), x.cpu().numpy()
            assert np.linalg.norm(xb - xa) / np.linalg.norm(xa) <= 1e-8
            # against the oracle's solve of the same request
            P = oracle_of[id(hh)]
            xo, its_o, _, ok = P.solve(b.cpu().numpy(), rtol=1e-10)
            assert ok and abs(its_o - its) <= 1
            assert np.linalg.norm(xb - xo) / np.linalg.norm(xo) <= 1e-8
    finally:
        cgs.cgs_server_free(server)
        h.free()
        hsm.free()


def test_drain_returns_each_finished_request_once(ctx):
    m = meshes.cube(9, perturb=0.1, seed=8)
    h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32")
    server = cgs.cgs_server_create(ctx, max_slots=2, pool_nv=4 * m.nv, pool_nr=4 * h.info["n_r"], prec="fp32",
                                   rtol=1e-9)
    try:
        rng = np.random.default_rng(9)
        bs = [dev(rng.standard_normal(m.nv)) for _ in range(5)]
        xs = [torch.zeros_like(b) for b in bs]
        tickets = [cgs.cgs_submit(server, h, b, x) for b, x in zip(bs, xs)]
        got = {}
        for _ in range(300):
            cgs.cgs_server_step(server, iterations=2)
            for t, its, rel, st in cgs.cgs_server_drain(server):
                assert t not in got
                got[t] = (its, rel, st)
            if len(got) == len(tickets):
                break
        assert sorted(got) == sorted(tickets)
        assert all(st == cgs.OK and rel <= 1e-9 * 1.01 and its > 0 for its, rel, st in got.values())
        assert cgs.cgs_server_drain(server) == []
        with pytest.raises(cgs.CGSError):
            cgs.cgs_poll(server, tickets[0])   # released by the drain
    finally:
        cgs.cgs_server_free(server)
        h.free()
