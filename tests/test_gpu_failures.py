"""Failure detection, exercised without any GPU fault.

* Bounded device waits: the testing aid cgs_mesh_set_wait_limits sets the
  iteration limits of the element-tile TMA waits and of the persistent loop's
  grid barriers.  A limit of 0 makes each such wait give up at once (the block
  still waits, with its own limit, for the copy it started), so the timeout
  path runs: the solve returns CGS_ERR_TIMEOUT, single steps record it in the
  mesh's step status word, and the next call with the default limits works.
* Non-finite input: a NaN in b stops the iteration with CGS_ERR_BREAKDOWN.
* Set-up errors (bad indices, inverted elements, a singular reduced operator)
  are covered in test_gpu_parity.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402

ALLOW = (cgs.ERR_NO_CONVERGENCE, cgs.ERR_BREAKDOWN, cgs.ERR_TIMEOUT)


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


@pytest.fixture(scope="module")
def cube32():
    m, b = meshes.workload_cube32()
    return m, b, O.Problem(m.xyz, m.conn, m.part, m.boxes)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_tile_wait_expiry_stops_the_solve(ctx, cube32, prec):
    m, b, P = cube32
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) as h:
        cgs.cgs_mesh_set_schedule(h.handle, tile_tma=1, persistent=0)
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_mesh_set_wait_limits(h.handle, 0, 1 << 22)
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8, allow=ALLOW)
        assert st == cgs.ERR_TIMEOUT
        assert "wait" in cgs.load().cgs_last_error().decode()
        # the context is still usable: default limits, same mesh, converged solve
        cgs.cgs_mesh_set_wait_limits(h.handle)
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8)
        assert st == cgs.OK and rel[0] <= 1.5e-8
        _, its_o, _, _ = P.solve(b, rtol=1e-8)
        assert abs(int(its[0]) - its_o) <= 1


@pytest.mark.parametrize("call", ["preconditioner", "noalloc", "inner", "outer"])
def test_tile_wait_expiry_in_single_steps(ctx, cube32, call):
    m, b, P = cube32
    # set up additive, then switched to hybrid: the hybrid step then forms
    # s = r - A l with the (TMA-staged) inner apply, whose tile wait the
    # limit of 0 makes expire (a hybrid set-up restricts r and l directly,
    # with no wait in the preconditioner)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32", form="additive") as h:
        cgs.cgs_mesh_set_form(h.handle, "hybrid")
        cgs.cgs_mesh_set_schedule(h.handle, tile_tma=1)
        r = dev(np.random.default_rng(3).standard_normal(m.nv))
        z = torch.empty_like(r)

        def run():
            if call == "preconditioner":
                cgs.cgs_apply_preconditioner(h.handle, r, z)
            elif call == "noalloc":
                cgs.cgs_apply_preconditioner_noalloc(h.handle, r, z)
            else:
                cgs.cgs_apply_A_prec(h.handle, r, z, call)

        assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
        cgs.cgs_mesh_set_wait_limits(h.handle, 0, 1 << 22)
        run()
        assert cgs.cgs_mesh_step_status(h.handle) == cgs.ERR_TIMEOUT
        assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK     # the query resets the word
        cgs.cgs_mesh_set_wait_limits(h.handle)
        run()
        assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
        got = z.cpu().numpy()
        rn = r.cpu().numpy()
        if call in ("preconditioner", "noalloc"):
            assert rel_inf(got, P.apply_M(rn, "hybrid")) <= 1e-5
        else:
            assert rel_inf(got, P.apply_A(np.where(P.dir, 0.0, rn))) <= (1e-5 if call == "inner" else 1e-12)


def test_persistent_barrier_expiry_stops_the_solve(ctx, cube32):
    m, b, P = cube32
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32", coarse="dense") as h:
        cgs.cgs_mesh_set_schedule(h.handle, persistent=1, tile_tma=0)
        assert cgs.cgs_mesh_info(h.handle)["loop"] == 2
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_mesh_set_wait_limits(h.handle, 1 << 20, 0)
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8, allow=ALLOW)
        assert st == cgs.ERR_TIMEOUT
        cgs.cgs_mesh_set_wait_limits(h.handle)
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8)
        assert st == cgs.OK and rel[0] <= 1.5e-8


def test_wait_limits_reject_negative(ctx, cube32):
    m, b, P = cube32
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_mesh_set_wait_limits(h.handle, -1, 0)
        assert ei.value.status == cgs.ERR_INVALID_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nan_rhs_reports_breakdown(ctx, cube32, prec):
    m, b, P = cube32
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) as h:
        bad = b.copy()
        bad[int(P.free[len(P.free) // 2])] = np.nan
        x = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        st, its, rel = cgs.cgs_solve(h.handle, dev(bad), x, rtol=1e-8, allow=ALLOW)
        assert st == cgs.ERR_BREAKDOWN
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8)
        assert st == cgs.OK and rel[0] <= 1.5e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_non_spd_local_block_is_reported(ctx, prec):
    """A local matrix negated on the host (the set-up's testing aid) makes its
    inverse fail: CGS_ERR_NOT_SPD, and a normal set-up of the same mesh
    afterwards works."""
    m, _ = meshes.workload_cube8()
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, elem_part=m.part, boxes=m.boxes, prec=prec,
                           fault_negate_subdomain=5)
    assert ei.value.status == cgs.ERR_NOT_SPD
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, elem_part=m.part, boxes=m.boxes, prec=prec,
                           fault_negate_subdomain=-1)
    assert ei.value.status == cgs.ERR_INVALID_ARG
    h = cgs.cgs_mesh_setup(ctx, m.xyz, m.conn, elem_part=m.part, boxes=m.boxes, prec=prec)
    cgs.cgs_mesh_free(h)
