"""The no-allocation preconditioner entry point against the regular one.

cgs_apply_preconditioner_noalloc serves callers that cannot allocate device
memory when they call (serving loops that forbid allocation after warm-up,
hosts whose device memory belongs to another runtime's pool).  It keeps its
working vectors in a static device array, so these tests check that it
returns what cgs_apply_preconditioner returns, call after call, and that it
refuses meshes beyond either of its size limits (vertices, reduced unknowns).
This file is collected last so a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_20496_b300 import cgs, meshes  # noqa: E402


def _rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


# The same tolerances as the preconditioner parity tests: FP64 results agree to
# 1e-11; the FP32/FP16 forms sum with float atomics whose order changes from
# launch to launch, so two launches of either entry differ by a few float
# ulps and the bar is the FP32 tolerance 1e-5.
TOL = {"fp64": 1e-11, "fp32": 1e-5, "fp16": 1e-5}


@pytest.mark.parametrize("prec,form,coarse", [("fp64", "hybrid", "auto"), ("fp64", "additive", "auto"),
                                              ("fp32", "hybrid", "auto"), ("fp16", "hybrid", "auto"),
                                              ("fp64", "hybrid", "xxt"), ("fp32", "additive", "xxt")])
def test_noalloc_matches_regular_preconditioner_twice(ctx, prec, form, coarse):
    m, _ = meshes.workload_cube32()
    rng = np.random.default_rng(21)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form, coarse=coarse) as h:
        for call in range(2):       # two calls in a row: the shared array keeps old contents
            r = torch.as_tensor(rng.standard_normal(m.nv), dtype=torch.float64, device="cuda")
            z_ref = torch.empty_like(r)
            z_new = torch.full_like(r, np.nan)
            cgs.cgs_apply_preconditioner(h.handle, r, z_ref)
            cgs.cgs_apply_preconditioner_noalloc(h.handle, r, z_new)
            torch.cuda.synchronize()
            a, b = z_new.cpu().numpy(), z_ref.cpu().numpy()
            assert np.isfinite(a).all()
            assert _rel_inf(a, b) <= TOL[prec], (call, _rel_inf(a, b))


@pytest.mark.parametrize("prec,form", [("fp32", "hybrid"), ("fp32", "additive"), ("fp16", "additive")])
def test_noalloc_with_subdomains_of_up_to_64_dofs(ctx, prec, form):
    """3- and 2-element segments: packs of the classes above 32 dofs, which
    the additive form's fused local-solve-and-restriction launch does not
    take (the entry point falls back to separate launches)."""
    m = meshes.cube(13, perturb=0.15, seed=[2, 13], part_mode="mixed", name="cube13_mixed")
    rng = np.random.default_rng(22)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form) as h:
        assert h.info["max_sub_dofs"] > 32
        for call in range(2):
            r = torch.as_tensor(rng.standard_normal(m.nv), dtype=torch.float64, device="cuda")
            z_ref = torch.empty_like(r)
            z_new = torch.full_like(r, np.nan)
            cgs.cgs_apply_preconditioner(h.handle, r, z_ref)
            cgs.cgs_apply_preconditioner_noalloc(h.handle, r, z_new)
            torch.cuda.synchronize()
            a, b = z_new.cpu().numpy(), z_ref.cpu().numpy()
            assert np.isfinite(a).all() and np.abs(b).max() > 0
            assert _rel_inf(a, b) <= TOL[prec], (call, _rel_inf(a, b))


def test_noalloc_rejects_meshes_beyond_its_limit(ctx):
    m, _ = meshes.workload_cylinder(scale=2)        # 137,280 vertices > the 131,072 limit
    assert m.nv > cgs.NOALLOC_MAX_NV
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        r = torch.zeros(m.nv, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_apply_preconditioner_noalloc(h.handle, r, z)
        assert ei.value.status == cgs.ERR_INVALID_ARG
        assert "limit" in cgs.load().cgs_last_error().decode()


def test_noalloc_rejects_reduced_spaces_beyond_its_limit(ctx):
    # 40 x 40 x 4 box cells over a 48 x 48 x 6 slab: every cell holds element
    # centroids, so all 41 * 41 * 5 = 8,405 box vertices are active (> 8,192)
    # while the mesh itself (16,807 vertices) is within the vertex limit
    m = meshes.cube((48, 48, 6), perturb=0.1, seed=5, boxes=(40, 40, 4))
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        assert h.info["n_r"] > cgs.NOALLOC_MAX_NR and m.nv <= cgs.NOALLOC_MAX_NV
        r = torch.zeros(m.nv, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_apply_preconditioner_noalloc(h.handle, r, z)
        assert ei.value.status == cgs.ERR_INVALID_ARG
        assert "n_r" in cgs.load().cgs_last_error().decode()
