"""Parity of every kernel variant a schedule can select, against the FP64 oracle.

The mixed forms (FP32 bulk, FP16 local) pick among kernel variants by the
mesh's schedule: lane packs (one lane per subdomain) or row packs (four lanes
per subdomain) for the local solves, TMA-staged or thread-streamed element
tiles for both operator applies, interpolation by vertex (dots fused) or by
cell-sorted entries, and one launch per phase or the persistent loop.  Each
variant is forced here and compared with the oracle on three meshes: cube32
(4,096 subdomains: row packs by default), the halved hollow cylinder
(137,280 vertices, 16,384 subdomains: lane packs by default, the layout the
full-size cylinder runs) and a perturbed 13^3 cube cut into 3- and
2-element segments (125 subdomains of 27 to 64 dofs: the size classes above
32 dofs, which run in kernels of their own).

Bars, as for the default schedule (Sec. 3 Eq. (4) for the local solves,
Eqs. (3) and (5) for M r, flexible PCG around them):
  local solves   every entry within the float bound gamma_{m+12} W sum_p
                 |A_p^{-1}||R_p r| (plus 2 u16 and the subnormal term in FP16)
  M r            relative max-norm difference <= 1e-5 (FP32) or 2e-3 (FP16)
  solve          rtol 1e-8: iterations within one of the oracle's, true
                 residual <= 1.5e-8 checked with the oracle's operator
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402

U32, U16 = 2.0 ** -24, 2.0 ** -11
MESHES = {"cube32": meshes.workload_cube32, "cyl2": lambda: meshes.workload_cylinder(scale=2),
          # 3- and 2-element segments: subdomains of 27 to 64 dofs, the
          # larger classes (40, 48, 64) in packs of their own
          "cube13_mixed": lambda: (lambda m: (m, meshes.rhs(m.nv, 13)))(
              meshes.cube(13, perturb=0.15, seed=[2, 13], part_mode="mixed", name="cube13_mixed"))}
# schedule fields forced by each variant (the rest keep the set-up defaults)
VARIANTS = {
    "lane_packs": dict(row_packs=0),
    "row_packs": dict(row_packs=1),
    "tile_tma": dict(tile_tma=1),
    "tile_stream": dict(tile_tma=0),
    "interp_cells": dict(interp_cells=1),
    "interp_vertex": dict(interp_cells=0),
}
SOLVE_VARIANTS = dict(VARIANTS, persistent=dict(persistent=1))


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


_oracle = {}


def oracle(name):
    """The oracle's problem and its results for one seeded r (cached)."""
    if name not in _oracle:
        m, b = MESHES[name]()
        P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
        r = np.where(P.dir, 0.0, np.random.default_rng(31).standard_normal(m.nv))
        _oracle[name] = {"m": m, "b": b, "P": P, "r": r, "local": P.local_solves(r, True),
                         "M_hybrid": P.apply_M(r, "hybrid"), "M_additive": P.apply_M(r, "additive"),
                         "bound": _abs_local_bound(P, r), "solve": None,
                         "inv_max": max(abs(np.linalg.inv(Ap)).max() for (_, _, Ap, _) in P.groups.values())}
    return _oracle[name]


def oracle_iters(name):
    o = oracle(name)
    if o["solve"] is None:
        _, its, _, ok = o["P"].solve(o["b"], rtol=1e-8, maxit=1000)
        assert ok
        o["solve"] = its
    return o["solve"]


def _abs_local_bound(P, r):
    out = np.zeros(P.nv)
    for mm, (ps, I, Ap, L) in P.groups.items():
        inv = np.abs(np.linalg.inv(Ap))
        np.add.at(out, I.ravel(), (inv @ np.abs(r[I])[..., None])[..., 0].ravel())
    nz = P.mult > 0
    out[nz] /= P.mult[nz]
    return out


@pytest.fixture(scope="module")
def mesh_cache(ctx):
    """Mesh handles per (workload, precision, form), freed before the context."""
    cache = {}
    yield cache
    for h, _ in cache.values():
        h.free()


@pytest.fixture
def mesh(ctx, mesh_cache):
    """A cached mesh handle per (workload, precision, form), schedule reset to
    the set-up default after each test."""
    used = []

    def get(name, prec, form="hybrid", **sched):
        key = (name, prec, form)
        if key not in mesh_cache:
            o = oracle(name)
            m = o["m"]
            h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, form=form)
            mesh_cache[key] = (h, cgs.cgs_mesh_get_schedule(h.handle))
        h, default = mesh_cache[key]
        if sched:
            cgs.cgs_mesh_set_schedule(h.handle, **sched)
        used.append((h, default))
        return h

    yield get
    for h, default in used:
        cgs.cgs_mesh_set_schedule(h.handle, **default)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_default_layouts(mesh):
    """cube32 solves its small subdomains with row packs and the halved cylinder
    (above the row-pack threshold) with lane packs by default."""
    assert cgs.cgs_mesh_get_schedule(mesh("cube32", "fp32").handle)["row_packs"] == 1
    h = mesh("cyl2", "fp32")
    assert h.info["n_sub"] == 16384 and h.info["n_lane_packs"] == 16384 // 32


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("variant", ["lane_packs", "row_packs"])
def test_local_solves(mesh, name, prec, variant):
    o = oracle(name)
    h = mesh(name, prec, **VARIANTS[variant])
    out = torch.empty(o["m"].nv, dtype=torch.float64, device="cuda")
    cgs.cgs_apply_local(h.handle, dev(o["r"]), out, True)
    assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
    err = np.abs(host(out) - o["local"])
    mmax = h.info["max_sub_dofs"]
    g = (mmax + 12) * U32 / (1 - (mmax + 12) * U32)
    bound = (g + (2 * U16 if prec == "fp16" else 0.0)) * o["bound"] + 1e-300
    if prec == "fp16":
        bound += U32 * o["inv_max"] * mmax * np.abs(o["r"]).max()
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("form", ["hybrid", "additive"])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_preconditioner(mesh, name, prec, form, variant):
    o = oracle(name)
    h = mesh(name, prec, form, **VARIANTS[variant])
    z = torch.empty(o["m"].nv, dtype=torch.float64, device="cuda")
    cgs.cgs_apply_preconditioner(h.handle, dev(o["r"]), z)
    assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
    tol = 1e-5 if prec == "fp32" else 2e-3
    assert rel_inf(host(z), o["M_" + form]) <= tol


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("variant", list(SOLVE_VARIANTS))
def test_solve(mesh, name, prec, variant):
    o = oracle(name)
    P, b = o["P"], o["b"]
    h = mesh(name, prec, **SOLVE_VARIANTS[variant])
    x = torch.empty(o["m"].nv, dtype=torch.float64, device="cuda")
    st, its, rel = cgs.cgs_solve(h.handle, dev(b), x, rtol=1e-8, maxit=1000)
    assert st == cgs.OK and rel[0] <= 1.5e-8
    assert abs(int(its[0]) - oracle_iters(name)) <= 1
    bb = np.where(P.dir, 0.0, b)
    assert np.linalg.norm(bb - P.apply_A(host(x))) / np.linalg.norm(bb) <= 1.5e-8
