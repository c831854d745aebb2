"""Per-result error bounds of the reduced-precision kernels, entry by entry,
against the FP64 oracle (the bounds the design notes derive; u = 2^-24 is the
float32 unit roundoff, gamma_k = k u / (1 - k u)).

* Inner operator (Eq. (5), s = r - A l, float32, difference form
  y_i += a_ij (x_j - x_i)): with k_i = 7 n_i + 8, n_i the elements at vertex i,
      |dy_i| <= gamma_{k_i} sum_e sum_{j != i} |a^e_ij| (|x_j| + |x_i|).
* Outer operator (q = A p, hi/lo float pairs, about 48 bits): the same sum of
  magnitudes with 2^-45 (k_i + 8) in place of gamma.
* Restriction and interpolation (Sec. 4, J~ = W Q^T J_L, float32 weights from
  float32 coordinates relative to the box origin): each weighted term
  carries gamma_23 |w| (weight product, input roundings, per-lane and warp
  sums) plus the effect of the rounded coordinates on the weights,
  sum_d dt_d prod_{d' != d} |f_d'|, with f_d = t_d or 1 - t_d and
  dt_d = u (3 (c_d + 1) + 4 |t_d| + 4) for the element's cell index c_d.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402

U32 = 2.0 ** -24
MESHES = {"cube32": meshes.workload_cube32, "cyl2": lambda: meshes.workload_cylinder(scale=2)}


def gamma(k):
    return k * U32 / (1 - k * U32)


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


_cache = {}


def problem(name):
    if name not in _cache:
        m, _ = MESHES[name]()
        _cache[name] = (m, O.Problem(m.xyz, m.conn, m.part, m.boxes))
    return _cache[name]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _operator_magnitude(P, x):
    """sum_e sum_{j != i} |a^e_ij| (|x_j| + |x_i|) and the term counts k_i."""
    xe = np.abs(x[P.conn])                                     # (E, 8)
    Aoff = np.abs(P.Ae).copy()
    Aoff[:, np.arange(8), np.arange(8)] = 0.0
    contrib = np.einsum("eij,ej->ei", Aoff, xe) + Aoff.sum(axis=2) * xe
    mag = np.zeros(P.nv)
    np.add.at(mag, P.conn.ravel(), contrib.ravel())
    k = 7 * P.cnt + 8
    return mag, k


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("op", ["inner", "outer"])
@pytest.mark.parametrize("tile_tma", [0, 1])
def test_operator_error_within_bound(ctx, name, op, tile_tma):
    m, P = problem(name)
    x = np.where(P.dir, 0.0, np.random.default_rng(41).standard_normal(m.nv))
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        cgs.cgs_mesh_set_schedule(h.handle, tile_tma=tile_tma)
        y = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_A_prec(h.handle, dev(x), y, op)
        assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
        got = host(y)
    ref = P.apply_A(x)
    mag, k = _operator_magnitude(P, x)
    bound = (gamma(k) if op == "inner" else 2.0 ** -45 * (k + 8)) * mag + 1e-300
    err = np.abs(got - ref)
    assert np.all(err[~P.dir] <= bound[~P.dir]), float((err / bound)[~P.dir].max())
    assert np.all(got[P.dir] == 0.0)


def _weight_terms(P):
    """Per (element, local vertex, corner): |w|, the coordinate-rounding term
    of the float weights, and the reduced column (-1 = inactive)."""
    X = P.xyz[P.conn]                                            # (E, 8, 3)
    t = (X - (P.box_lo + P.cell * P.box_H)[:, None, :]) / P.box_H
    dt = U32 * (3.0 * (P.cell[:, None, :] + 1) + 4.0 * np.abs(t) + 4.0)
    dw = np.zeros((P.ne, 8, 8))
    for mc in range(8):
        f = np.stack([t[..., d] if (mc >> d) & 1 else 1.0 - t[..., d] for d in range(3)], axis=-1)
        for d in range(3):
            others = np.prod(np.abs(np.delete(f, d, axis=-1)), axis=-1)
            dw[:, :, mc] += dt[..., d] * others
    dw[P.dir[P.conn]] = 0.0
    return np.abs(P.Je), dw


@pytest.mark.parametrize("name", list(MESHES))
def test_restriction_error_within_bound(ctx, name):
    m, P = problem(name)
    s = np.where(P.dir, 0.0, np.random.default_rng(42).standard_normal(m.nv))
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        rr = torch.empty(P.nr, dtype=torch.float64, device="cuda")
        cgs.cgs_restrict(h.handle, dev(s), rr)
        got = host(rr)
    ref = P.restrict(s)
    aw, dw = _weight_terms(P)
    a = (np.abs(s) / P.cnt)[P.conn]                              # (E, 8)
    terms = a[:, :, None] * (gamma(23) * aw + dw)                # (E, 8 nodes, 8 corners)
    per_corner = terms.sum(axis=1)                               # (E, 8 corners)
    bound = np.zeros(P.nr + 1)
    np.add.at(bound, np.where(P.corner_col >= 0, P.corner_col, P.nr).ravel(), per_corner.ravel())
    bound = bound[:P.nr] + 1e-300
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("interp_cells", [0, 1])
def test_interpolation_error_within_bound(ctx, name, interp_cells):
    m, P = problem(name)
    u = np.random.default_rng(43).standard_normal(P.nr)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h:
        cgs.cgs_mesh_set_schedule(h.handle, interp_cells=interp_cells)
        z = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_interp(h.handle, dev(u), z)
        got = host(z)
    ref = P.interp(u)
    aw, dw = _weight_terms(P)
    ux = np.append(np.abs(u), 0.0)[np.where(P.corner_col >= 0, P.corner_col, P.nr)]   # (E, 8 corners)
    per_node = np.einsum("ekm,em->ek", gamma(23) * aw + dw, ux)
    bound = np.zeros(P.nv)
    np.add.at(bound, P.conn.ravel(), per_node.ravel())
    bound = bound / P.cnt + 1e-300
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())
