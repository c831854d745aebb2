"""The operator by rows of the assembled free block (sliced ELL) against the
element form and the oracle: the FP64 row apply and the float-pair row apply
of the mixed forms each give the same A x as the element-by-element kernels
(Sec. 3, A = Q^T A_L Q) up to the order of the additions, and the stored rows
hold exactly the oracle's nonzeros."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402

MESHES = {"cube32": meshes.workload_cube32, "cyl2": lambda: meshes.workload_cylinder(scale=2),
          "cube8_outflow": meshes.workload_cube8}


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _mesh(name):
    m, _ = MESHES[name]()
    d = meshes.outflow_dirichlet(m) if name.endswith("outflow") else None
    return m, d


@pytest.mark.parametrize("name", list(MESHES))
def test_rows_hold_the_oracles_nonzeros(ctx, name):
    m, d = _mesh(name)
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes, dirichlet=None if d is None else d.astype(bool))
    for prec in ("fp64", "fp32"):
        with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec, dirichlet=d) as h:
            info = cgs.cgs_mesh_info(h.handle)
            # the assembled free block: structural nonzeros (entries of
            # coupled vertex pairs), never fewer than the oracle's stored ones
            A = P.A.tocsr()
            assert info["ell_nnz"] == A.nnz
            assert info["ell_slots"] % 32 == 0 and info["ell_slots"] >= info["ell_nnz"]


@pytest.mark.parametrize("name", list(MESHES))
def test_fp64_rows_equal_the_element_form(ctx, name):
    m, d = _mesh(name)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(m.nv)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64", dirichlet=d) as h64, \
            cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32", dirichlet=d) as h32:
        y_rows = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        y_elem = torch.empty_like(y_rows)
        cgs.cgs_apply_A(h64.handle, dev(x), y_rows)                       # rows, float64
        cgs.cgs_apply_A_prec(h32.handle, dev(x), y_elem, "fp64")          # elements, float64
        a, b = host(y_rows), host(y_elem)
    scale = np.abs(b).max()
    assert np.abs(a - b).max() <= 1e-13 * scale


@pytest.mark.parametrize("name", list(MESHES))
def test_pair_rows_equal_the_tiled_element_form(ctx, name):
    """The outer operator of the mixed forms (float pairs, about 48 bits):
    by rows (schedule tile_tma 0) and by TMA-staged element tiles (tile_tma
    1) agree to the pair arithmetic's 2^-44 of the operator's magnitude."""
    m, d = _mesh(name)
    x = np.random.default_rng(4).standard_normal(m.nv)
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32", dirichlet=d) as h:
        y = {}
        for tma in (0, 1):
            cgs.cgs_mesh_set_schedule(h.handle, tile_tma=tma)
            out = torch.empty(m.nv, dtype=torch.float64, device="cuda")
            cgs.cgs_apply_A_prec(h.handle, dev(x), out, "outer")
            assert cgs.cgs_mesh_step_status(h.handle) == cgs.OK
            y[tma] = host(out)
        ref = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_A_prec(h.handle, dev(x), ref, "fp64")
        ref = host(ref)
    mag = np.abs(ref).max() + np.abs(x).max()
    assert np.abs(y[0] - y[1]).max() <= 2.0 ** -40 * mag * 64
    assert np.abs(y[0] - ref).max() <= 2.0 ** -40 * mag * 64
