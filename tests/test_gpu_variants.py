"""The paper's variants of the method on the GPU, against the FP64 oracle.

* Neumann boundaries everywhere except an outflow cap (Sec. 5, the boundary
  conditions of the production runs): the set-up takes the Dirichlet mask;
  the operator, both preconditioner forms and the solve follow the oracle
  with the same mask.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402


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


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


_outflow = {}


def outflow_case():
    if not _outflow:
        m, b = meshes.workload_cylinder(scale=8)
        d = meshes.outflow_dirichlet(m)
        P = O.Problem(m.xyz, m.conn, m.part, m.boxes, dirichlet=d.astype(bool))
        _outflow.update(m=m, b=b, d=d, P=P, its={})
    return _outflow


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_outflow_boundary(ctx, prec, form):
    c = outflow_case()
    m, b, d, P = c["m"], c["b"], c["d"], c["P"]
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, dirichlet=d, prec=prec, form=form) as h:
        ex = cgs.cgs_mesh_export(h.handle)
        np.testing.assert_array_equal(ex["dirichlet"], d)
        np.testing.assert_array_equal(ex["box_active"], P.box_active)
        r = np.random.default_rng(51).standard_normal(m.nv)
        y = torch.empty(m.nv, dtype=torch.float64, device="cuda")
        cgs.cgs_apply_A(h.handle, dev(r), y)
        assert rel_inf(host(y), P.apply_A(np.where(P.dir, 0.0, r))) <= 1e-12
        cgs.cgs_apply_preconditioner(h.handle, dev(r), y)
        assert rel_inf(host(y), P.apply_M(r, form)) <= (1e-11 if prec == "fp64" else 1e-5)
        st, its, rel = cgs.cgs_solve(h.handle, dev(b), y, rtol=1e-8, maxit=4000)
        assert st == cgs.OK and rel[0] <= 1.5e-8
        if form not in c["its"]:
            _, c["its"][form], _, ok = P.solve(b, rtol=1e-8, maxit=4000, form=form)
            assert ok
        assert abs(int(its[0]) - c["its"][form]) <= 1
        bb = np.where(P.dir, 0.0, b)
        assert np.linalg.norm(bb - P.apply_A(host(y))) <= 1.5e-8 * np.linalg.norm(bb)
