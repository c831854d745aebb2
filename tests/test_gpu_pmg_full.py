"""The p-multigrid wrap at full size (32^3 deformed cube, order 7, schedule
7 -> 3 -> 1, 11,390,625 nodes) against stored oracle results
(tests/golden/pmg_oracle.json, written by tests/golden/make_pmg_golden.py
from the FP64 oracle only).  Values are compared at sampled element-local
positions (element, k, j, i), which both node numberings share."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_20496_b300 import cgs, meshes  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pmg_oracle.json")


@pytest.fixture(scope="module")
def setup():
    if not os.path.exists(GOLDEN):
        pytest.skip("no stored oracle results")
    gold = json.load(open(GOLDEN))
    m, orders = meshes.workload_sem()
    assert list(orders) == gold["orders"]
    ctx = cgs.cgs_create(0)
    h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64")
    g = cgs.PMG(h, m.xyz, m.conn, orders)
    gmap = cgs.cgs_pmg_node_map(g.handle, 0, m.ne)
    pos = np.asarray(gold["positions"])
    idx = gmap[pos[:, 0], pos[:, 1], pos[:, 2], pos[:, 3]]
    X = cgs.cgs_pmg_node_coords(g.handle, 0)
    b = torch.as_tensor(meshes.sem_rhs(X), device="cuda")
    yield gold, g, b, idx
    g.free()
    h.free()
    cgs.cgs_destroy(ctx)


def test_sizes(setup):
    gold, g, b, idx = setup
    assert g.levels[0]["n_nodes"] == gold["n_nodes"] and g.levels[0]["n_free"] == gold["n_free"]


def test_operator_and_preconditioner_at_sampled_nodes(setup):
    gold, g, b, idx = setup
    y = torch.empty_like(b)
    cgs.cgs_pmg_apply_A(g.handle, 0, b, y)
    ref = np.asarray(gold["apply_A"])
    got = y.cpu().numpy()[idx]
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    cgs.cgs_pmg_apply_preconditioner(g.handle, b, y)
    ref = np.asarray(gold["m_pmg"])
    got = y.cpu().numpy()[idx]
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_solve_against_stored_oracle(setup):
    gold, g, b, idx = setup
    s = gold["solve"]
    x = torch.empty_like(b)
    st, its, rel = cgs.cgs_pmg_solve(g.handle, b, x, rtol=s["rtol"], maxit=300, restart=s["restart"])
    assert st == cgs.OK and rel <= s["rtol"]
    assert abs(its - s["iters"]) <= 1, (its, s["iters"])
    xs = x.cpu().numpy()
    ref = np.asarray(s["x"])
    assert np.linalg.norm(xs[idx] - ref) <= 1e-6 * np.linalg.norm(ref)
    assert abs(float(np.linalg.norm(xs)) - s["x_norm"]) <= 1e-6 * s["x_norm"]
    # the true residual on the device: A x is exactly 0 at the Dirichlet nodes
    # (and nowhere else for this x), where b is ignored
    y = torch.empty_like(b)
    cgs.cgs_pmg_apply_A(g.handle, 0, x, y)
    ys = y.cpu().numpy()
    dirm = ys == 0.0
    assert dirm.sum() == g.levels[0]["n_nodes"] - g.levels[0]["n_free"]
    bb = np.where(dirm, 0.0, b.cpu().numpy())
    assert np.linalg.norm(bb - ys) <= 1.01 * s["rtol"] * np.linalg.norm(bb)
