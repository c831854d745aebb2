"""The p-multigrid wrap on the GPU (Sec. 1, Sec. 5, Eqs. (13) and (14))
against the oracle (oracle/sem_oracle.py), entry by entry.

The two sides number the spectral-element nodes differently, so vectors are
compared element by element: u_L[e, k, j, i] = u[l2g[e, k, j, i]] with each
side's own map.  Inputs are oracle vectors carried over the same way (every
copy of a node holds the same value, so the scatter is well defined).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sem_oracle as S  # noqa: E402
from paper_2606_20496_b300 import cgs, meshes  # noqa: E402

CASES = {
    "cube8_7_3": (lambda: meshes.workload_cube8()[0], (7, 3)),
    "cyl8_5_2": (lambda: meshes.workload_cylinder(scale=8)[0], (5, 2)),
}


@pytest.fixture(scope="module")
def ctx():
    c = cgs.cgs_create(0)
    yield c
    cgs.cgs_destroy(c)


@pytest.fixture(scope="module")
def built(ctx):
    store = {}
    yield lambda name: _get(ctx, store, name)
    for m, h, g, P, maps in store.values():
        g.free()
        h.free()


def _get(ctx, store, name):
    if name not in store:
        fn, orders = CASES[name]
        m = fn()
        h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64")
        g = cgs.PMG(h, m.xyz, m.conn, orders)
        P = S.PMG(m.xyz, m.conn, m.part, m.boxes, orders=orders)
        maps = [cgs.cgs_pmg_node_map(g.handle, l, m.ne) for l in range(len(orders) + 1)]
        store[name] = (m, h, g, P, maps)
    return store[name]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def to_gpu_numbering(u_or, lev_or, gmap, ng):
    out = np.zeros(ng)
    out[gmap.ravel()] = u_or[lev_or.l2g].ravel()
    return out


def local(u, l2g):
    return u[l2g]


def rand_level(P, l, seed):
    lev = P.levels[l]
    return np.where(lev.dir, 0.0, np.random.default_rng(seed).standard_normal(lev.ng))


def assert_close(got_L, ref_L, tol):
    scale = np.abs(ref_L).max()
    err = np.abs(got_L - ref_L).max()
    assert err <= tol * scale, (err, scale)


@pytest.mark.parametrize("name", list(CASES))
def test_numbering_and_coordinates(built, name):
    m, h, g, P, maps = built(name)
    for l, lev in enumerate(P.levels):
        info = g.levels[l]
        assert info["n_nodes"] == lev.ng and info["n_free"] == int((~lev.dir).sum())
        gm = maps[l]
        assert gm.min() == 0 and gm.max() == lev.ng - 1 and np.unique(gm).size == lev.ng
        X = cgs.cgs_pmg_node_coords(g.handle, l)
        assert np.abs(X[gm] - lev.coords).max() <= 1e-13 * np.abs(lev.coords).max()
        # the two numberings identify the same nodes: one oracle node per GPU node
        pairs = np.unique(np.stack([gm.ravel(), lev.l2g.ravel()], 1), axis=0)
        assert pairs.shape[0] == lev.ng
    assert np.array_equal(maps[-1].reshape(m.ne, 8), m.conn)


@pytest.mark.parametrize("name", list(CASES))
def test_operator_every_level(built, name):
    m, h, g, P, maps = built(name)
    for l in range(len(g.orders)):
        lev = P.levels[l]
        u = rand_level(P, l, 10 + l)
        y = torch.empty(lev.ng, dtype=torch.float64, device="cuda")
        cgs.cgs_pmg_apply_A(g.handle, l, dev(to_gpu_numbering(u, lev, maps[l], lev.ng)), y)
        got = host(y)
        assert_close(local(got, maps[l]), local(lev.apply_A(u), lev.l2g), 1e-12)
        assert np.all(got[maps[l][lev.dir[lev.l2g]]] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_smoother_every_level(built, name):
    m, h, g, P, maps = built(name)
    for l in range(len(g.orders)):
        lev = P.levels[l]
        r = rand_level(P, l, 20 + l)
        z = torch.empty(lev.ng, dtype=torch.float64, device="cuda")
        cgs.cgs_pmg_smooth(g.handle, l, dev(to_gpu_numbering(r, lev, maps[l], lev.ng)), z)
        assert_close(local(host(z), maps[l]), local(P.smoothers[l].apply(r), lev.l2g), 1e-11)


@pytest.mark.parametrize("name", list(CASES))
def test_transfers_every_level(built, name):
    m, h, g, P, maps = built(name)
    for l in range(len(g.orders)):
        f, c, T = P.levels[l], P.levels[l + 1], P.transfers[l]
        rf = rand_level(P, l, 30 + l)
        rc = torch.empty(c.ng, dtype=torch.float64, device="cuda")
        cgs.cgs_pmg_restrict(g.handle, l, dev(to_gpu_numbering(rf, f, maps[l], f.ng)), rc)
        assert_close(local(host(rc), maps[l + 1]), local(T.restrict(rf), c.l2g), 1e-12)
        uc = rand_level(P, l + 1, 40 + l)
        uf = torch.empty(f.ng, dtype=torch.float64, device="cuda")
        cgs.cgs_pmg_prolong(g.handle, l, dev(to_gpu_numbering(uc, c, maps[l + 1], c.ng)), uf)
        assert_close(local(host(uf), maps[l]), local(T.prolong(uc), f.l2g), 1e-12)


@pytest.mark.parametrize("name", list(CASES))
def test_preconditioner_eq13(built, name):
    m, h, g, P, maps = built(name)
    f = P.fine
    r = rand_level(P, 0, 50)
    z = torch.full((f.ng,), float("nan"), dtype=torch.float64, device="cuda")
    cgs.cgs_pmg_apply_preconditioner(g.handle, dev(to_gpu_numbering(r, f, maps[0], f.ng)), z)
    assert_close(local(host(z), maps[0]), local(P.apply_M(r), f.l2g), 1e-11)


@pytest.mark.parametrize("name", list(CASES))
def test_solve_against_oracle(built, name):
    m, h, g, P, maps = built(name)
    f = P.fine
    b = np.where(f.dir, 0.0, meshes.sem_rhs(f.node_coords()))
    x_or, its_or, rel_or, ok = P.solve(b, rtol=1e-8, maxit=300, restart=30)
    assert ok
    x = torch.empty(f.ng, dtype=torch.float64, device="cuda")
    st, its, rel = cgs.cgs_pmg_solve(g.handle, dev(to_gpu_numbering(b, f, maps[0], f.ng)), x, rtol=1e-8,
                                     maxit=300, restart=30)
    assert st == cgs.OK and rel <= 1e-8
    assert abs(its - its_or) <= 1, (its, its_or)
    xg = local(host(x), maps[0])
    xo = local(x_or, f.l2g)
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    # the true residual of the GPU solution, by the oracle's operator
    xg_or = np.zeros(f.ng)
    xg_or[f.l2g.ravel()] = xg.ravel()
    assert np.linalg.norm(b - f.apply_A(xg_or)) <= 1.01e-8 * np.linalg.norm(b)


def test_setup_rejects_bad_arguments(ctx):
    m, _ = meshes.workload_cube8()
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64") as h:
        for orders in ((3, 3), (9,), (1,), (3, 5), (7, 5, 4, 3, 2)):
            with pytest.raises(cgs.CGSError) as ei:
                cgs.cgs_pmg_setup(h.handle, m.xyz, m.conn, orders)
            assert ei.value.status == cgs.ERR_INVALID_ARG
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_pmg_setup(h.handle, m.xyz[:-1], m.conn, (3,))
        assert ei.value.status == cgs.ERR_INVALID_ARG
    # a mesh whose Dirichlet set is not the boundary faces
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64",
                  dirichlet=meshes.outflow_dirichlet(m)) as h:
        with pytest.raises(cgs.CGSError) as ei:
            cgs.cgs_pmg_setup(h.handle, m.xyz, m.conn, (3,))
        assert ei.value.status == cgs.ERR_INVALID_ARG


def test_single_level_schedule(ctx):
    """orders = (4,): the smoother of order 4 and the coarse Schwarz sweep."""
    m, _ = meshes.workload_cube8()
    P = S.PMG(m.xyz, m.conn, m.part, m.boxes, orders=(4,))
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64") as h, \
            cgs.PMG(h, m.xyz, m.conn, (4,)) as g:
        gm = cgs.cgs_pmg_node_map(g.handle, 0, m.ne)
        f = P.fine
        r = np.where(f.dir, 0.0, np.random.default_rng(60).standard_normal(f.ng))
        z = torch.empty(f.ng, dtype=torch.float64, device="cuda")
        cgs.cgs_pmg_apply_preconditioner(g.handle, dev(to_gpu_numbering(r, f, gm, f.ng)), z)
        assert_close(local(host(z), gm), local(P.apply_M(r), f.l2g), 1e-11)


@pytest.mark.parametrize("name", list(CASES))
def test_float_smoothers_under_a_mixed_coarse_mesh(ctx, built, name):
    """Under an FP32-bulk coarse mesh the operator runs in float pairs (within
    1e-11 of its largest entry) and the smoothers and transfers in float
    (level vectors below the finest in float): every entry of M r within
    2e-5 max|M r| of the FP64 oracle (float rounding of six contractions of
    length p and of the FP32-bulk coarse sweep), GMRES within one product of
    the oracle's FP64 count, and the true residual at the tolerance."""
    m, _, _, P, maps = built(name)
    orders = CASES[name][1]
    f = P.fine
    with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32") as h, \
            cgs.PMG(h, m.xyz, m.conn, orders) as g:
        gm = cgs.cgs_pmg_node_map(g.handle, 0, m.ne)
        assert np.array_equal(gm, maps[0])
        # the operator in float-pair arithmetic (about 48 bits)
        for l in range(len(orders)):
            lev = P.levels[l]
            u = rand_level(P, l, 80 + l)
            y = torch.empty(lev.ng, dtype=torch.float64, device="cuda")
            cgs.cgs_pmg_apply_A(g.handle, l, dev(to_gpu_numbering(u, lev, maps[l], lev.ng)), y)
            assert_close(local(host(y), maps[l]), local(lev.apply_A(u), lev.l2g), 1e-11)
        r = rand_level(P, 0, 70)
        z = torch.empty(f.ng, dtype=torch.float64, device="cuda")
        cgs.cgs_pmg_smooth(g.handle, 0, dev(to_gpu_numbering(r, f, gm, f.ng)), z)
        assert_close(local(host(z), gm), local(P.smoothers[0].apply(r), f.l2g), 1e-5)
        cgs.cgs_pmg_apply_preconditioner(g.handle, dev(to_gpu_numbering(r, f, gm, f.ng)), z)
        assert_close(local(host(z), gm), local(P.apply_M(r), f.l2g), 2e-5)
        b = np.where(f.dir, 0.0, meshes.sem_rhs(f.node_coords()))
        _, its_or, _, _ = P.solve(b, rtol=1e-8, maxit=300, restart=30)
        x = torch.empty(f.ng, dtype=torch.float64, device="cuda")
        st, its, rel = cgs.cgs_pmg_solve(g.handle, dev(to_gpu_numbering(b, f, gm, f.ng)), x, rtol=1e-8)
        assert st == cgs.OK and rel <= 1e-8 and abs(its - its_or) <= 1, (st, its, its_or)
        xg = np.zeros(f.ng)
        xg[f.l2g.ravel()] = local(host(x), gm).ravel()
        assert np.linalg.norm(b - f.apply_A(xg)) <= 1.01e-8 * np.linalg.norm(b)
