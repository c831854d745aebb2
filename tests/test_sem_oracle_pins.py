"""Pins of the p-multigrid oracle (oracle/sem_oracle.py) against closed forms,
invariants and brute force: textbook GLL rules, exact differentiation and
interpolation of polynomials, node counts of structured meshes, the patch test
and an exact energy of the SEM operator, a dense element matrix built by
loops, the 1D fast-diagonalisation factors from a 1D assembly, the dense
Kronecker-sum inverse, and the dense form of Eqs. (13) and (14)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import cgs_oracle as CO
from oracle import sem_oracle as S
from paper_2606_20496_b300 import meshes


@pytest.fixture(scope="module")
def cube2():
    return meshes.cube(2, perturb=0.2, seed=3, boxes=(2, 2, 2))


@pytest.fixture(scope="module")
def cube3():
    return meshes.cube(3, perturb=0.2, seed=5, boxes=(2, 2, 2))


# -- one dimension -------------------------------------------------------------

def test_gll_textbook_values():
    x, w = S.gll(2)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = S.gll(3)
    assert np.allclose(x, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = S.gll(4)
    a = np.sqrt(3 / 7)
    assert np.allclose(x, [-1, -a, 0, a, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8])
def test_gll_quadrature_degree(n):
    """Exact for every monomial of degree <= 2n - 1; not for x^(2n)."""
    x, w = S.gll(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    assert abs(np.dot(w, x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("n", [2, 3, 7])
def test_derivative_and_interpolation_exact_on_polynomials(n):
    x, _ = S.gll(n)
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n + 1)
    p = np.polynomial.Polynomial(c)
    assert np.allclose(S.derivative_matrix(x) @ p(x), p.deriv()(x), atol=1e-11)
    xf, _ = S.gll(n + 4)
    assert np.allclose(S.interpolation_matrix(x, xf) @ p(x), p(xf), atol=1e-12)
    assert np.allclose(S.interpolation_matrix(x, x), np.eye(n + 1), atol=1e-14)


# -- numbering, Dirichlet nodes, geometry ----------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_node_counts_structured_cube(n):
    m = meshes.cube((3, 2, 4), perturb=0.2, seed=1)
    L = S.Level(m.xyz, m.conn, n)
    assert L.ng == (3 * n + 1) * (2 * n + 1) * (4 * n + 1)
    # Dirichlet nodes are the nodes on the brick's surface
    assert L.dir.sum() == L.ng - (3 * n - 1) * (2 * n - 1) * (4 * n - 1)
    # every copy of a node has the same physical position
    X = L.node_coords()
    assert np.abs(L.coords.reshape(-1, 3) - X[L.l2g.ravel()]).max() < 1e-14
    # distinct nodes are at distinct positions
    q = np.round(X / 1e-9).astype(np.int64)
    assert np.unique(q, axis=0).shape[0] == L.ng


def test_node_counts_periodic_cylinder():
    m = meshes.cylinder(3, 8, 4, boxes=(2, 2, 2))
    for n in (1, 3):
        L = S.Level(m.xyz, m.conn, n)
        assert L.ng == (3 * n + 1) * (8 * n) * (4 * n + 1)


def test_order_one_level_is_the_vertex_mesh(cube3):
    L = S.Level(cube3.xyz, cube3.conn, 1)
    assert L.ng == cube3.nv
    v = np.zeros(L.ng, dtype=np.int64)
    v[L.l2g.reshape(-1, 8)] = cube3.conn
    assert np.abs(L.node_coords() - cube3.xyz[v]).max() < 1e-15
    assert np.array_equal(L.dir, CO.dirichlet_mask(cube3.conn, cube3.nv)[v])


# -- the operator ---------------------------------------------------------------

def _lagrange_deriv_brute(x, j, t):
    """d/dt of the j-th Lagrange polynomial on the nodes x, by the product rule."""
    s = 0.0
    for m in range(len(x)):
        if m == j:
            continue
        term = 1.0 / (x[j] - x[m])
        for k in range(len(x)):
            if k != j and k != m:
                term *= (t - x[k]) / (x[j] - x[k])
        s += term
    return s


def test_element_matrix_brute_force():
    """A^e_IJ = sum_q w_q det J_q grad phi_I . grad phi_J, every index by loops,
    the Jacobian from finite differences of the trilinear map, against the
    tensor-product apply on unit vectors."""
    n = 2
    m = meshes.cube(1, boxes=(2, 2, 2))
    xyz = m.xyz.copy()
    xyz += np.random.default_rng(8).uniform(-0.12, 0.12, size=xyz.shape)
    L = S.Level(xyz, m.conn, n)
    x, w = L.x, L.w
    p = n + 1
    X = xyz[m.conn[0]]

    def pos(r, s, t):
        out = np.zeros(3)
        for v in range(8):
            a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
            out += ((1 + r) / 2 if a else (1 - r) / 2) * ((1 + s) / 2 if b else (1 - s) / 2) \
                * ((1 + t) / 2 if c else (1 - t) / 2) * X[v]
        return out

    def val1(j, t):
        v = 1.0
        for k in range(p):
            if k != j:
                v *= (t - x[k]) / (x[j] - x[k])
        return v

    A = np.zeros((p ** 3, p ** 3))
    h = 1e-6
    for qk in range(p):
        for qj in range(p):
            for qi in range(p):
                r, s, t = x[qi], x[qj], x[qk]
                J = np.stack([(pos(r + h, s, t) - pos(r - h, s, t)) / (2 * h),
                              (pos(r, s + h, t) - pos(r, s - h, t)) / (2 * h),
                              (pos(r, s, t + h) - pos(r, s, t - h)) / (2 * h)], axis=1)
                Jinv = np.linalg.inv(J)
                grads = np.zeros((p ** 3, 3))
                for k in range(p):
                    for j in range(p):
                        for i in range(p):
                            gref = np.array([_lagrange_deriv_brute(x, i, r) * val1(j, s) * val1(k, t),
                                             val1(i, r) * _lagrange_deriv_brute(x, j, s) * val1(k, t),
                                             val1(i, r) * val1(j, s) * _lagrange_deriv_brute(x, k, t)])
                            grads[i + p * (j + p * k)] = Jinv.T @ gref
                A += w[qi] * w[qj] * w[qk] * np.linalg.det(J) * grads @ grads.T
    cols = np.stack([L.local_apply(np.eye(p ** 3)[c].reshape(1, p, p, p)).ravel() for c in range(p ** 3)], axis=1)
    assert np.abs(cols - A).max() < 1e-8 * np.abs(A).max()
    assert np.abs(cols - cols.T).max() < 1e-13 * np.abs(cols).max()


@pytest.mark.parametrize("n", [2, 3, 7])
def test_patch_test_linear_fields(n):
    """A_N u = 0 at every free node for a linear u (GLL quadrature of order n
    integrates the trilinear-map integrand exactly, n >= 2)."""
    m, _ = meshes.workload_cube8()
    L = S.Level(m.xyz, m.conn, n)
    X = L.node_coords()
    u = 0.3 + X @ np.array([1.0, -2.0, 0.5])
    y = L.scatter(L.local_apply(L.gather(u)))
    assert np.abs(y[~L.dir]).max() < 1e-12 * np.abs(u).max()
    # and constants: zero row sums everywhere
    assert np.abs(L.scatter(L.local_apply(L.gather(np.ones(L.ng))))).max() < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_energy_of_a_quadratic_on_an_affine_mesh(n):
    """u = x^2 + y z on the unit cube: u^T A u = int |grad u|^2 = 4/3 + 1/3 + 1/3."""
    m = meshes.cube(3)
    L = S.Level(m.xyz, m.conn, n)
    X = L.node_coords()
    u = X[:, 0] ** 2 + X[:, 1] * X[:, 2]
    e = float(u @ L.scatter(L.local_apply(L.gather(u))))
    assert abs(e - 2.0) < 1e-12


# -- transfers --------------------------------------------------------------------

def test_transfer_is_transposed_and_reproduces_polynomials(cube2):
    f, c = S.Level(cube2.xyz, cube2.conn, 3), S.Level(cube2.xyz, cube2.conn, 2)
    T = S.Transfer(f, c)
    J = np.stack([T.prolong(np.eye(c.ng)[j]) for j in range(c.ng)], axis=1)
    JT = np.stack([T.restrict(np.eye(f.ng)[i]) for i in range(f.ng)], axis=1)
    assert np.abs(J.T - JT).max() < 1e-14
    # a bubble of degree 2 per direction on an affine mesh lives in both spaces
    m = meshes.cube(2)
    f, c = S.Level(m.xyz, m.conn, 7), S.Level(m.xyz, m.conn, 3)
    T = S.Transfer(f, c)
    bub = lambda X: X[:, 0] * (1 - X[:, 0]) * X[:, 1] * (1 - X[:, 1]) * X[:, 2] * (1 - X[:, 2])
    assert np.abs(T.prolong(bub(c.node_coords())) - bub(f.node_coords())).max() < 1e-14


# -- the smoother ----------------------------------------------------------------

def _assembled_1d(n, length, nel):
    x, w = S.gll(n)
    D = S.derivative_matrix(x)
    Ae = (2 / length) * D.T @ np.diag(w) @ D
    Be = (length / 2) * np.diag(w)
    N = nel * n + 1
    A, B = np.zeros((N, N)), np.zeros((N, N))
    for e in range(nel):
        s = slice(e * n, e * n + n + 1)
        A[s, s] += Ae
        B[s, s] += Be
    return A, B


@pytest.mark.parametrize("n", [2, 3, 7])
def test_extended_1d_factors_from_a_1d_assembly(n):
    L = 0.37
    A3, B3 = _assembled_1d(n, L, 3)
    mid = np.arange(n, 2 * n + 1)                       # the middle element's nodes
    A, B, keep = S.extended_1d(n, L, False, False)
    assert keep == list(range(n + 1))
    assert np.allclose(A, A3[np.ix_(mid, mid)], atol=1e-12) and np.allclose(B, B3[np.ix_(mid, mid)], atol=1e-15)
    # a Dirichlet low side: the element is the first of a two-element line whose
    # first node is dropped
    A2, B2 = _assembled_1d(n, L, 2)
    A, B, keep = S.extended_1d(n, L, True, False)
    assert keep == list(range(1, n + 1))
    sub = np.arange(1, n + 1)
    assert np.allclose(A[np.ix_(keep, keep)], A2[np.ix_(sub, sub)], atol=1e-12)
    assert np.allclose(B[np.ix_(keep, keep)], B2[np.ix_(sub, sub)], atol=1e-15)


def test_element_lengths_of_a_brick():
    """Mean edge length per reference direction: 1/3, 1/2, 1/4 on a 3 x 2 x 4
    brick of the unit cube, and the cylinder's radial, azimuthal-chord and
    axial sizes."""
    m = meshes.cube((3, 2, 4))
    assert np.allclose(S.element_lengths(m.xyz, m.conn), [1 / 3, 1 / 2, 1 / 4], atol=1e-15)
    c = meshes.cylinder(2, 8, 3, grading=1.0, aspect=10.0, boxes=(2, 2, 2))
    L = S.element_lengths(c.xyz, c.conn)
    r0, r1 = 1.0 + 0.5 * c.eijk[:, 0], 1.5 + 0.5 * c.eijk[:, 0]
    chord = lambda r: 2 * r * np.sin(np.pi / 8)
    assert np.allclose(L[:, 0], 0.5, atol=1e-14)
    assert np.allclose(L[:, 1], 0.5 * (chord(r0) + chord(r1)), atol=1e-14)
    assert np.allclose(L[:, 2], 5.0, atol=1e-13)


def test_fdm_is_the_inverse_of_the_kronecker_sum(cube3):
    lev = S.Level(cube3.xyz, cube3.conn, 3)
    sm = S.Smoother(lev)
    lengths = S.element_lengths(cube3.xyz, cube3.conn)
    p = lev.p
    for e in (0, 13, 26):                                # a corner, the centre, a corner
        fac = []
        for d in range(3):
            A, B, keep = S.extended_1d(3, lengths[e, d], lev.face_bdry[e, 2 * d], lev.face_bdry[e, 2 * d + 1])
            P = np.zeros((p, p))
            P[keep, keep] = 1.0
            fac.append((P @ A @ P, P @ B @ P, P))
        (Ax, Bx, Px), (Ay, By, Py), (Az, Bz, Pz) = fac
        K = np.kron(Bz, np.kron(By, Ax)) + np.kron(Bz, np.kron(Ay, Bx)) + np.kron(Az, np.kron(By, Bx))
        Pk = np.kron(Pz, np.kron(Py, Px))
        idx = np.flatnonzero(np.diag(Pk))
        Kinv = np.zeros_like(K)
        Kinv[np.ix_(idx, idx)] = np.linalg.inv(K[np.ix_(idx, idx)])
        rL = np.zeros((lev.ne, p, p, p))
        cols = []
        for c in range(p ** 3):
            rL[:] = 0.0
            rL[e].flat[c] = 1.0
            cols.append(sm.local_solve(rL)[e].ravel())
        assert np.abs(np.stack(cols, 1) - Kinv).max() < 1e-11 * np.abs(Kinv).max()


def _dense(fn, n):
    return np.stack([fn(np.eye(n)[j]) for j in range(n)], axis=1)


def test_smoother_dense_formula(cube2):
    """Eq. (14): W_N sum_e R_e^T A~_e^-1 R_e from dense R_e."""
    lev = S.Level(cube2.xyz, cube2.conn, 2)
    sm = S.Smoother(lev)
    p3 = lev.p ** 3
    M = np.zeros((lev.ng, lev.ng))
    for e in range(lev.ne):
        R = np.zeros((p3, lev.ng))
        R[np.arange(p3), lev.l2g[e].ravel()] = 1.0
        Ainv = np.stack([sm.local_solve(np.eye(p3)[c].reshape(1, lev.p, lev.p, lev.p).repeat(lev.ne, 0))[e].ravel()
                         for c in range(p3)], axis=1)
        M += R.T @ Ainv @ R
    Pm = np.diag((~lev.dir).astype(float))
    M = Pm @ np.diag(1.0 / lev.mult) @ M @ Pm
    assert np.abs(_dense(sm.apply, lev.ng) - M).max() < 1e-13 * np.abs(M).max()


def test_pmg_dense_formula(cube3):
    """Eq. (13) with orders 3 -> 2 -> 1 from dense blocks."""
    P = S.PMG(cube3.xyz, cube3.conn, cube3.part, cube3.boxes, orders=(3, 2))
    f, m, c = P.levels
    M3, M2 = _dense(P.smoothers[0].apply, f.ng), _dense(P.smoothers[1].apply, m.ng)
    J1 = _dense(P.transfers[0].prolong, m.ng)
    J2 = _dense(P.transfers[1].prolong, c.ng)
    Mc = _dense(P.coarse_apply, c.ng)
    Pm = np.diag((~f.dir).astype(float))
    M = (M3 + J1 @ (M2 + J2 @ Mc @ J2.T) @ J1.T) @ Pm
    assert np.abs(_dense(P.apply_M, f.ng) - M).max() < 1e-12 * np.abs(M).max()
    # the order-1 level's M_c is the coarse problem's preconditioner on the vertices
    r = np.where(c.dir, 0.0, np.random.default_rng(2).standard_normal(c.ng))
    rv = np.zeros(cube3.nv)
    rv[P.c2v] = r
    assert np.allclose(P.coarse_apply(r), P.coarse.apply_M(rv, "hybrid")[P.c2v], atol=1e-15)


def test_pmg_solve_matches_a_direct_solve(cube3):
    P = S.PMG(cube3.xyz, cube3.conn, cube3.part, cube3.boxes, orders=(4, 2))
    f = P.fine
    A = _dense(f.apply_A, f.ng)
    free = ~f.dir
    b = np.where(f.dir, 0.0, meshes.sem_rhs(f.node_coords()))
    x_direct = np.zeros(f.ng)
    x_direct[free] = sla.solve(A[np.ix_(free, free)], b[free], assume_a="pos")
    x, its, rel, ok = P.solve(b, rtol=1e-12, maxit=200)
    assert ok and rel <= 1e-12
    assert np.linalg.norm(x - x_direct) <= 1e-10 * np.linalg.norm(x_direct)
    assert np.all(x[f.dir] == 0.0)
