"""Pins of the CPU oracle against closed forms, invariants and brute force.

Each test checks one oracle function against something other than the oracle
itself: a textbook closed form, an exact identity the paper states (Sec. 3,
Sec. 4), a brute-force construction written differently, or a dense direct
solve.  They are chosen so that a dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

from oracle import cgs_oracle as O
from paper_2606_20496_b300 import meshes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kron_q1(hx, hy, hz):
    """Q1 box-element stiffness as a Kronecker sum of 1D stiffness/mass."""
    K = lambda h: np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    M = lambda h: h * np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    return (np.kron(M(hz), np.kron(M(hy), K(hx))) + np.kron(M(hz), np.kron(K(hy), M(hx)))
            + np.kron(K(hz), np.kron(M(hy), M(hx))))


def _corners(lo, h):
    return np.array([[lo[0] + (k & 1) * h[0], lo[1] + ((k >> 1) & 1) * h[1],
                      lo[2] + ((k >> 2) & 1) * h[2]] for k in range(8)])


# --------------------------------------------------------------------------
# element matrices
# --------------------------------------------------------------------------

def test_unit_cube_element_matches_golden():
    gold = np.loadtxt(os.path.join(GOLDEN, "q1_unit_cube.txt")) / 12.0
    A, _ = O.element_matrices(_corners([0, 0, 0], [1, 1, 1]), np.arange(8)[None, :])
    np.testing.assert_allclose(A[0], gold, atol=1e-15)


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.3, 2.0, 0.7), (1e-2, 1.0, 1.0)])
def test_box_element_matches_kronecker_closed_form(h):
    A, _ = O.element_matrices(_corners([0.2, -1.0, 3.0], h), np.arange(8)[None, :])
    ref = _kron_q1(*h)
    np.testing.assert_allclose(A[0], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def _ref_integrals():
    """1D integrals over [-1,1] of the linear basis l_0=(1-x)/2, l_1=(1+x)/2."""
    mass = np.array([[2 / 3, 1 / 3], [1 / 3, 2 / 3]])
    s = np.array([-0.5, 0.5])                      # l_s'
    dl_l = np.outer(s, [1.0, 1.0])                 # int l_i' l_j = s_i * 1
    dl_dl = 2.0 * np.outer(s, s)                   # int l_i' l_j'
    return mass, dl_l, dl_dl


def test_affine_element_matches_exact_integral():
    """For x = B xi + c the stiffness is |det B| sum_ab (B^-1 B^-T)_ab K^ab with
    K^ab_ij = int d_a l_i d_b l_j over the reference cube (exact 1D products)."""
    rng = np.random.default_rng(7)
    B = np.eye(3) * 0.5 + 0.2 * rng.standard_normal((3, 3))
    assert np.linalg.det(B) > 0
    c = rng.standard_normal(3)
    xi = np.array([[2 * (k & 1) - 1, 2 * ((k >> 1) & 1) - 1, 2 * ((k >> 2) & 1) - 1] for k in range(8)], float)
    X = xi @ B.T + c
    mass, dl_l, dl_dl = _ref_integrals()
    bits = [[(k >> d) & 1 for d in range(3)] for k in range(8)]
    G = np.linalg.inv(B) @ np.linalg.inv(B).T
    ref = np.zeros((8, 8))
    for i in range(8):
        for j in range(8):
            tot = 0.0
            for a in range(3):
                for b in range(3):
                    prod = 1.0
                    for d in range(3):
                        si, sj = bits[i][d], bits[j][d]
                        if d == a and d == b:
                            prod *= dl_dl[si, sj]
                        elif d == a:
                            prod *= dl_l[si, sj]
                        elif d == b:
                            prod *= dl_l[sj, si]
                        else:
                            prod *= mass[si, sj]
                    tot += G[a, b] * prod
            ref[i, j] = np.linalg.det(B) * tot
    A, _ = O.element_matrices(X, np.arange(8)[None, :])
    np.testing.assert_allclose(A[0], ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_element_matrix_invariants_on_distorted_elements():
    m, _ = meshes.workload_cube8()
    A, min_det = O.element_matrices(m.xyz, m.conn)
    assert min_det > 0
    np.testing.assert_allclose(A, np.swapaxes(A, 1, 2), atol=1e-16)
    assert np.abs(A.sum(axis=2)).max() < 1e-15 * np.abs(A).max() * 8
    # rigid rotation leaves A^e unchanged; uniform scaling by s multiplies it by s (3D)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    Ar, _ = O.element_matrices(m.xyz @ Q.T + 1.5, m.conn)
    As, _ = O.element_matrices(2.5 * m.xyz, m.conn)
    np.testing.assert_allclose(Ar, A, atol=1e-13)
    np.testing.assert_allclose(As, 2.5 * A, atol=1e-13)


@pytest.mark.parametrize("wl", ["cube8", "cube_deformed", "cylinder"])
def test_patch_test_linear_fields(wl):
    """int grad phi_i . grad u dV = 0 at interior vertices for linear u, on
    distorted trilinear meshes (2x2x2 Gauss integrates this exactly)."""
    if wl == "cube8":
        m, _ = meshes.workload_cube8()
    elif wl == "cube_deformed":
        m = meshes.cube(6, deform=True, permute_seed=4)
    else:
        m = meshes.cylinder(4, 16, 4, grading=1.2, aspect=5.0, boxes=(2, 2, 2))
    Ae, _ = O.element_matrices(m.xyz, m.conn)
    A = O.assemble(m.conn.astype(np.int64), Ae, m.nv)
    interior = ~O.dirichlet_mask(m.conn, m.nv)
    rng = np.random.default_rng(11)
    g = rng.standard_normal(3)
    u = m.xyz @ g + 0.7
    y = A @ u
    assert np.abs(y[interior]).max() < 1e-12 * np.abs(A.data).max() * np.abs(u).max()
    # constants are in the null space everywhere
    assert np.abs(A @ np.ones(m.nv)).max() < 1e-13 * np.abs(A.data).max()


def test_assembled_free_block_is_spd_and_27_point_on_uniform_mesh():
    n = 4
    m = meshes.cube(n)
    P = O.Problem(m.xyz, m.conn, m.part, (2, 2, 2))
    Ad = P.A.toarray()
    np.testing.assert_allclose(Ad, Ad.T, atol=1e-15)
    assert np.linalg.eigvalsh(Ad).min() > 0
    # the assembled uniform-grid stencil: centre 8h/3, faces 0, edges -h/6, corners -h/12
    h = 1.0 / n
    c = 2 + (n + 1) * (2 + (n + 1) * 2)
    row = P.A_full[[c], :].toarray()[0]
    assert row[c] == pytest.approx(8 * h / 3, rel=1e-13)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for dk in (-1, 0, 1):
                nz = abs(di) + abs(dj) + abs(dk)
                if nz == 0:
                    continue
                v = c + di + (n + 1) * (dj + (n + 1) * dk)
                expect = {1: 0.0, 2: -h / 6, 3: -h / 12}[nz]
                assert row[v] == pytest.approx(expect, abs=1e-15)


# --------------------------------------------------------------------------
# Dirichlet set, subdomains
# --------------------------------------------------------------------------

def test_dirichlet_mask_cube_and_cylinder():
    m = meshes.cube((3, 4, 5), perturb=0.1, seed=1)
    d = O.dirichlet_mask(m.conn, m.nv)
    i = np.arange(m.nv) % 4
    j = (np.arange(m.nv) // 4) % 5
    k = np.arange(m.nv) // 20
    expect = (i == 0) | (i == 3) | (j == 0) | (j == 4) | (k == 0) | (k == 5)
    np.testing.assert_array_equal(d, expect)
    c = meshes.cylinder(3, 8, 2, grading=1.1, aspect=3.0, boxes=(2, 2, 2))
    d = O.dirichlet_mask(c.conn, c.nv)
    ir = np.arange(c.nv) % 4
    iz = np.arange(c.nv) // (4 * 8)
    np.testing.assert_array_equal(d, (ir == 0) | (ir == 3) | (iz == 0) | (iz == 2))


def test_subdomain_restriction_matches_structured_brute_force():
    """R_p of a 2^3 block grown by one element layer = free vertices strictly
    inside the grown block's vertex range (structured mesh, any perturbation)."""
    dims = (6, 5, 7)
    m = meshes.cube(dims, perturb=0.1, seed=2)
    P = O.Problem(m.xyz, m.conn, m.part, (2, 2, 2))
    nvx, nvy = dims[0] + 1, dims[1] + 1
    vid = np.arange(m.nv)
    vi, vj, vk = vid % nvx, (vid // nvx) % nvy, vid // (nvx * nvy)
    nb = [-(-d // 2) for d in dims]
    for p in range(len(P.sub_idx)):
        bi, bj, bk = p % nb[0], (p // nb[0]) % nb[1], p // (nb[0] * nb[1])
        ok = np.ones(m.nv, bool)
        for v, b, d in ((vi, bi, dims[0]), (vj, bj, dims[1]), (vk, bk, dims[2])):
            lo = max(2 * b - 1, 0)
            hi = min(2 * b + 2 + 1, d)
            ok &= (v > lo) & (v < hi)
        expect = np.flatnonzero(ok & ~P.dir)
        np.testing.assert_array_equal(P.sub_idx[p], expect)


def test_local_solve_satisfies_interior_equations():
    """y = A_p^{-1} R_p r extended by zero solves (A R_p^T y)_i = r_i on R_p:
    A_p is the principal submatrix of A (Sec. 3)."""
    m, b = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    r = np.where(P.dir, 0.0, b)
    for p in (0, 5, 21, 63):
        idx = P.sub_idx[p]
        ext = np.zeros(m.nv)
        ext[idx] = P.local_solve_one(p, r)
        np.testing.assert_allclose(P.apply_A(ext)[idx], r[idx], atol=1e-12)
    # the batched (grouped Cholesky) path gives the same sum as one-by-one solves
    tot = np.zeros(m.nv)
    for p in range(len(P.sub_idx)):
        tot[P.sub_idx[p]] += P.local_solve_one(p, r)
    np.testing.assert_allclose(P.local_solves(r, weighted=False), tot, atol=1e-12)
    w = tot.copy()
    w[P.mult > 0] /= P.mult[P.mult > 0]
    np.testing.assert_allclose(P.local_solves(r, weighted=True), w, atol=1e-12)


# --------------------------------------------------------------------------
# box coarse space
# --------------------------------------------------------------------------

def _trilinear(c, X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z
            + c[6] * x * z + c[7] * x * y * z)


def _box_vertex_xyz(P):
    nb = P.box_b + 1
    a = P.box_active
    ijk = np.stack([a % nb[0], (a // nb[0]) % nb[1], a // (nb[0] * nb[1])], axis=1)
    return P.box_lo + ijk * P.box_H


@pytest.mark.parametrize("wl", ["cube8", "cube_deformed", "cylinder"])
def test_interpolation_reproduces_trilinear_fields(wl):
    if wl == "cube8":
        m, _ = meshes.workload_cube8()
    elif wl == "cube_deformed":
        m = meshes.cube(10, deform=True, permute_seed=4, boxes=(3, 4, 3))
    else:
        m = meshes.cylinder(6, 24, 6, grading=1.1, aspect=4.0, boxes=(4, 4, 3))
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    c = np.random.default_rng(5).standard_normal(8)
    z = P.interp(_trilinear(c, _box_vertex_xyz(P)))
    f = _trilinear(c, m.xyz)
    free = ~P.dir
    np.testing.assert_allclose(z[free], f[free], rtol=1e-13, atol=1e-13 * np.abs(f).max())
    assert np.all(z[P.dir] == 0)


def test_restriction_is_transpose_of_interpolation():
    m = meshes.cube((7, 5, 6), perturb=0.15, seed=9, boxes=(3, 2, 3))
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(P.nr)
    s = np.where(P.dir, 0.0, rng.standard_normal(m.nv))
    assert P.interp(u) @ s == pytest.approx(u @ P.restrict(s), rel=1e-13)


def _vertex_based_J(P):
    """J_ij = Phi_j(x_i) from each free node's bounding box (Sec. 4, the
    vertex-oriented construction), as a dense (n_free, n_r) matrix."""
    nb = P.box_b + 1
    col = -np.ones(int(np.prod(nb)), int)
    col[P.box_active] = np.arange(P.nr)
    J = np.zeros((P.free.size, P.nr))
    for row, v in enumerate(P.free):
        t = (P.xyz[v] - P.box_lo) / P.box_H
        cell = np.clip(np.floor(t).astype(int), 0, P.box_b - 1)
        f = t - cell
        for m in range(8):
            bit = [(m >> d) & 1 for d in range(3)]
            w = np.prod([f[d] if bit[d] else 1 - f[d] for d in range(3)])
            g = cell + bit
            gid = g[0] + nb[0] * (g[1] + nb[1] * g[2])
            if abs(w) > 0:
                assert col[gid] >= 0
                J[row, col[gid]] += w
    return J


def test_galerkin_equality_on_box_aligned_mesh():
    """When element planes align with box planes J_L is continuous and the
    cell-wise assembly (Eq. (12)) equals the Galerkin A_r = J^T A J."""
    m = meshes.cube(8, boxes=(4, 2, 4))
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    J = _vertex_based_J(P)
    np.testing.assert_allclose(P.Ar, J.T @ P.A.toarray() @ J, atol=1e-14 * np.abs(P.Ar).max() * 10)


def test_boxes_equal_to_elements_give_exact_inverse():
    n = 4
    m = meshes.cube(n, boxes=(n, n, n))
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    assert P.nr == P.free.size
    np.testing.assert_allclose(P.Ar, P.A.toarray(), atol=1e-14)
    r = np.where(P.dir, 0.0, np.random.default_rng(2).standard_normal(m.nv))
    np.testing.assert_allclose(P.box_correction(r), P.to_full(np.linalg.solve(P.A.toarray(), r[P.free])),
                               atol=1e-12)


def test_hybrid_residual_is_orthogonal_to_coarse_space_when_galerkin():
    """With A_r = J~^T A J~ the coarse step of Eq. (5) is an A-orthogonal
    projection: J~^T (r - A z) = 0 for z = M r (hybrid)."""
    m = meshes.cube(8, boxes=(2, 4, 2), perturb=0.0)
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    r = np.where(P.dir, 0.0, np.random.default_rng(4).standard_normal(m.nv))
    z = P.apply_M(r, "hybrid")
    res = P.restrict(r - P.apply_A(z))
    assert np.abs(res).max() < 1e-12 * np.abs(P.restrict(r)).max()


def test_reduced_space_count_golden():
    gold = json.load(open(os.path.join(GOLDEN, "reduced_space_counts.json")))
    b = tuple(gold["boxes"])
    m = meshes.cube((14, 14, 24), perturb=0.1, seed=3, boxes=b)
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    assert P.nr == gold["nominal_nr"]
    c = meshes.cylinder(6, 32, 24, grading=1.0, aspect=6.0, boxes=b)
    Pc = O.Problem(c.xyz, c.conn, c.part, c.boxes)
    assert Pc.nr < gold["nominal_nr"]
    nb = np.array(b) + 1
    a = Pc.box_active
    i, j = a % nb[0], (a // nb[0]) % nb[1]
    corner = ((i == 0) | (i == b[0])) & ((j == 0) | (j == b[1]))
    assert not corner.any()


def test_reduced_matrix_spd_and_coarse_solve_exact():
    m, _ = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    np.testing.assert_allclose(P.Ar, P.Ar.T, atol=1e-15)
    assert np.linalg.eigvalsh(P.Ar).min() > 0
    rr = np.random.default_rng(0).standard_normal(P.nr)
    np.testing.assert_allclose(P.Ar @ P.coarse_solve(rr), rr, atol=1e-11)


# --------------------------------------------------------------------------
# preconditioners and iteration
# --------------------------------------------------------------------------

def _dense_M(P, form):
    cols = []
    for j in P.free:
        e = np.zeros(P.nv)
        e[j] = 1.0
        cols.append(P.apply_M(e, form)[P.free])
    return np.array(cols).T


def _cell_by_search(P, point):
    """Box cell holding `point`, by searching the cell intervals along each
    axis (the top face belongs to the last cell)."""
    c = []
    for d in range(3):
        edges = P.box_lo[d] + P.box_H[d] * np.arange(P.box_b[d] + 1)
        k = 0
        while k < P.box_b[d] - 1 and not (edges[k] <= point[d] < edges[k + 1]):
            k += 1
        c.append(k)
    return np.array(c)


def _brute_force_coarse(P, m):
    """Cell of each element's centroid, the averaged interpolant J~ = W Q^T J_L
    (dense, free rows, active columns) and A_r = sum_e J_e^T A^e J_e (Eq. (12)),
    element by element with Python loops (Sec. 4: each element belongs to the
    box cell holding its centroid, and interpolates trilinearly from that
    cell's eight corners, extrapolating where its vertices lie outside)."""
    nb = P.box_b + 1
    col = {g: j for j, g in enumerate(P.box_active)}
    nf = P.free.size
    Jt = np.zeros((nf, P.nr))
    Ar = np.zeros((P.nr, P.nr))
    cells = np.zeros((m.ne, 3), dtype=np.int64)
    cnt = np.bincount(m.conn.ravel(), minlength=m.nv)
    for e in range(m.ne):
        X = m.xyz[m.conn[e]]
        c = _cell_by_search(P, X.mean(axis=0))
        cells[e] = c
        Je = np.zeros((8, 8))
        cols = []
        for q in range(8):          # cell corner q = a + 2b + 4c
            bits = np.array([q & 1, (q >> 1) & 1, (q >> 2) & 1])
            cols.append(col.get(int((c[0] + bits[0]) + nb[0] * ((c[1] + bits[1]) + nb[1] * (c[2] + bits[2]))), -1))
            for k in range(8):
                t = (X[k] - (P.box_lo + c * P.box_H)) / P.box_H
                w = 1.0
                for d in range(3):
                    w *= t[d] if bits[d] else 1.0 - t[d]
                Je[k, q] = 0.0 if P.dir[m.conn[e, k]] else w
        Ke = Je.T @ P.Ae[e] @ Je
        for q in range(8):
            if cols[q] < 0:
                continue
            for k in range(8):
                v = m.conn[e, k]
                if not P.dir[v]:
                    Jt[P.free_pos[v], cols[q]] += Je[k, q] / cnt[v]
            for q2 in range(8):
                if cols[q2] >= 0:
                    Ar[cols[q], cols[q2]] += Ke[q, q2]
    return cells, Jt, Ar


@pytest.fixture(scope="module")
def perturbed4():
    m = meshes.cube(4, perturb=0.15, seed=0, boxes=(2, 2, 2))
    return m, O.Problem(m.xyz, m.conn, m.part, m.boxes)


def test_element_cells_follow_the_centroid(perturbed4):
    """Sec. 4 assigns each element to the box cell holding its centroid.  On
    this perturbed mesh the cell of an element's first vertex differs from
    its centroid's for some elements, so a rule that took any vertex's cell
    fails here; the reduced operator assembled from the searched cells equals
    the oracle's A_r."""
    m, P = perturbed4
    cells, Jt, Ar = _brute_force_coarse(P, m)
    np.testing.assert_array_equal(P.cell, cells)
    first = np.array([_cell_by_search(P, m.xyz[m.conn[e, 0]]) for e in range(m.ne)])
    assert (first != cells).any(axis=1).sum() >= 4
    np.testing.assert_allclose(P.Ar, Ar, rtol=0, atol=1e-13 * np.abs(Ar).max())


@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_preconditioner_matches_its_dense_formula(perturbed4, form):
    """M applied to every unit vector equals the matrix composed from dense
    factors (Sec. 3, Eqs. (3)-(5); Sec. 4, J~ = W Q^T J_L):
      additive  sum_p R_p^T A_p^{-1} R_p + J~ A_r^{-1} J~^T
      hybrid    M_1 + J~ A_r^{-1} J~^T (I - A M_1),  M_1 = W_ov sum_p R_p^T A_p^{-1} R_p
    with R_p the selection matrices of the subdomain index sets, W_ov their
    inverse multiplicities, and J~ and A_r from the element-by-element
    construction."""
    m, P = perturbed4
    _, Jt, Ar = _brute_force_coarse(P, m)
    A = P.A.toarray()
    nf = P.free.size
    S = np.zeros((nf, nf))
    mult = np.zeros(nf)
    for idx in P.sub_idx:
        R = np.zeros((idx.size, nf))
        R[np.arange(idx.size), P.free_pos[idx]] = 1.0
        S += R.T @ np.linalg.inv(R @ A @ R.T) @ R
        mult += R.sum(axis=0)
    B = Jt @ np.linalg.inv(Ar) @ Jt.T
    if form == "additive":
        ref = S + B
    else:
        M1 = np.diag(1.0 / mult) @ S
        ref = M1 + B @ (np.eye(nf) - A @ M1)
    M = _dense_M(P, form)
    assert np.abs(M - ref).max() <= 1e-13 * np.abs(ref).max()


def test_additive_preconditioner_symmetric_positive_definite():
    m = meshes.cube(4, perturb=0.15, seed=0, boxes=(2, 2, 2))
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    M = _dense_M(P, "additive")
    assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_single_subdomain_hybrid_is_exact():
    m = meshes.cube(4, perturb=0.15, seed=0, boxes=(2, 2, 2))
    part = np.zeros(m.ne, dtype=np.int32)
    P = O.Problem(m.xyz, m.conn, part, m.boxes)
    r = np.where(P.dir, 0.0, np.random.default_rng(8).standard_normal(m.nv))
    exact = P.to_full(np.linalg.solve(P.A.toarray(), r[P.free]))
    np.testing.assert_allclose(P.apply_M(r, "hybrid"), exact, atol=1e-12)
    x, its, relres, ok = P.solve(r, rtol=1e-12)
    assert ok and its == 1 and relres < 1e-12


@pytest.mark.parametrize("form", ["hybrid", "additive"])
def test_pcg_matches_dense_direct_solve(form):
    m, b = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    x, its, relres, ok = P.solve(b, rtol=1e-13, form=form)
    exact = P.to_full(np.linalg.solve(P.A.toarray(), b[P.free]))
    assert ok and relres < 1e-12
    assert np.linalg.norm(x - exact) / np.linalg.norm(exact) < 1e-11


def test_zero_rhs_gives_zero_solution():
    m, _ = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    x, its, relres, ok = P.solve(np.zeros(m.nv))
    assert ok and its == 0 and not x.any()


@pytest.mark.parametrize("n", [8, 16])
def test_both_halves_needed_and_hybrid_beats_additive(n):
    """Sec. 5: ASM_2 needs both the local and the box part; Sec. 3: the
    multiplicative form takes fewer iterations than the additive one."""
    m = meshes.cube(n, perturb=0.15, seed=0, boxes=(n // 2,) * 3 if n == 8 else (8, 8, 8))
    b = meshes.rhs(m.nv, 1)
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    its = {f: P.solve(b, 1e-8, maxit=400, form=f) for f in ("hybrid", "additive", "local", "box")}
    assert its["hybrid"][3] and its["additive"][3] and its["local"][3]
    assert not its["box"][3]
    assert its["hybrid"][1] < its["additive"][1]
    assert its["hybrid"][1] < its["local"][1]


def test_flexible_cg_equals_textbook_pcg_for_symmetric_preconditioner():
    """With a symmetric M the Polak-Ribiere beta of flexible CG equals the
    Fletcher-Reeves beta of textbook PCG in exact arithmetic, so the iterates
    agree to rounding; a wrong beta or alpha breaks this."""
    m, b = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    bb = np.where(P.dir, 0.0, b)
    M = lambda r: P.apply_M(r, "additive")
    for k in (1, 2, 5, 8):
        x_f, its, _, _ = O.fcg(P.apply_A, M, bb, 0.0, k)
        assert its == k
        # textbook PCG (Hestenes-Stiefel with z = M r, beta = r1.z1 / r0.z0)
        x = np.zeros_like(bb)
        r = bb.copy()
        z = M(r)
        p = z.copy()
        rz = r @ z
        for _ in range(k):
            q = P.apply_A(p)
            a = rz / (p @ q)
            x += a * p
            r -= a * q
            z = M(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        np.testing.assert_allclose(x_f, x, rtol=1e-9, atol=1e-9 * np.abs(x).max())


# --------------------------------------------------------------------------
# XX^T reduced solver (Sec. 2: A_c-conjugate sparse basis, A_c^{-1} = X X^T)
# --------------------------------------------------------------------------

def _lattice_27(n):
    """Interior points of an (n+1)^3 unit box lattice and the assembled Q1
    27-point stencil on them (centre 8/3, face 0, edge -1/6, corner -1/12,
    the closed form of the unit-cube element assembled)."""
    pts = np.array([(i, j, k) for k in range(1, n) for j in range(1, n) for i in range(1, n)])
    index = {tuple(p): a for a, p in enumerate(pts)}
    w = {0: 8.0 / 3.0, 1: 0.0, 2: -1.0 / 6.0, 3: -1.0 / 12.0}
    A = np.zeros((len(pts), len(pts)))
    for a, p in enumerate(pts):
        for d in np.ndindex(3, 3, 3):
            q = tuple(p + np.array(d) - 1)
            if q in index:
                A[a, index[q]] = w[int(np.abs(np.array(d) - 1).sum())]
    return pts, A


@pytest.mark.parametrize("wl", ["cube8", "ragged"])
def test_xxt_basis_is_conjugate_and_solves(wl):
    if wl == "cube8":
        m, _ = meshes.workload_cube8()
    else:
        m = meshes.cube((5, 3, 7), perturb=0.15, seed=3, boxes=(3, 2, 3), name="ragged")
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    X = P.xxt_factor()
    assert np.abs(X.T @ P.Ar @ X - np.eye(P.nr)).max() <= 1e-12
    b = np.random.default_rng(9).standard_normal(P.nr)
    ref = np.linalg.solve(P.Ar, b)                   # dense LU, not the oracle's Cholesky
    assert np.abs(P.coarse_solve_xxt(b) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_xxt_natural_order_on_a_chain_is_inverse_cholesky_transpose():
    """Gram-Schmidt of the unit vectors in the A inner product, in natural
    order, is the textbook L^{-T} of A = L L^T (a tridiagonal chain)."""
    n = 40
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1) + 0.01 * np.eye(n)
    X = O.xxt_basis(A, np.arange(n))
    L = np.linalg.cholesky(A)
    assert np.allclose(X, np.linalg.inv(L).T, rtol=0, atol=1e-12)


def test_nested_dissection_separator_decouples_the_halves():
    """The first cut is a plane; vectors of the points below it vanish exactly
    on the points above it and on the plane, and vice versa below."""
    pts, A = _lattice_27(8)
    order = O.nested_dissection(pts)
    assert sorted(order.tolist()) == list(range(len(pts)))
    X = O.xxt_basis(A, order)
    # the top separator: the trailing points that share one coordinate plane
    ax = int(np.argmax(pts.max(0) - pts.min(0)))
    mid = np.unique(pts[:, ax])[len(np.unique(pts[:, ax])) // 2]
    below = np.flatnonzero(pts[:, ax] < mid)
    above = np.flatnonzero(pts[:, ax] > mid)
    sep = np.flatnonzero(pts[:, ax] == mid)
    nb, na = len(below), len(above)
    assert set(order[:nb]) == set(below) and set(order[nb:nb + na]) == set(above)
    assert set(order[nb + na:]) == set(sep)
    assert np.all(X[np.concatenate([above, sep])][:, :nb] == 0.0)
    assert np.all(X[np.concatenate([below, sep])][:, nb:nb + na] == 0.0)


def test_nested_dissection_keeps_x_sparse():
    """On a 9^3-point lattice the conjugate basis in nested-dissection order
    has under a quarter of the entries of a dense matrix; in lexicographic
    order it fills the whole upper triangle (L^{-T} of a banded matrix)."""
    pts, A = _lattice_27(10)
    n = len(pts)
    nd = np.count_nonzero(O.xxt_basis(A, O.nested_dissection(pts)))
    lex = np.count_nonzero(O.xxt_basis(A, np.arange(n)))
    assert nd < 0.25 * n * n
    assert lex > 0.45 * n * n


# --------------------------------------------------------------------------
# projection onto prior solutions (Sec. 5: solve for the change from the
# A-orthogonal best fit onto l prior solutions)
# --------------------------------------------------------------------------

def _direct(P, b):
    """Exact solution by a dense direct solve of the free block."""
    x = np.zeros(P.nv)
    x[P.free] = np.linalg.solve(P.A.toarray(), np.asarray(b)[P.free])
    return x


@pytest.fixture(scope="module")
def cube8_problem():
    m, _ = meshes.workload_cube8()
    return O.Problem(m.xyz, m.conn, m.part, m.boxes)


def test_projection_start_is_the_a_orthogonal_best_fit(cube8_problem):
    """u_bar equals U c with (U^T A U) c = U^T b, U the raw prior solutions
    (the normal equations of min ||u* - U c||_A, solved densely)."""
    P = cube8_problem
    rng = np.random.default_rng(12)
    proj = O.Projection(P.apply_A, 5)
    U = []
    for _ in range(4):
        u = _direct(P, np.where(P.dir, 0.0, rng.standard_normal(P.nv)))
        proj.add(u)
        U.append(u[P.free])
    U = np.array(U).T
    b = np.where(P.dir, 0.0, rng.standard_normal(P.nv))
    ubar, bp = proj.start(b)
    A = P.A.toarray()
    c = np.linalg.solve(U.T @ A @ U, U.T @ b[P.free])
    assert np.abs(ubar[P.free] - U @ c).max() <= 1e-10 * np.abs(U @ c).max()
    assert np.abs(bp - (b - P.apply_A(ubar))).max() <= 1e-10 * np.abs(b).max()


def test_projection_is_exact_for_a_combination_of_prior_right_hand_sides(cube8_problem):
    P = cube8_problem
    rng = np.random.default_rng(13)
    b1, b2 = (np.where(P.dir, 0.0, rng.standard_normal(P.nv)) for _ in range(2))
    proj = O.Projection(P.apply_A, 4)
    proj.add(_direct(P, b1))
    proj.add(_direct(P, b2))
    b = 0.3 * b1 - 1.7 * b2
    ubar, bp = proj.start(b)
    ref = _direct(P, b)
    assert np.abs(ubar - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.linalg.norm(bp) <= 1e-10 * np.linalg.norm(b)


def test_projection_basis_is_a_orthonormal_and_restarts(cube8_problem):
    P = cube8_problem
    rng = np.random.default_rng(14)
    proj = O.Projection(P.apply_A, 3)
    for k in range(3):
        proj.add(_direct(P, np.where(P.dir, 0.0, rng.standard_normal(P.nv))))
        X = np.array(proj.X)
        G = X @ np.array([P.apply_A(x) for x in proj.X]).T
        assert len(proj.X) == k + 1 and np.abs(G - np.eye(k + 1)).max() <= 1e-12
    proj.add(_direct(P, np.where(P.dir, 0.0, rng.standard_normal(P.nv))))
    assert len(proj.X) == 1                     # full basis restarts with the newest solution
    proj.add(2.0 * proj.X[0])                   # no new direction: not appended
    assert len(proj.X) == 1


def test_projected_sequence_converges_with_fewer_iterations(cube8_problem):
    P = cube8_problem
    rng = np.random.default_rng(3)
    b0, b1 = rng.standard_normal(P.nv), rng.standard_normal(P.nv)
    bs = [b0 + 0.05 * k * b1 for k in range(6)]
    res = O.solve_projected(P, bs, 3, rtol=1e-10)
    plain = [P.solve(b, rtol=1e-10)[1] for b in bs]
    assert res[0][1] == plain[0]                # empty basis: the plain solve
    assert all(r[1] <= p for r, p in zip(res, plain)) and sum(r[1] for r in res) < sum(plain)
    for (x, it, rel, _, _), b in zip(res, bs):
        ref = _direct(P, np.where(P.dir, 0.0, b))
        assert rel <= 5e-10 and np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max()


# --------------------------------------------------------------------------
# coarse-operator variants (Sec. 4): Galerkin J~^T A J~ and the vertex-based J
# --------------------------------------------------------------------------

def test_coarse_operators_coincide_on_box_aligned_mesh():
    """With element planes on box planes J_L is continuous: the cell-wise
    A_r (Eq. (12)), the Galerkin J~^T A J~ and the vertex-based J^T A J agree."""
    m = meshes.cube(8, boxes=(4, 2, 4))
    Ps = {op: O.Problem(m.xyz, m.conn, m.part, m.boxes, coarse_operator=op)
          for op in ("broken", "galerkin", "vertex")}
    ref = Ps["broken"]
    for op in ("galerkin", "vertex"):
        assert np.array_equal(Ps[op].box_active, ref.box_active)
        np.testing.assert_allclose(Ps[op].Ar, ref.Ar, atol=1e-13 * np.abs(ref.Ar).max())


def test_vertex_based_J_reproduces_trilinear_fields():
    """J u_r with u_r = f at the box vertices gives f at every free node for a
    trilinear f (Sec. 4: J interpolates box-vertex values to each node)."""
    m = meshes.cube(9, perturb=0.2, seed=5, boxes=(3, 4, 2))
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes, coarse_operator="vertex")
    c = np.random.default_rng(2).standard_normal(8)
    f = lambda X: (c[0] + c[1] * X[:, 0] + c[2] * X[:, 1] + c[3] * X[:, 2] + c[4] * X[:, 0] * X[:, 1]
                   + c[5] * X[:, 1] * X[:, 2] + c[6] * X[:, 0] * X[:, 2] + c[7] * X[:, 0] * X[:, 1] * X[:, 2])
    nb = P.box_b + 1
    g = P.box_active
    Xb = P.box_lo + np.stack([g % nb[0], (g // nb[0]) % nb[1], g // (nb[0] * nb[1])], axis=1) * P.box_H
    z = P.interp(f(Xb))
    ref = f(P.xyz)
    assert np.abs(z[P.free] - ref[P.free]).max() <= 1e-12 * np.abs(ref).max()
    assert np.all(z[P.dir] == 0.0)


@pytest.mark.parametrize("op", ["galerkin", "vertex"])
def test_full_support_variants_have_the_wider_stencil(op):
    """On a perturbed mesh the cell-wise assembly keeps 3^3 = 27 nonzeros per
    row; the full-support operators reach up to 5^3 = 125 (Sec. 4)."""
    m, _ = meshes.workload_cube8()
    Pb = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    Pv = O.Problem(m.xyz, m.conn, m.part, m.boxes, coarse_operator=op)
    nz = lambda A: (np.abs(A) > 1e-14 * np.abs(A).max()).sum(axis=1)
    assert nz(Pb.Ar).max() <= 27
    assert 27 < nz(Pv.Ar).max() <= 125
    np.testing.assert_allclose(Pv.Ar, Pv.Ar.T, atol=1e-14 * np.abs(Pv.Ar).max())
    assert np.linalg.eigvalsh(Pv.Ar).min() > 0.0
    # the reduced solve and restriction are each other's transposes
    rng = np.random.default_rng(6)
    s, u = rng.standard_normal(m.nv), rng.standard_normal(Pv.nr)
    s[Pv.dir] = 0.0
    assert abs(Pv.restrict(s) @ u - s @ Pv.interp(u)) <= 1e-12 * np.abs(s).sum() * np.abs(u).max()


# --------------------------------------------------------------------------
# wrappers and local variants (Sec. 3 RAS, Sec. 5 boundary conditions,
# Sec. 6 inexact local solves; the Schwarz-Richardson and GMRES wrappers)
# --------------------------------------------------------------------------

def test_ras_without_overlap_equals_the_additive_local_sum():
    m, _ = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes, overlap=0)
    r = np.random.default_rng(21).standard_normal(m.nv)
    np.testing.assert_allclose(P.local_solves(r, "ras"), P.local_solves(r, False), rtol=0, atol=1e-14)


def test_ras_prolongation_is_a_partition_of_unity():
    """With overlap the restricted prolongations sum to one at every free
    node, and a single subdomain gives A^{-1} r."""
    m, _ = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    tot = np.zeros(m.nv)
    for mm, (ps, I, Ap, L) in P.groups.items():
        np.add.at(tot, I.ravel(), P.ras_w[mm].ravel())
    assert np.allclose(tot[P.free], 1.0, rtol=0, atol=1e-15)
    one = O.Problem(m.xyz, m.conn, np.zeros(m.ne, int), m.boxes)
    r = np.random.default_rng(22).standard_normal(m.nv)
    x = np.zeros(m.nv)
    x[one.free] = np.linalg.solve(one.A.toarray(), r[one.free])
    np.testing.assert_allclose(one.local_solves(r, "ras"), x, rtol=0, atol=1e-12 * np.abs(x).max())


def test_inexact_local_solves():
    """m_p CG steps solve each local system (to rounding); two steps do not."""
    m, _ = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    r = np.random.default_rng(23).standard_normal(m.nv)
    exact = P.local_solves(r, True)
    full = P.local_solves(r, True, inner=max(P.groups))
    assert np.abs(full - exact).max() <= 1e-9 * np.abs(exact).max()
    assert np.abs(P.local_solves(r, True, inner=2) - exact).max() > 1e-3 * np.abs(exact).max()
    # the same inner steps inside every form of M (Sec. 6): m_p steps give the
    # exact preconditioner
    k = max(P.groups)
    for form in ("hybrid", "additive", "ras"):
        ex = P.apply_M(r, form)
        assert np.abs(P.apply_M(r, form, inner=k) - ex).max() <= 1e-9 * np.abs(ex).max()


def test_schwarz_richardson_converges_at_the_spectral_radius():
    """x += M (b - A x) with the hybrid M: the fixed point is A^{-1} b, and the
    residual shrinks at the spectral radius of I - M A (dense eigenvalues)."""
    m, b = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    bb = np.where(P.dir, 0.0, b)
    x, it, rel, ok = O.richardson(P.apply_A, P.apply_M, bb, 1e-10, 200)
    ref = _direct(P, bb)
    assert ok and np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max()
    n = P.free.size
    E = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(P.nv)
        e[P.free[j]] = 1.0
        E[:, j] = e[P.free] - P.apply_M(P.apply_A(e))[P.free]
    rho = np.abs(np.linalg.eigvals(E)).max()
    assert rho < 1.0
    # iterations needed for 1e-10 agree with the rate within a few steps
    assert abs(it - np.log(1e-10) / np.log(rho)) <= 0.25 * it + 3


def test_fgmres_minimises_the_residual_over_the_krylov_space():
    """Without a preconditioner, k steps give the least-squares minimum of
    ||b - A x|| over span{b, A b, ..., A^{k-1} b} (formed densely)."""
    m, b = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    bb = np.where(P.dir, 0.0, b)
    k = 6
    x, it, rel, ok = O.fgmres(P.apply_A, lambda v: v.copy(), bb, 1e-30, k, restart=k)
    A = P.A.toarray()
    K = [bb[P.free]]
    for _ in range(k - 1):
        K.append(A @ K[-1])
    Q, _ = np.linalg.qr(np.array(K).T)
    c, *_ = np.linalg.lstsq(A @ Q, bb[P.free], rcond=None)
    best = np.linalg.norm(bb[P.free] - A @ (Q @ c)) / np.linalg.norm(bb)
    assert it == k and abs(rel - best) <= 1e-9 * best


def test_fgmres_with_schwarz_matches_direct_and_pcg():
    m, b = meshes.workload_cube8()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    bb = np.where(P.dir, 0.0, b)
    ref = _direct(P, bb)
    for form in ("hybrid", "ras"):
        x, it, rel, ok = O.fgmres(P.apply_A, lambda r: P.apply_M(r, form), bb, 1e-10, 200)
        assert ok and np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max()
    # inexact local solves need the flexible outer iteration
    x, it, rel, ok = O.fgmres(P.apply_A, lambda r: P.local_solves(r, True, inner=3) + P.box_correction(r),
                              bb, 1e-10, 300)
    assert ok and np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max()


def test_outflow_dirichlet_problem():
    """Neumann everywhere except the outflow cap (Sec. 5): A stays SPD, the
    box functions inherit the condition through J (zero rows at the cap),
    and the hybrid PCG solve matches the dense solve."""
    m, b = meshes.workload_cylinder(scale=8)
    d = meshes.outflow_dirichlet(m).astype(bool)
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes, dirichlet=d)
    assert d.sum() > 0 and P.free.size == m.nv - d.sum()
    assert np.linalg.eigvalsh(P.A.toarray()).min() > 0.0
    u = np.random.default_rng(7).standard_normal(P.nr)
    assert np.all(P.interp(u)[d] == 0.0)
    bb = np.where(d, 0.0, b)
    ref = _direct(P, bb)
    x, it, rel, ok = P.solve(bb, rtol=1e-10, maxit=1000, form="additive")
    assert ok and rel <= 2e-10 and np.abs(x - ref).max() <= 1e-7 * np.abs(ref).max()
    # the weighted hybrid form converges too, far more slowly on this 2^3-box
    # space (about 1,500 products against about 250)
    x, it2, rel, ok = P.solve(bb, rtol=1e-10, maxit=3000)
    assert ok and it2 > it and np.abs(x - ref).max() <= 1e-7 * np.abs(ref).max()
