"""FP64 CPU oracle of the p-multigrid wrap around the coarse-grid solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or calls this
module; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` use it.  It shares no code with the CUDA path.

What it computes (paper notation, Sec. 1 and Sec. 5):

* spectral elements of order N on the hexahedral mesh: Gauss-Lobatto-Legendre
  (GLL) nodes xi_0..xi_N per direction, element-local values u^e_ijk in
  lexicographic order (i fastest, Sec. 1), the element geometry given by the
  trilinear map of the hexahedron's 8 vertices;
* the SEM Poisson operator A_N = Q^T A_L Q with A^e = Dhat^T G^e Dhat, the
  quadrature at the GLL nodes themselves (the diagonal-mass SEM rule), G^e the
  metric w_q det J (J^-1 J^-T) at every node, Q the global-to-local map;
* interpolation between orders (the J_3, J_1 of Eq. (13)): element-wise
  tensor-product Lagrange interpolation from the coarse order's GLL nodes to
  the fine order's, J = W_f Q_f^T I Q_c, and its transpose;
* the element-local additive Schwarz smoother of Eq. (14),
  M_N^-1 = W_N sum_e R_{N,e}^T A~_{N,e}^-1 R_{N,e}, with A~ the separable
  (fast-diagonalisation) approximation of the element problem;
* the additive multilevel preconditioner of Eq. (13) for a schedule of orders
  N_0 > N_1 > ... > 1, whose N = 1 level is one application of the two-level
  Schwarz preconditioner (``cgs_oracle.Problem.apply_M``) on the hexahedral
  mesh itself: the coarse problem needs no exact solve inside a Krylov method
  (Sec. 3, opening paragraph), so a single sweep stands for M_1^-1;
* flexible GMRES on A_N x = b with that preconditioner (Sec. 5).

Readings where the paper is silent (it defers the smoother and the
fast-diagonalisation details to its references):

* geometry: the SEM element is the trilinear image of its 8 vertices (the
  meshes carry no curved-element data);
* Dirichlet nodes: every node on a boundary face (a face owned by one
  element), as the coarse problem's default;
* R_{N,e} extracts the element's own (N+1)^3 nodes (neighbouring elements
  overlap on the shared faces); A~_{N,e} = B_z(x)B_y(x)A_x + B_z(x)A_y(x)B_x +
  A_z(x)B_y(x)B_x with 1D factors on the element's nodes from a 1D SEM mesh
  of three equal elements (the element and one neighbour of the same length
  on either side), the unknowns beyond the element held at zero: the 1D
  stiffness and mass of the element with the neighbour's corner entry added at
  each shared end; the length of direction d is the mean length of the
  element's four edges along d; a side on a Dirichlet face drops its end node
  instead (no neighbour term);
* W_N = 1 / (number of elements holding the node);
* the schedule 7 -> 3 -> 1 (NekRS, Sec. 5) unless given.

Every function here is pinned by tests under ``tests/`` against closed forms,
invariants or brute force; none is "parity unpinned".
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cgs_oracle as CO

# hexahedron vertex k = a + 2b + 4c sits at the corner (a, b, c) of [-1, 1]^3
_CORNERS = np.array([[(k >> d) & 1 for d in range(3)] for k in range(8)])
# vertex pairs of the four edges along each reference direction
_EDGES = [[(k, k | (1 << d)) for k in range(8) if not (k >> d) & 1] for d in range(3)]


# ----------------------------------------------------------------------------
# One dimension: GLL nodes and weights, differentiation, interpolation
# ----------------------------------------------------------------------------

def legendre(n: int, x):
    """P_n(x) and P_n'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    # (1 - x^2) P_n' = n (P_{n-1} - x P_n), away from the endpoints
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    end = np.abs(np.abs(x) - 1.0) < 1e-15
    dp = np.where(end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gll(n: int):
    """GLL nodes (ascending) and weights of order n >= 1: the endpoints and the
    roots of P_n'; w_i = 2 / (n (n + 1) P_n(x_i)^2)."""
    if n < 1:
        raise ValueError("order >= 1")
    x = -np.cos(np.pi * np.arange(n + 1) / n)          # Chebyshev-Lobatto start
    interior = x[1:-1].copy()
    for _ in range(100):
        # Newton on q(x) = P_n'(x), with q' from the Legendre equation
        # (1 - x^2) P_n'' = 2 x P_n' - n (n + 1) P_n
        p, dp = legendre(n, interior)
        d2p = (2.0 * interior * dp - n * (n + 1) * p) / (1.0 - interior ** 2)
        step = dp / d2p
        interior = interior - step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    x[1:-1] = interior
    x[0], x[-1] = -1.0, 1.0
    x = 0.5 * (x - x[::-1])                            # exact symmetry
    p, _ = legendre(n, x)
    w = 2.0 / (n * (n + 1) * p ** 2)
    return x, w


def barycentric_weights(x):
    return np.array([1.0 / np.prod([x[j] - x[k] for k in range(len(x)) if k != j]) for j in range(len(x))])


def derivative_matrix(x):
    """D[i, j] = l_j'(x_i) for the Lagrange basis on the nodes x (barycentric
    form; the diagonal makes every row sum to zero)."""
    b = barycentric_weights(x)
    n = len(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (b[j] / b[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i])
    return D


def interpolation_matrix(xc, xf):
    """I[i, j] = l_j(xf_i): values at the points xf of the Lagrange basis on
    the nodes xc."""
    I = np.ones((len(xf), len(xc)))
    for j in range(len(xc)):
        for k in range(len(xc)):
            if k != j:
                I[:, j] *= (xf - xc[k]) / (xc[j] - xc[k])
    return I


# ----------------------------------------------------------------------------
# Tensor products on element-local arrays u[e, k, j, i] (i fastest)
# ----------------------------------------------------------------------------

def apply_1d(M, u, axis):
    """Apply the matrix M along one reference direction (0 = i, 1 = j, 2 = k)
    of u[..., k, j, i]; M may be one matrix or one per element."""
    sub = {0: "i", 1: "j", 2: "k"}[axis]
    src = "ekji".replace(sub, "m")
    dst = "ekji"
    if M.ndim == 2:
        return np.einsum(f"{sub}m,{src}->{dst}", M, u)
    return np.einsum(f"e{sub}m,{src}->{dst}", M, u)


# ----------------------------------------------------------------------------
# The SEM discretisation of order N on a hexahedral mesh
# ----------------------------------------------------------------------------

class Level:
    """Spectral elements of order n on the mesh (xyz, conn)."""

    def __init__(self, xyz, conn, n: int):
        self.n = n
        self.p = n + 1
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.ne = self.conn.shape[0]
        self.x, self.w = gll(n)
        self.D = derivative_matrix(self.x)
        self._numbering()
        self._geometry()
        self._dirichlet()
        self.mult = np.bincount(self.l2g.ravel(), minlength=self.ng).astype(np.float64)

    # -- global numbering (the Q of Sec. 3) ------------------------------------
    def _numbering(self):
        """Nodes shared between elements get one global number.  The key of a
        node is its set of (hexahedron vertex, integer trilinear weight)
        pairs: along each direction the node with GLL index i has the integer
        weights (n - i, i) on the two ends, so the weight of vertex (a, b, c)
        is the product of the three factors.  The key does not depend on the
        element it is seen from (it is the node's position on the shared face,
        edge or vertex in integer form)."""
        n, p, ne = self.n, self.p, self.ne
        i = np.arange(p)
        ii = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1)[..., ::-1].reshape(-1, 3)  # (p^3, 3): (i, j, k)
        codes = np.ones((p ** 3, 8), dtype=np.int64)
        for v in range(8):
            for d in range(3):
                codes[:, v] *= np.where(_CORNERS[v, d] == 1, ii[:, d], n - ii[:, d])
        # per (element, node): vertex ids with their weights, zero weights as (-1, 0)
        vid = np.broadcast_to(self.conn[:, None, :], (ne, p ** 3, 8))
        cw = np.broadcast_to(codes[None], (ne, p ** 3, 8))
        vid = np.where(cw > 0, vid, -1)
        # sort each node's pairs by vertex id so the key is order-free
        order = np.argsort(vid, axis=2, kind="stable")
        vid = np.take_along_axis(vid, order, 2)
        cw = np.take_along_axis(cw, order, 2)
        keys = np.concatenate([vid, cw], axis=2).reshape(ne * p ** 3, 16)
        uniq, inv = np.unique(keys, axis=0, return_inverse=True)
        self.ng = uniq.shape[0]
        self.l2g = inv.reshape(ne, p, p, p)           # [e, k, j, i]

    # -- geometry: trilinear map, its Jacobian and the metric at GLL nodes ----
    def _geometry(self):
        x, p = self.x, self.p
        X = self.xyz[self.conn]                        # (E, 8, 3)
        # trilinear shape functions and their reference gradients at the nodes
        xi = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)[..., ::-1]   # [k, j, i, (r, s, t)]
        f = [(1 - xi) / 2, (1 + xi) / 2]
        phi = np.empty((p, p, p, 8))
        dphi = np.empty((p, p, p, 8, 3))
        for v in range(8):
            a = [f[_CORNERS[v, d]][..., d] for d in range(3)]
            phi[..., v] = a[0] * a[1] * a[2]
            for d in range(3):
                s = 0.5 if _CORNERS[v, d] else -0.5
                o = [a[m] for m in range(3) if m != d]
                dphi[..., v, d] = s * o[0] * o[1]
        self.coords = np.einsum("kjiv,evc->ekjic", phi, X)            # (E, p, p, p, 3)
        J = np.einsum("kjiva,evc->ekjica", dphi, X)                    # J[c, a] = dx_c / dxi_a
        self.detJ = np.linalg.det(J)
        if not self.detJ.min() > 0.0:
            raise ValueError("element with non-positive Jacobian")
        Jinv = np.linalg.inv(J)                                        # [a, c] = dxi_a / dx_c
        wq = self.w[:, None, None] * self.w[None, :, None] * self.w[None, None, :]   # [k, j, i]
        self.G = (wq[None] * self.detJ)[..., None, None] * np.einsum("ekjiac,ekjibc->ekjiab", Jinv, Jinv)
        self.mass = wq[None] * self.detJ                               # diagonal of B^e

    # -- Dirichlet nodes: every node of a boundary face -----------------------
    def _dirichlet(self):
        faces = [[v for v in range(8) if _CORNERS[v, d] == s] for d in range(3) for s in range(2)]
        keyset = {}
        for e in range(self.ne):
            for fi, fv in enumerate(faces):
                keyset.setdefault(tuple(sorted(self.conn[e, fv])), []).append((e, fi))
        self.face_bdry = np.zeros((self.ne, 6), dtype=bool)             # [e, 2 d + side]
        for owners in keyset.values():
            if len(owners) == 1:
                e, fi = owners[0]
                self.face_bdry[e, fi] = True
        self.dir = np.zeros(self.ng, dtype=bool)
        p = self.p
        for e, fi in zip(*np.nonzero(self.face_bdry)):
            d, s = divmod(fi, 2)
            sl = [slice(None)] * 3
            sl[2 - d] = p - 1 if s else 0                               # axis order k, j, i
            self.dir[self.l2g[e][tuple(sl)].ravel()] = True

    # -- vectors --------------------------------------------------------------
    def gather(self, u):
        """Q u: element-local copies, (E, p, p, p)."""
        return np.asarray(u, dtype=np.float64)[self.l2g]

    def scatter(self, uL):
        """Q^T u_L: sum of element-local copies into the global numbering."""
        return np.bincount(self.l2g.ravel(), weights=uL.ravel(), minlength=self.ng)

    def mask(self, u):
        return np.where(self.dir, 0.0, u)

    # -- the operator (Sec. 1: A^e = Dhat^T G Dhat at the GLL quadrature) -----
    def local_apply(self, uL):
        g = [apply_1d(self.D, uL, a) for a in range(3)]                # du/dr, du/ds, du/dt
        y = np.zeros_like(uL)
        for a in range(3):
            wa = sum(self.G[..., a, b] * g[b] for b in range(3))
            y += apply_1d(self.D.T, wa, a)
        return y

    def apply_A(self, u):
        """y = A_N u with Dirichlet nodes held at zero on input and output."""
        return self.mask(self.scatter(self.local_apply(self.gather(self.mask(u)))))

    def node_coords(self):
        """Coordinates of every global node (from its first element copy)."""
        out = np.zeros((self.ng, 3))
        out[self.l2g.ravel()] = self.coords.reshape(-1, 3)
        return out


# ----------------------------------------------------------------------------
# Interpolation between orders (the J_3, J_1 of Eq. (13))
# ----------------------------------------------------------------------------

class Transfer:
    """J from the coarse level to the fine level of the same mesh:
    J = W_f Q_f^T I Q_c with I the element-wise tensor-product interpolation."""

    def __init__(self, fine: Level, coarse: Level):
        self.f, self.c = fine, coarse
        self.I = interpolation_matrix(coarse.x, fine.x)               # (pf, pc)

    def interp_local(self, uL):
        for a in range(3):
            uL = apply_1d(self.I, uL, a)
        return uL

    def restrict_local(self, rL):
        for a in range(3):
            rL = apply_1d(self.I.T, rL, a)
        return rL

    def prolong(self, uc):
        """J u_c: every fine node takes the (weighted mean of the) values its
        element copies interpolate."""
        fL = self.interp_local(self.c.gather(self.c.mask(uc)))
        return self.f.mask(self.f.scatter(fL) / self.f.mult)

    def restrict(self, rf):
        """J^T r_f = Q_c^T I^T Q_f W_f r_f."""
        rL = self.f.gather(self.f.mask(rf) / self.f.mult)
        return self.c.mask(self.c.scatter(self.restrict_local(rL)))


# ----------------------------------------------------------------------------
# The element-local Schwarz smoother of Eq. (14), fast diagonalisation
# ----------------------------------------------------------------------------

def element_lengths(xyz, conn):
    """(E, 3): mean length of the four edges along each reference direction."""
    X = np.asarray(xyz)[np.asarray(conn)]
    L = np.zeros((X.shape[0], 3))
    for d in range(3):
        L[:, d] = np.mean([np.linalg.norm(X[:, b] - X[:, a], axis=1) for a, b in _EDGES[d]], axis=0)
    return L


def extended_1d(n: int, length: float, lo_dirichlet: bool, hi_dirichlet: bool):
    """1D stiffness and mass of the element's n + 1 nodes inside a line of three
    equal elements whose outer unknowns are held at zero: the element's own
    matrices plus the neighbour's corner entry at each shared end.  A side on
    a Dirichlet face has no neighbour and its end node is dropped.  Returns
    (A, B, keep) with keep the retained node indices."""
    x, w = gll(n)
    D = derivative_matrix(x)
    Ahat = D.T @ np.diag(w) @ D
    A = (2.0 / length) * Ahat
    B = (length / 2.0) * np.diag(w)
    keep = list(range(n + 1))
    if lo_dirichlet:
        keep.remove(0)
    else:
        A[0, 0] += (2.0 / length) * Ahat[n, n]
        B[0, 0] += (length / 2.0) * w[n]
    if hi_dirichlet:
        keep.remove(n)
    else:
        A[n, n] += (2.0 / length) * Ahat[0, 0]
        B[n, n] += (length / 2.0) * w[0]
    return A, B, keep


class Smoother:
    """M_N^-1 = W_N sum_e R_e^T A~_e^-1 R_e (Eq. (14)) by fast diagonalisation:
    A~_e^-1 = S (Lx + Ly + Lz)^-1 S^T with S = S_z (x) S_y (x) S_x and, per
    direction, A_d S_d = B_d S_d L_d, S_d^T B_d S_d = I on the kept nodes (the
    rows of dropped Dirichlet nodes and the columns of their modes are zero)."""

    def __init__(self, lev: Level):
        self.lev = lev
        n, p, ne = lev.n, lev.p, lev.ne
        L = element_lengths(lev.xyz, lev.conn)
        self.S = np.zeros((ne, 3, p, p))
        self.lam = np.ones((ne, 3, p))
        for e in range(ne):
            for d in range(3):
                A, B, keep = extended_1d(n, L[e, d], lev.face_bdry[e, 2 * d], lev.face_bdry[e, 2 * d + 1])
                lam, S = sla.eigh(A[np.ix_(keep, keep)], B[np.ix_(keep, keep)])
                self.S[e, d][np.ix_(keep, range(len(keep)))] = S
                self.lam[e, d, :len(keep)] = lam

    def local_solve(self, rL):
        """A~_e^-1 r_e for every element."""
        u = rL
        for a in range(3):
            u = apply_1d(np.transpose(self.S[:, a], (0, 2, 1)), u, a)   # S^T
        lam = (self.lam[:, 2][:, :, None, None] + self.lam[:, 1][:, None, :, None]
               + self.lam[:, 0][:, None, None, :])
        u = u / lam
        for a in range(3):
            u = apply_1d(self.S[:, a], u, a)
        return u

    def apply(self, r):
        lev = self.lev
        uL = self.local_solve(lev.gather(lev.mask(r)))
        return lev.mask(lev.scatter(uL) / lev.mult)


# ----------------------------------------------------------------------------
# The multilevel preconditioner of Eq. (13) and the outer GMRES
# ----------------------------------------------------------------------------

class PMG:
    """z = M_{N0}^-1 r + J_1 (M_{N1}^-1 r_1 + J_2 (... + J_c M_c J_c^T ...)),
    r_{l+1} = J_{l+1}^T r_l, additive between levels (Eq. (13)); the last
    level is order 1 (the hexahedral mesh's vertices), where M_c is one
    application of the two-level Schwarz preconditioner."""

    def __init__(self, xyz, conn, part, boxes, orders=(7, 3), coarse_form: str = "hybrid"):
        if list(orders) != sorted(orders, reverse=True) or orders[-1] <= 1:
            raise ValueError("orders must decrease and stay above 1")
        self.levels = [Level(xyz, conn, n) for n in orders] + [Level(xyz, conn, 1)]
        self.smoothers = [Smoother(l) for l in self.levels[:-1]]
        self.transfers = [Transfer(self.levels[i], self.levels[i + 1]) for i in range(len(orders))]
        self.coarse = CO.Problem(xyz, conn, part, boxes)
        self.coarse_form = coarse_form
        # the order-1 level's nodes are the mesh vertices: map its numbering to
        # the vertex numbering the coarse problem uses
        c = self.levels[-1]
        self.c2v = np.zeros(c.ng, dtype=np.int64)
        self.c2v[c.l2g.reshape(c.ne, 8)] = np.asarray(conn)
        self.fine = self.levels[0]
        self._exact = None

    def coarse_apply(self, rc):
        """M_c on an order-1 level vector (Sec. 3: one sweep, not a solve)."""
        rv = np.zeros(self.coarse.nv)
        rv[self.c2v] = rc
        if self.coarse_form == "exact":                 # A_c^-1 itself, for comparison
            if self._exact is None:
                self._exact = spla.factorized(sp.csc_matrix(self.coarse.A))
            zv = self.coarse.to_full(self._exact(self.coarse.to_free(rv)))
        else:
            zv = self.coarse.apply_M(rv, self.coarse_form)
        return self.levels[-1].mask(zv[self.c2v])

    def apply_M(self, r):
        def level(i, r_i):
            if i == len(self.levels) - 1:
                return self.coarse_apply(r_i)
            z = self.smoothers[i].apply(r_i)
            T = self.transfers[i]
            return z + T.prolong(level(i + 1, T.restrict(r_i)))
        return level(0, self.fine.mask(r))

    def apply_A(self, u):
        return self.fine.apply_A(u)

    def solve(self, b, rtol: float = 1e-8, maxit: int = 300, restart: int = 30):
        """Flexible GMRES(restart) from x = 0 (Sec. 5: GMRES on the pressure
        with the p-multigrid preconditioner).  Returns (x, products A z,
        relres, converged)."""
        return CO.fgmres(self.apply_A, self.apply_M, self.fine.mask(b), rtol, maxit, restart)
