"""FP64 CPU oracle of the two-level Schwarz coarse-grid solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or calls this
module; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` use it.  It shares no code with the CUDA path: every step below is
written out again from the paper ("Coarse Solvers for Exascale Solution of
Poisson Problems", Sec. 3 and Sec. 4) in plain numpy/scipy, in float64, with no
blocking, fusion or reordering beyond what the definitions state.

What it computes (paper notation; the coarse system A_c u_c = b_c is written
A u = b, Sec. 3):

* element matrices a^e_ij = int grad l_i . grad l_j dV of trilinear hexes
  (Sec. 3, the equation defining a^e_ij), 2x2x2 Gauss-Legendre quadrature;
* assembly A = Q^T A_L Q (Sec. 3) restricted to the free (non-Dirichlet) dofs;
* overlapping subdomains: Omega_p grown by delta element layers, R_p the free
  nodes interior to the grown subdomain, A_p = R_p A R_p^T (Sec. 3);
* the box coarse space (Sec. 4): bounding box split into b_x*b_y*b_z cells,
  each element assigned to the cell holding its centroid, element-local
  trilinear interpolant J_L, averaging W Q^T (Sec. 4, the centroid-assignment
  paragraph), active-vertex compression, and A_r assembled cell-wise (Eq. (12));
* three coarse operators (Sec. 4): the cell-wise A_r of Eq. (12) (default),
  the Galerkin J~^T A J~ of the averaged interpolant, and the vertex-based J
  (each node in the box cell holding it) with A_r = J^T A J;
* the reduced solve exactly (Cholesky) and by XX^T (Sec. 2): A_r-conjugate
  basis vectors formed by Gram-Schmidt in the A_r inner product, in a
  nested-dissection order of the box lattice;
* the preconditioners ASM (Eq. (3)) and the hybrid ASM_1 + ASM_2 (Eqs. (4)
  and (5));
* variants and wrappers for the next steps: restricted additive Schwarz
  (Sec. 3, R~_p without the grown part), inexact local solves by a fixed
  number of CG steps (Sec. 6), Schwarz-Richardson and flexible GMRES
  wrappers, and any Dirichlet set (Neumann except an outflow cap, Sec. 5);
* repeated right-hand sides (Sec. 5, the projection onto prior solutions):
  the start is the A-orthogonal best fit onto up to l earlier solutions and
  the iteration solves for the change;
* flexible preconditioned CG around them.

Readings taken where the paper is silent or ambiguous (listed with the design
notes): 2x2x2 Gauss; Dirichlet = vertices of boundary faces; delta = 1 layer
of vertex-sharing elements; R_p = free vertices whose elements all lie in the
grown subdomain; W_ov = 1/multiplicity for the hybrid local step, no weight in
the additive form; J^T (not J) in the coarse term; A_r by broken (cell-wise)
assembly with Dirichlet rows of J_e zeroed; Polak-Ribiere beta; nested
dissection by median coordinate planes of the longest extent; the projection
basis restarts from the newest solution once it holds l vectors.

Every function here is pinned by tests under ``tests/`` against closed forms,
invariants or brute force; none is "parity unpinned".
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# 2-point Gauss-Legendre on [-1, 1]: nodes +-1/sqrt(3), weights 1.
_G = 1.0 / np.sqrt(3.0)
# corner signs of the reference hexahedron, local vertex k = a + 2b + 4c
_SIGNS = np.array([[2 * (k & 1) - 1, 2 * ((k >> 1) & 1) - 1, 2 * ((k >> 2) & 1) - 1]
                   for k in range(8)], dtype=np.float64)
# the six faces of a hexahedron as local vertex sets
_FACES = [[k for k in range(8) if ((k >> d) & 1) == s] for d in range(3) for s in range(2)]


# ----------------------------------------------------------------------------
# Element level (Sec. 3: a^e_ij = int_{Omega^e} grad l_i . grad l_j dV)
# ----------------------------------------------------------------------------

def reference_gradients(xi: np.ndarray) -> np.ndarray:
    """Gradients d l_k / d xi_a of the 8 trilinear Lagrange basis functions
    l_k(xi) = prod_d (1 + s_kd xi_d)/8 at one point xi of [-1,1]^3; (8, 3)."""
    f = 1.0 + _SIGNS * xi[None, :]          # (8,3) factors (1 + s xi)
    g = np.empty((8, 3))
    for a in range(3):
        others = [d for d in range(3) if d != a]
        g[:, a] = _SIGNS[:, a] * f[:, others[0]] * f[:, others[1]] / 8.0
    return g


def element_matrices(xyz: np.ndarray, conn: np.ndarray):
    """Stiffness matrices A^e (E, 8, 8) of the isoparametric trilinear map and
    the smallest Jacobian determinant seen at a quadrature point."""
    X = xyz[conn]                            # (E, 8, 3) vertex coordinates
    A = np.zeros((conn.shape[0], 8, 8))
    min_det = np.inf
    for q in range(8):
        xi = np.array([_G if (q >> d) & 1 else -_G for d in range(3)])
        G = reference_gradients(xi)          # (8, 3)
        J = np.einsum("ekd,ka->eda", X, G)   # J[d, a] = dx_d / dxi_a
        det = np.linalg.det(J)
        min_det = min(min_det, float(det.min()) if det.size else np.inf)
        Jinv = np.linalg.inv(J)              # Jinv[a, d] = dxi_a / dx_d
        grad = np.einsum("ka,ead->ekd", G, Jinv)
        A += det[:, None, None] * np.einsum("eid,ejd->eij", grad, grad)
    return A, min_det


# ----------------------------------------------------------------------------
# Global level
# ----------------------------------------------------------------------------

def dirichlet_mask(conn: np.ndarray, nv: int) -> np.ndarray:
    """Vertices on boundary faces (a face owned by exactly one element)."""
    faces = np.concatenate([np.sort(conn[:, f], axis=1) for f in _FACES], axis=0)
    uniq, inv, counts = np.unique(faces, axis=0, return_inverse=True, return_counts=True)
    boundary = uniq[counts == 1]
    mask = np.zeros(nv, dtype=bool)
    mask[boundary.ravel()] = True
    return mask


def assemble(conn: np.ndarray, Ae: np.ndarray, nv: int) -> sp.csr_array:
    """A = Q^T A_L Q: sum of element matrices into the global vertex numbering."""
    rows = np.repeat(conn, 8, axis=1).ravel()
    cols = np.tile(conn, (1, 8)).ravel()
    return sp.csr_array(sp.coo_array((Ae.ravel(), (rows, cols)), shape=(nv, nv)))


def vertex_element_counts(conn: np.ndarray, nv: int) -> np.ndarray:
    """Counting vector w = Q Q^T e_L at the vertices: elements per vertex."""
    return np.bincount(conn.ravel(), minlength=nv).astype(np.float64)


class Problem:
    """Setup of the two-level Schwarz preconditioner for one mesh."""

    def __init__(self, xyz, conn, part, boxes, overlap: int = 1, margin: float = 0.0,
                 dirichlet=None, coarse_operator: str = "broken"):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.part = np.asarray(part, dtype=np.int64)
        self.nv = self.xyz.shape[0]
        self.ne = self.conn.shape[0]
        self.Ae, self.min_det = element_matrices(self.xyz, self.conn)
        if not self.min_det > 0.0:
            raise ValueError("element with non-positive Jacobian")
        self.dir = dirichlet_mask(self.conn, self.nv) if dirichlet is None else np.asarray(dirichlet, bool)
        self.free = np.flatnonzero(~self.dir)
        self.A_full = assemble(self.conn, self.Ae, self.nv)
        self.A = self.A_full[self.free][:, self.free]          # free block, SPD
        self.cnt = vertex_element_counts(self.conn, self.nv)
        self._setup_subdomains(overlap)
        if coarse_operator not in ("broken", "galerkin", "vertex"):
            raise ValueError(coarse_operator)
        self.coarse_operator = coarse_operator
        self._setup_boxes(tuple(int(b) for b in boxes), margin)

    # -- vectors of length nv (Dirichlet entries zero) ------------------------
    def to_free(self, v):
        return np.asarray(v, dtype=np.float64)[self.free]

    def to_full(self, vf):
        out = np.zeros(self.nv)
        out[self.free] = vf
        return out

    # -- operator (Sec. 3: w = A u) -------------------------------------------
    def apply_A(self, x):
        """y = A x on the free dofs; x, y of length nv, Dirichlet entries 0."""
        return self.to_full(self.A @ self.to_free(x))

    # -- subdomains (Sec. 3, the overlapping-subdomain paragraph) -------------
    def _setup_subdomains(self, overlap: int):
        ne, nv = self.ne, self.nv
        nparts = int(self.part.max()) + 1 if ne else 0
        E2V = sp.csr_array((np.ones(8 * ne), (np.repeat(np.arange(ne), 8), self.conn.ravel())),
                           shape=(ne, nv))
        E2V.data[:] = 1.0
        E2V.sum_duplicates()
        E2V.data[:] = 1.0
        S = sp.csr_array((np.ones(ne), (self.part, np.arange(ne))), shape=(nparts, ne))
        # vertices of the original (not grown) subdomains, for RAS
        own = (S @ E2V).tocsr()
        own.data[:] = 1.0
        self.own_mult = np.asarray(own.sum(axis=0)).ravel()         # original subdomains holding v
        self._own = own
        for _ in range(overlap):   # add every element sharing a vertex with Omega_p
            touched_v = (S @ E2V)
            touched_v.data[:] = 1.0
            S = touched_v @ E2V.T
            S.data[:] = 1.0
        # number of elements of each vertex that lie in the grown subdomain
        inside = (S @ E2V).tocsr()
        inside.sort_indices()
        self.sub_idx = []
        free = ~self.dir
        for p in range(nparts):
            lo, hi = inside.indptr[p], inside.indptr[p + 1]
            v = inside.indices[lo:hi]
            c = inside.data[lo:hi]
            keep = v[(c == self.cnt[v]) & free[v]]
            self.sub_idx.append(np.sort(keep))
        # map vertex id -> position in the free numbering
        self.free_pos = -np.ones(nv, dtype=np.int64)
        self.free_pos[self.free] = np.arange(self.free.size)
        # local matrices A_p = R_p A R_p^T (principal submatrices), Cholesky
        self.mult = np.zeros(nv)
        for idx in self.sub_idx:
            self.mult[idx] += 1.0
        self.groups = {}
        sizes = np.array([len(i) for i in self.sub_idx])
        for m in np.unique(sizes):
            if m == 0:
                continue
            ps = np.flatnonzero(sizes == m)
            I = np.stack([self.sub_idx[p] for p in ps])            # (G, m) vertex ids
            F = self.free_pos[I]
            rows = np.repeat(F, m, axis=1).ravel()
            cols = np.tile(F, (1, m)).ravel()
            Ap = np.asarray(self.A[rows, cols]).reshape(len(ps), m, m)
            try:
                L = np.linalg.cholesky(Ap)
            except np.linalg.LinAlgError as exc:
                raise ValueError("local matrix not SPD") from exc
            self.groups[int(m)] = (ps, I, Ap, L)
        # RAS prolongation weights (Sec. 3: R~_p^T is R_p^T with the columns of
        # the grown part Omega~_p minus Omega_p null; the surface nodes that
        # several original subdomains store are averaged for continuity)
        self.ras_w = {}
        for m, (ps, I, Ap, L) in self.groups.items():
            inown = np.stack([np.asarray(self._own[[p]].toarray()).ravel()[I[g]] for g, p in enumerate(ps)])
            self.ras_w[m] = np.where(inown > 0, 1.0 / np.maximum(self.own_mult[I], 1.0), 0.0)

    def local_solves(self, r, weighted, inner: int = 0):
        """sum_p R~_p^T A_p^{-1} R_p r (Eqs. (3), (4)).  weighted: True scales
        by W_ov = 1/multiplicity (R~_p = R_p); False adds plainly; "ras" uses
        the restricted prolongation.  inner > 0 replaces A_p^{-1} by that many
        CG steps on A_p from zero (an inexact local solve, Sec. 6)."""
        r = np.asarray(r, dtype=np.float64)
        out = np.zeros(self.nv)
        for m, (ps, I, Ap, L) in self.groups.items():
            rp = r[I]                                               # R_p r
            if inner > 0:
                y = _batched_cg(Ap, rp, inner)
            else:
                y = sla.solve_triangular(L, rp[..., None], lower=True)
                y = sla.solve_triangular(np.swapaxes(L, 1, 2), y, lower=False)[..., 0]
            if weighted == "ras":
                y = y * self.ras_w[m]
            np.add.at(out, I.ravel(), y.ravel())                    # R~_p^T, summed
        if weighted is True:
            nz = self.mult > 0
            out[nz] /= self.mult[nz]
        return out

    def local_solve_one(self, p: int, r):
        """A_p^{-1} R_p r for a single subdomain p (values at sub_idx[p])."""
        idx = self.sub_idx[p]
        if idx.size == 0:
            return np.zeros(0)
        F = self.free_pos[idx]
        Ap = self.A[F][:, F].toarray()
        return np.linalg.solve(Ap, np.asarray(r)[idx])

    # -- box coarse space (Sec. 4) --------------------------------------------
    def _setup_boxes(self, boxes, margin):
        b = np.array(boxes, dtype=np.int64)
        lo = self.xyz.min(axis=0)
        hi = self.xyz.max(axis=0)
        ext = hi - lo
        lo = lo - margin * ext
        hi = hi + margin * ext
        H = (hi - lo) / b
        self.box_lo, self.box_H, self.box_b = lo, H, b
        X = self.xyz[self.conn]                                   # (E, 8, 3)
        centroid = X.mean(axis=1)
        cell = np.floor((centroid - lo) / H).astype(np.int64)
        cell = np.clip(cell, 0, b - 1)
        self.cell = cell
        # element-local trilinear interpolant J_e (8 nodes x 8 cell corners)
        t = (X - (lo + cell * H)[:, None, :]) / H                  # (E, 8, 3)
        Je = np.ones((self.ne, 8, 8))
        for m in range(8):
            for d in range(3):
                bit = (m >> d) & 1
                Je[:, :, m] *= t[:, :, d] if bit else (1.0 - t[:, :, d])
        Je[self.dir[self.conn]] = 0.0                              # Psi_j vanish on Dirichlet nodes
        nb = b + 1
        corner = np.empty((self.ne, 8), dtype=np.int64)
        for m in range(8):
            c = cell + np.array([m & 1, (m >> 1) & 1, (m >> 2) & 1])
            corner[:, m] = c[:, 0] + nb[0] * (c[:, 1] + nb[1] * c[:, 2])
        if self.coarse_operator == "vertex":
            self._setup_vertex_J(nb)
            return self._factor_Ar()
        # active vertices: corners of occupied cells with a nontrivial column
        colmax = np.zeros(int(np.prod(nb)))
        np.maximum.at(colmax, corner.ravel(), np.abs(Je).max(axis=1).ravel())
        occupied = np.zeros(int(np.prod(nb)), dtype=bool)
        occupied[corner.ravel()] = True
        active = occupied & (colmax > 1e-12)
        self.box_active = np.flatnonzero(active)                   # lexicographic order
        col = -np.ones(int(np.prod(nb)), dtype=np.int64)
        col[self.box_active] = np.arange(self.box_active.size)
        self.corner_col = col[corner]                              # (E, 8); -1 = dropped
        self.Je = Je
        self.nr = int(self.box_active.size)
        if self.coarse_operator == "galerkin":
            # A_r = J~^T A J~ with J~ = W Q^T J_L (Sec. 4: the Galerkin reading
            # of A_r; full support of the averaged interpolant, 5^3 stencil)
            keep = self.corner_col >= 0
            e_idx, k_idx, m_idx = np.nonzero(np.broadcast_to(keep[:, None, :], (self.ne, 8, 8)))
            rows = self.conn[e_idx, k_idx]
            vals = Je[e_idx, k_idx, m_idx] / self.cnt[rows]
            Jt = sp.coo_array((vals, (rows, self.corner_col[e_idx, m_idx])), shape=(self.nv, self.nr)).tocsr()
            Jf = Jt[self.free]
            self.Ar = (Jf.T @ self.A @ Jf).toarray()
            return self._factor_Ar()
        # A_r = sum_e J_e^T A^e J_e (Eq. (12), cell-wise assembly)
        Jk = np.where((self.corner_col >= 0)[:, None, :], Je, 0.0)
        Ke = np.einsum("ekm,ekl,eln->emn", Jk, self.Ae, Jk)
        cc = np.where(self.corner_col >= 0, self.corner_col, 0)
        rows = np.repeat(cc, 8, axis=1).ravel()
        cols = np.tile(cc, (1, 8)).ravel()
        self.Ar = sp.coo_array((Ke.ravel(), (rows, cols)), shape=(self.nr, self.nr)).toarray()
        return self._factor_Ar()

    def _setup_vertex_J(self, nb):
        """Vertex-based J (Sec. 4, the nodal construction): each node x_i takes
        the trilinear interpolants of the 8 corners of the box cell holding it
        (clamped to the grid); J_ij = Phi_j(x_i), Dirichlet rows zero; box
        vertices with no entry above 1e-12 are compressed out; A_r = J^T A J
        (full support, 5^3 stencil)."""
        t = (self.xyz - self.box_lo) / self.box_H
        vcell = np.clip(np.floor(t).astype(np.int64), 0, self.box_b - 1)
        f = t - vcell
        W = np.ones((self.nv, 8))
        corner = np.empty((self.nv, 8), dtype=np.int64)
        for m in range(8):
            bit = np.array([m & 1, (m >> 1) & 1, (m >> 2) & 1])
            for d in range(3):
                W[:, m] *= f[:, d] if bit[d] else (1.0 - f[:, d])
            c = vcell + bit
            corner[:, m] = c[:, 0] + nb[0] * (c[:, 1] + nb[1] * c[:, 2])
        W[self.dir] = 0.0
        colmax = np.zeros(int(np.prod(nb)))
        np.maximum.at(colmax, corner.ravel(), np.abs(W).ravel())
        self.box_active = np.flatnonzero(colmax > 1e-12)
        col = -np.ones(int(np.prod(nb)), dtype=np.int64)
        col[self.box_active] = np.arange(self.box_active.size)
        self.nr = int(self.box_active.size)
        c = col[corner]
        keep = c >= 0
        r = np.repeat(np.arange(self.nv), 8).reshape(self.nv, 8)
        self.Jv = sp.coo_array((W[keep], (r[keep], c[keep])), shape=(self.nv, self.nr)).tocsr()
        Jf = self.Jv[self.free]
        self.Ar = (Jf.T @ self.A @ Jf).toarray()

    def _factor_Ar(self):
        try:
            self.Ar_chol = sla.cho_factor(self.Ar, lower=True)
        except np.linalg.LinAlgError as exc:
            raise ValueError("reduced matrix not SPD") from exc

    def interp(self, ur):
        """z = W Q^T J_L u_r: element-local trilinear values, averaged at the
        vertices by the inverse element counts (Sec. 4); z = J u_r with the
        vertex-based J."""
        if self.coarse_operator == "vertex":
            z = self.Jv @ np.asarray(ur, dtype=np.float64)
            z[self.dir] = 0.0
            return z
        urx = np.append(np.asarray(ur, dtype=np.float64), 0.0)     # dropped columns read 0
        zl = np.einsum("ekm,em->ek", self.Je, urx[self.corner_col])     # J_L u_r, (E, 8)
        z = np.zeros(self.nv)
        np.add.at(z, self.conn.ravel(), zl.ravel())
        z /= self.cnt
        z[self.dir] = 0.0
        return z

    def restrict(self, s):
        """r_r = J_L^T Q W s (the transpose of interp)."""
        if self.coarse_operator == "vertex":
            return self.Jv.T @ np.where(self.dir, 0.0, np.asarray(s, dtype=np.float64))
        w = np.asarray(s, dtype=np.float64) / self.cnt
        w = np.where(self.dir, 0.0, w)
        contrib = np.einsum("ekm,ek->em", self.Je, w[self.conn])   # (E, 8)
        rr = np.zeros(self.nr + 1)
        np.add.at(rr, np.where(self.corner_col >= 0, self.corner_col, self.nr).ravel(), contrib.ravel())
        return rr[:self.nr]

    def coarse_solve(self, rr):
        """u_r = A_r^{-1} r_r (exact; the paper uses XX^T, Sec. 2)."""
        return sla.cho_solve(self.Ar_chol, rr)

    def box_lattice_coords(self):
        """Integer lattice coordinates (i, j, k) of the active box vertices,
        from their lexicographic ids i + (b_x+1)(j + (b_y+1)k)."""
        nb = self.box_b + 1
        g = self.box_active
        return np.stack([g % nb[0], (g // nb[0]) % nb[1], g // (nb[0] * nb[1])], axis=1)

    def xxt_factor(self):
        """X of the XX^T reduced solve (Sec. 2), built once: A_r-conjugate
        columns in the nested-dissection order of the box lattice."""
        if getattr(self, "_xxt", None) is None:
            order = nested_dissection(self.box_lattice_coords())
            self._xxt = xxt_basis(self.Ar, order)
        return self._xxt

    def coarse_solve_xxt(self, rr):
        """u_r = X X^T r_r (Sec. 2: the projection onto the full conjugate
        basis is the exact solution)."""
        X = self.xxt_factor()
        return X @ (X.T @ np.asarray(rr, dtype=np.float64))

    def box_correction(self, r):
        """B_C r = J~ A_r^{-1} J~^T r."""
        return self.interp(self.coarse_solve(self.restrict(r)))

    # -- preconditioners -------------------------------------------------------
    def apply_M(self, r, form: str = "hybrid", inner: int = 0):
        """M r; inner > 0 replaces every A_p^{-1} by that many CG steps on
        A_p (the inexact local solves of Sec. 6)."""
        r = np.where(self.dir, 0.0, np.asarray(r, dtype=np.float64))
        if form == "hybrid":                    # Eqs. (4), (5)
            l = self.local_solves(r, weighted=True, inner=inner)
            s = r - self.apply_A(l)
            return l + self.box_correction(s)
        if form == "additive":                  # Eq. (3)
            return self.local_solves(r, weighted=False, inner=inner) + self.box_correction(r)
        if form == "ras":                       # Eq. (3) with the restricted R~_p (RAS)
            return self.local_solves(r, weighted="ras", inner=inner) + self.box_correction(r)
        if form == "local":                     # ASM_1 alone
            return self.local_solves(r, weighted=True, inner=inner)
        if form == "box":                       # J A_r^{-1} J^T alone
            return self.box_correction(r)
        if form == "none":
            return r.copy()
        raise ValueError(form)

    # -- outer iteration -------------------------------------------------------
    def solve(self, b, rtol: float = 1e-8, maxit: int = 500, form: str = "hybrid", inner: int = 0):
        """Flexible PCG, x0 = 0, Polak-Ribiere beta; stops when the recursive
        residual satisfies ||r|| <= rtol ||b||.  Returns (x, iters, true relres);
        iters counts the products A p; see fcg for the return tuple."""
        return fcg(self.apply_A, lambda r: self.apply_M(r, form, inner),
                   np.where(self.dir, 0.0, np.asarray(b, dtype=np.float64)), rtol, maxit)


# ----------------------------------------------------------------------------
# XX^T reduced solver (Sec. 2, the paragraph on the sparse factorisation
# A_c^{-1} = X X^T)
# ----------------------------------------------------------------------------

def nested_dissection(coords, leaf: int = 8):
    """Nested-dissection order of lattice points (rows of `coords`).

    Reading (the paper names nested dissection without details): a set of
    more than `leaf` points is cut by the coordinate plane through the median
    of its distinct coordinates along its longest extent; the points below
    the plane come first, then those above, each ordered the same way, then
    the points on the plane (the separator).  Smaller sets keep their order.
    Returns a permutation of range(len(coords))."""
    coords = np.asarray(coords)

    def rec(ids):
        if len(ids) <= leaf:
            return list(ids)
        p = coords[ids]
        ext = p.max(axis=0) - p.min(axis=0)
        ax = int(np.argmax(ext))            # first axis of the longest extent
        planes = np.unique(p[:, ax])
        mid = planes[len(planes) // 2]
        below = [i for i in ids if coords[i, ax] < mid]
        above = [i for i in ids if coords[i, ax] > mid]
        sep = [i for i in ids if coords[i, ax] == mid]
        return rec(below) + rec(above) + sep

    return np.array(rec(list(range(len(coords)))), dtype=np.int64)


def xxt_basis(A, order):
    """Columns x_1..x_n with x_i^T A x_j = delta_ij (Sec. 2), formed in the
    given order: the k-th is the unit vector of order[k] minus its A-projection
    on the earlier ones, scaled to unit A-norm (Gram-Schmidt in the A inner
    product).  Under a nested-dissection order the columns stay sparse; with
    all n of them, X X^T = A^{-1}."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    X = np.zeros((n, n))
    for k, j in enumerate(order):
        x = np.zeros(n)
        x[j] = 1.0
        c = X[:, :k].T @ A[:, j]            # x_i^T A e_j, i < k
        x -= X[:, :k] @ c
        x /= np.sqrt(x @ A @ x)
        X[:, k] = x
    return X


def _batched_cg(Ap, rp, steps: int):
    """`steps` CG iterations on each A_p y = r_p of a group, from y = 0."""
    y = np.zeros_like(rp)
    res = rp.copy()
    d = res.copy()
    rr = np.einsum("gi,gi->g", res, res)
    for _ in range(steps):
        Ad = np.einsum("gij,gj->gi", Ap, d)
        dAd = np.einsum("gi,gi->g", d, Ad)
        a = np.where(dAd > 0, rr / np.where(dAd > 0, dAd, 1.0), 0.0)
        y += a[:, None] * d
        res -= a[:, None] * Ad
        rr_new = np.einsum("gi,gi->g", res, res)
        d = res + np.where(rr > 0, rr_new / np.where(rr > 0, rr, 1.0), 0.0)[:, None] * d
        rr = rr_new
    return y


def richardson(apply_A, apply_M, b, rtol, maxit, theta: float = 1.0):
    """Schwarz-Richardson (the paper's alternative wrapper): x += theta M (b -
    A x) from x = 0 until ||b - A x|| <= rtol ||b||.  Returns (x, iters,
    relres, converged)."""
    x = np.zeros_like(b)
    nb = float(np.linalg.norm(b))
    r = b.copy()
    for k in range(maxit + 1):
        rel = float(np.linalg.norm(r)) / nb if nb > 0 else 0.0
        if rel <= rtol:
            return x, k, rel, True
        if k == maxit:
            return x, k, rel, False
        x = x + theta * apply_M(r)
        r = b - apply_A(x)


def fgmres(apply_A, apply_M, b, rtol, maxit, restart: int = 30):
    """Right-preconditioned flexible GMRES(restart) from x = 0 (the paper's
    GMRES wrapping; flexible, so M may change between steps): the Arnoldi
    basis V of the preconditioned directions Z = M V, x = Z y with y the
    least-squares minimiser of ||beta e_1 - H y||.  Returns (x, products A z,
    relres of b - A x, converged)."""
    x = np.zeros_like(b)
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return x, 0, 0.0, True
    its = 0
    while True:
        r = b - apply_A(x)
        beta = float(np.linalg.norm(r))
        if beta <= rtol * nb or its >= maxit:
            return x, its, beta / nb, beta <= rtol * nb
        V, Z = [r / beta], []
        H = np.zeros((restart + 1, restart))
        for j in range(restart):
            Z.append(apply_M(V[j]))
            w = apply_A(Z[j])
            its += 1
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = float(V[i] @ w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            res = float(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y))
            if res <= rtol * nb or its >= maxit or H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
        x = x + np.array(Z).T @ y


class Projection:
    """A-orthogonal projection onto prior solutions (Sec. 5: solve for the
    change u - u_bar, u_bar = sum_j beta_j u^{m-j} the A-orthogonal best fit
    onto l prior solutions).

    Keeps an A-orthonormal basis x~_1..x~_k (k <= l) of the span of earlier
    solutions, so the best fit of the new solution is u_bar = sum_j
    (x~_j . b) x~_j (x~_j^T A u = x~_j . b).  After a solve, the new solution
    is made A-orthogonal to the basis (coefficients (A x~_j) . u, by the
    symmetry of A), its A x~ formed by one product with A, scaled to unit
    A-norm and appended; a full basis first restarts empty (reading: the
    paper does not say how the l solutions are chosen; this keeps the newest
    one).  A solution that adds no direction (A-norm of the orthogonal part
    below 1e-6 of its own, far above the solve tolerances used) is not
    appended: its orthogonal part would be solver error and rounding."""

    def __init__(self, apply_A, l: int):
        self.apply_A, self.l = apply_A, int(l)
        self.X = []          # x~_j
        self.AX = []         # A x~_j

    def start(self, b):
        """(u_bar, b - A u_bar)."""
        ubar = np.zeros_like(b)
        bp = np.array(b, dtype=np.float64)
        for x, ax in zip(self.X, self.AX):
            c = float(x @ b)
            ubar += c * x
            bp -= c * ax
        return ubar, bp

    def add(self, u):
        if len(self.X) >= self.l:
            self.X, self.AX = [], []
        w = np.array(u, dtype=np.float64)
        e = [float(ax @ w) for ax in self.AX]     # x~_j^T A u
        for c, x in zip(e, self.X):
            w -= c * x
        Aw = self.apply_A(w)
        nrm2 = float(w @ Aw)
        if nrm2 > 1e-12 * (sum(c * c for c in e) + nrm2):
            self.X.append(w / np.sqrt(nrm2))
            self.AX.append(Aw / np.sqrt(nrm2))


def solve_projected(P, bs, l: int, rtol: float = 1e-8, maxit: int = 500, form: str = "hybrid"):
    """Solve A u = b for each b of the sequence with the projection onto up
    to l prior solutions.  The correction solve stops when its residual
    (which is b - A u) is below rtol ||b||.  Returns a list of (x, iters,
    true relres, u_bar, basis size after the solve)."""
    proj = Projection(P.apply_A, l)
    out = []
    for b in bs:
        b = np.where(P.dir, 0.0, np.asarray(b, dtype=np.float64))
        ubar, bp = proj.start(b)
        nb, nbp = float(np.linalg.norm(b)), float(np.linalg.norm(bp))
        if nbp > 0.0:
            d, it, _, _ = fcg(P.apply_A, lambda r: P.apply_M(r, form), bp, rtol * nb / nbp, maxit)
        else:
            d, it = np.zeros_like(b), 0
        x = ubar + d
        rel = float(np.linalg.norm(b - P.apply_A(x)) / nb) if nb > 0 else 0.0
        proj.add(x)
        out.append((x, it, rel, ubar, len(proj.X)))
    return out


def fcg(apply_A, apply_M, b, rtol, maxit):
    """Flexible PCG.  Returns (x, iters, true relres, converged).  A breakdown
    (r.z = 0 or p.q <= 0, which a singular preconditioner such as the box term
    alone can cause) stops the iteration unconverged."""
    x = np.zeros_like(b)
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return x, 0, 0.0, True
    r = b.copy()
    z = apply_M(r)
    p = z.copy()
    rho = float(r @ z)
    its = 0
    converged = False
    for k in range(1, maxit + 1):
        if not rho > 0.0:
            break
        q = apply_A(p)
        pq = float(p @ q)
        if not pq > 0.0:
            break
        alpha = rho / pq
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        its = k
        if np.linalg.norm(r) <= rtol * nb:
            converged = True
            break
        z = apply_M(r)
        beta = float(z @ (r - r_old)) / rho
        rho = float(r @ z)
        p = z + beta * p
    relres = float(np.linalg.norm(b - apply_A(x))) / nb
    return x, its, relres, converged
