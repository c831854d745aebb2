// Host setup of the two-level Schwarz coarse solver: everything that is built
// once per mesh and then kept resident on the device.
//
//   element matrices   a^e_ij = int grad l_i . grad l_j dV, trilinear map,
//                      2x2x2 Gauss-Legendre (Sec. 3)
//   Dirichlet set      vertices of faces owned by one element (homogeneous
//                      Dirichlet, Sec. 3), unless the caller gives a mask
//   subdomains         Omega_p grown by delta layers of vertex-sharing
//                      elements; R_p = free vertices whose elements all lie in
//                      the grown set ("interior to the extended subdomain",
//                      Sec. 3); A_p = R_p A R_p^T and its explicit inverse
//   box coarse space   bounding box split in b_x*b_y*b_z cells; each element
//                      belongs to the cell holding its centroid; J_L evaluates
//                      the cell's trilinear hats at the element's vertices
//                      (rows of Dirichlet vertices zero); active box vertices
//                      are the corners of occupied cells with a nonzero column
//                      (Sec. 4); A_r = sum_e J_e^T A^e J_e cell by cell
//                      (Eq. (12)) and its inverse.
//
// The device keeps explicit inverses instead of sparse Cholesky factors (the
// paper's CHOLMOD and XX^T): a GEMV with a 27..64-dof inverse is one coalesced
// stream per subdomain, where a triangular solve would be two dependent sweeps.
// Each symmetric inverse is stored by cyclic diagonals, entry (i, (i+d) mod m)
// at d*m + i for d = 0..floor(m/2): m(m+1)/2 entries for odd m (m/2 more for
// even m), and lane i of a warp reads diagonal d at i and at (i-d) mod m.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include <omp.h>

#include "internal.h"

namespace cgs {
namespace {

constexpr int kMaxSubDofs = 16384;

// Stiffness of one trilinear hexahedron, 2x2x2 Gauss points (weights 1).
// Returns the smallest Jacobian determinant met at a quadrature point.
double hex_stiffness(const double X[8][3], double A[8][8]) {
    const double g = 1.0 / std::sqrt(3.0);
    double min_det = 1e300;
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) A[i][j] = 0.0;
    for (int q = 0; q < 8; ++q) {
        double xi[3];
        for (int d = 0; d < 3; ++d) xi[d] = ((q >> d) & 1) ? g : -g;
        // reference gradients dN[k][a]
        double dN[8][3];
        for (int k = 0; k < 8; ++k) {
            double s[3], f[3];
            for (int d = 0; d < 3; ++d) {
                s[d] = ((k >> d) & 1) ? 1.0 : -1.0;
                f[d] = 1.0 + s[d] * xi[d];
            }
            dN[k][0] = 0.125 * s[0] * f[1] * f[2];
            dN[k][1] = 0.125 * s[1] * f[0] * f[2];
            dN[k][2] = 0.125 * s[2] * f[0] * f[1];
        }
        // Jacobian J[d][a] = dx_d / dxi_a
        double J[3][3] = {{0}};
        for (int k = 0; k < 8; ++k)
            for (int d = 0; d < 3; ++d)
                for (int a = 0; a < 3; ++a) J[d][a] += X[k][d] * dN[k][a];
        // cofactors: inverse(J)[a][d] = C[d][a] / det
        double C[3][3];
        C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
        min_det = std::min(min_det, det);
        if (!(det > 0.0)) continue;
        // physical gradients B[k][d] = sum_a dN[k][a] * inv(J)[a][d]
        double B[8][3];
        for (int k = 0; k < 8; ++k)
            for (int d = 0; d < 3; ++d)
                B[k][d] = (dN[k][0] * C[d][0] + dN[k][1] * C[d][1] + dN[k][2] * C[d][2]) / det;
        for (int i = 0; i < 8; ++i)
            for (int j = i; j < 8; ++j)
                A[i][j] += det * (B[i][0] * B[j][0] + B[i][1] * B[j][1] + B[i][2] * B[j][2]);
    }
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < i; ++j) A[i][j] = A[j][i];
    return min_det;
}

inline double dot(const double* a, const double* b, int n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

// Cholesky factor of an SPD n x n row-major matrix in place: a = L L^T, L in
// the lower triangle.  Returns false if a pivot is not positive.  `threads`
// > 1 parallelises the row updates.
bool cholesky_lower(double* a, int n, int threads) {
    for (int j = 0; j < n; ++j) {
        double* Lj = a + (size_t)j * n;
        const double d = Lj[j] - dot(Lj, Lj, j);
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        Lj[j] = ljj;
#pragma omp parallel for schedule(static) num_threads(threads) if (threads > 1 && n - j > 64)
        for (int i = j + 1; i < n; ++i) {
            double* Li = a + (size_t)i * n;
            Li[j] = (Li[j] - dot(Li, Lj, j)) / ljj;
        }
    }
    return true;
}

// Y = L^{-1} of the factor in the lower triangle of `a`, column c stored
// contiguously in Y[c*n + i] for i >= c (zero above).  Entries that are
// structurally zero come out as exact zeros (sums of products with zeros).
std::vector<double> lower_inverse(const double* a, int n, int threads) {
    std::vector<double> Y((size_t)n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads) if (threads > 1)
    for (int c = 0; c < n; ++c) {
        double* y = Y.data() + (size_t)c * n;
        y[c] = 1.0 / a[(size_t)c * n + c];
        for (int i = c + 1; i < n; ++i) {
            const double* Li = a + (size_t)i * n;
            double s = 0.0;
            for (int k = c; k < i; ++k) s += Li[k] * y[k];
            y[i] = -s / Li[i];
        }
    }
    return Y;
}

// Explicit inverse of an SPD n x n row-major matrix `a` (destroyed) through
// its Cholesky factor: a = L L^T, Y = L^{-1}, inv = Y^T Y.  Returns false if
// a pivot is not positive.
bool spd_inverse(double* a, int n, double* inv, int threads) {
    if (!cholesky_lower(a, n, threads)) return false;
    const std::vector<double> Y = lower_inverse(a, n, threads);
    // inv[i][j] = sum_{k >= max(i,j)} Y[k][i] Y[k][j]
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads) if (threads > 1)
    for (int i = 0; i < n; ++i) {
        const double* yi = Y.data() + (size_t)i * n;
        for (int j = 0; j <= i; ++j) {
            const double* yj = Y.data() + (size_t)j * n;
            const double v = dot(yi + i, yj + i, n - i);
            inv[(size_t)i * n + j] = v;
            inv[(size_t)j * n + i] = v;
        }
    }
    return true;
}

// Nested-dissection order of lattice points (the active box vertices): a set
// of more than kNdLeaf points is split at the median coordinate plane of its
// longest extent; the points below the plane are ordered first, then those
// above (recursively), then the plane itself, which separates the two
// halves of a box-lattice stencil.  Appends to `out`.
constexpr size_t kNdLeaf = 8;
void nd_order(const std::vector<std::array<int, 3>>& c, std::vector<int32_t> ids, std::vector<int32_t>& out) {
    if (ids.size() <= kNdLeaf) {
        out.insert(out.end(), ids.begin(), ids.end());
        return;
    }
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int32_t i : ids)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], c[i][d]);
            hi[d] = std::max(hi[d], c[i][d]);
        }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    if (hi[ax] == lo[ax]) {   // a single point repeated cannot occur; keep the order
        out.insert(out.end(), ids.begin(), ids.end());
        return;
    }
    // the median of the distinct plane coordinates
    std::vector<int> planes;
    for (int32_t i : ids) planes.push_back(c[i][ax]);
    std::sort(planes.begin(), planes.end());
    planes.erase(std::unique(planes.begin(), planes.end()), planes.end());
    const int mid = planes[planes.size() / 2];
    std::vector<int32_t> below, above, sep;
    for (int32_t i : ids) (c[i][ax] < mid ? below : c[i][ax] > mid ? above : sep).push_back(i);
    nd_order(c, std::move(below), out);
    nd_order(c, std::move(above), out);
    out.insert(out.end(), sep.begin(), sep.end());
}

// XX^T factors of the SPD reduced matrix `Ar` (row-major nr x nr, destroyed):
// in the nested-dissection order P, P A_r P^T = L L^T and X~ = L^{-T} has
// A-conjugate columns (x~_i^T (P A_r P^T) x~_j = delta_ij); X = P^T X~ gives
// A_r^{-1} = X X^T.  Column k of X (nested-dissection position k) is
// supported on k and the positions before it in its dissection subtree.
bool xxt_factor(const double* Ar, int64_t nr, const std::vector<int32_t>& perm, int threads, HostSetup& S) {
    const int n = (int)nr;
    std::vector<double> a((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = Ar[(size_t)perm[i] * n + perm[j]];
    if (!cholesky_lower(a.data(), n, threads)) return false;
    const std::vector<double> Y = lower_inverse(a.data(), n, threads);
    // X~[c][k] = Y[k][c] = Y[c*n + k] (k >= c); row of X = perm[c]
    S.xc_ptr.assign(n + 1, 0);
    S.xr_ptr.assign(n + 1, 0);
    for (int c = 0; c < n; ++c)
        for (int k = c; k < n; ++k)
            if (Y[(size_t)c * n + k] != 0.0) {
                S.xc_ptr[k + 1]++;
                S.xr_ptr[perm[c] + 1]++;
            }
    for (int k = 0; k < n; ++k) {
        S.xc_ptr[k + 1] += S.xc_ptr[k];
        S.xr_ptr[k + 1] += S.xr_ptr[k];
    }
    const size_t nnz = (size_t)S.xc_ptr[n];
    S.xc_idx.assign(nnz, 0);
    S.xc_val.assign(nnz, 0.0);
    S.xr_idx.assign(nnz, 0);
    S.xr_val.assign(nnz, 0.0);
    // columns in ascending row order: walk the reduced rows in order
    std::vector<int32_t> inv(n);
    for (int c = 0; c < n; ++c) inv[perm[c]] = c;
    std::vector<int32_t> fc(S.xc_ptr.begin(), S.xc_ptr.end() - 1), fr(S.xr_ptr.begin(), S.xr_ptr.end() - 1);
    for (int row = 0; row < n; ++row) {
        const int c = inv[row];
        for (int k = c; k < n; ++k) {
            const double v = Y[(size_t)c * n + k];
            if (v == 0.0) continue;
            S.xc_idx[fc[k]] = (uint16_t)row;
            S.xc_val[fc[k]++] = v;
            S.xr_idx[fr[row]] = (uint16_t)k;   // ascending k within the row
            S.xr_val[fr[row]++] = v;
        }
    }
    S.xs_seg.clear();
    for (int k = 0; k < n; ++k)
        for (int32_t b = S.xc_ptr[k]; b < S.xc_ptr[k + 1]; b += kXxtSeg) {
            S.xs_seg.push_back(k);
            S.xs_seg.push_back(b);
            S.xs_seg.push_back(std::min(S.xc_ptr[k + 1], b + kXxtSeg));
            S.xs_seg.push_back(0);
        }
    return true;
}

// Upper-triangle slot of the pair (i, j), i <= j, in the 36-entry layout.
inline int upper_slot(int i, int j) { return i * 8 - i * (i - 1) / 2 + (j - i); }
// Strict-upper slot of (i, j), i < j, in the 28-entry layout.
inline int off_slot(int i, int j) { return i * 7 - i * (i - 1) / 2 + (j - i - 1); }

}  // namespace

cgs_status host_setup(const double* xyz, int64_t nv, const int32_t* conn, int64_t ne,
                      const uint8_t* dirichlet, const int32_t* elem_part,
                      const cgs_params& prm, HostSetup& S, std::string& err) {
    const auto t0 = std::chrono::steady_clock::now();
    const int nthreads = std::max(1, omp_get_max_threads());
    if (!xyz || !conn || nv <= 0 || ne <= 0) {
        err = "empty mesh or null input";
        return nv <= 0 || ne <= 0 ? CGS_ERR_INVALID_MESH : CGS_ERR_INVALID_ARG;
    }
    if (nv >= INT32_MAX || ne >= INT32_MAX / 8) {
        err = "mesh too large for 32-bit indices";
        return CGS_ERR_INVALID_ARG;
    }
    for (int d = 0; d < 3; ++d)
        if (prm.box[d] < 1 || prm.box[d] > kMaxBoxes) {
            err = "box counts must lie in [1, 1023]";
            return CGS_ERR_INVALID_ARG;
        }
    if (prm.overlap_layers < 0 || !(prm.box_margin >= 0.0)) {
        err = "negative overlap or margin";
        return CGS_ERR_INVALID_ARG;
    }
    if (prm.coarse_solver < CGS_COARSE_AUTO || prm.coarse_solver > CGS_COARSE_XXT) {
        err = "coarse_solver must be CGS_COARSE_AUTO, _DENSE or _XXT";
        return CGS_ERR_INVALID_ARG;
    }
    if (prm.coarse_operator < CGS_COARSE_OP_CELLWISE || prm.coarse_operator > CGS_COARSE_OP_VERTEX) {
        err = "coarse_operator must be CGS_COARSE_OP_CELLWISE, _GALERKIN or _VERTEX";
        return CGS_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < ne * 8; ++i)
        if (conn[i] < 0 || conn[i] >= nv) {
            err = "connectivity index out of range at entry " + std::to_string(i);
            return CGS_ERR_INVALID_MESH;
        }
    int64_t n_sub = 1;
    if (elem_part) {
        int64_t mx = -1;
        for (int64_t e = 0; e < ne; ++e) {
            if (elem_part[e] < 0) {
                err = "negative subdomain id";
                return CGS_ERR_INVALID_ARG;
            }
            mx = std::max<int64_t>(mx, elem_part[e]);
        }
        n_sub = mx + 1;
    }
    S.nv = nv;
    S.ne = ne;
    S.n_sub = n_sub;

    // ---- element matrices ---------------------------------------------------
    std::vector<double> Ae((size_t)ne * 64);
    double min_det = 1e300;
#pragma omp parallel for schedule(static) reduction(min : min_det)
    for (int64_t e = 0; e < ne; ++e) {
        double X[8][3];
        for (int k = 0; k < 8; ++k)
            for (int d = 0; d < 3; ++d) X[k][d] = xyz[(size_t)conn[e * 8 + k] * 3 + d];
        double A[8][8];
        min_det = std::min(min_det, hex_stiffness(X, A));
        std::memcpy(&Ae[(size_t)e * 64], A, sizeof(A));
    }
    if (!(min_det > 0.0)) {
        err = "element with non-positive Jacobian at a quadrature point";
        return CGS_ERR_INVALID_MESH;
    }

    // ---- Dirichlet set ------------------------------------------------------
    S.dir.assign(nv, 0);
    if (dirichlet) {
        for (int64_t v = 0; v < nv; ++v) S.dir[v] = dirichlet[v] ? 1 : 0;
    } else {
        struct Face { int32_t v[4]; };
        std::vector<Face> faces((size_t)ne * 6);
        for (int64_t e = 0; e < ne; ++e) {
            for (int d = 0; d < 3; ++d)
                for (int side = 0; side < 2; ++side) {
                    Face f;
                    int n = 0;
                    for (int k = 0; k < 8; ++k)
                        if (((k >> d) & 1) == side) f.v[n++] = conn[e * 8 + k];
                    std::sort(f.v, f.v + 4);
                    faces[(size_t)e * 6 + d * 2 + side] = f;
                }
        }
        auto less = [](const Face& a, const Face& b) {
            return std::lexicographical_compare(a.v, a.v + 4, b.v, b.v + 4);
        };
        std::sort(faces.begin(), faces.end(), less);
        for (size_t i = 0; i < faces.size();) {
            size_t j = i + 1;
            while (j < faces.size() && std::equal(faces[i].v, faces[i].v + 4, faces[j].v)) ++j;
            if (j - i == 1)
                for (int k = 0; k < 4; ++k) S.dir[faces[i].v[k]] = 1;
            i = j;
        }
    }
    S.n_free = 0;
    for (int64_t v = 0; v < nv; ++v) S.n_free += !S.dir[v];

    // ---- vertex -> element adjacency, element counts --------------------------
    std::vector<int64_t> v2e_ptr(nv + 1, 0);
    for (int64_t i = 0; i < ne * 8; ++i) v2e_ptr[conn[i] + 1]++;
    for (int64_t v = 0; v < nv; ++v) v2e_ptr[v + 1] += v2e_ptr[v];
    std::vector<int32_t> v2e(ne * 8);
    {
        std::vector<int64_t> fill(v2e_ptr.begin(), v2e_ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int k = 0; k < 8; ++k) {
                const int32_t v = conn[e * 8 + k];
                // an element listing one vertex twice is degenerate (caught by det)
                v2e[fill[v]++] = (int32_t)e;
            }
    }
    S.invcnt.assign(nv, 0.0);
    for (int64_t v = 0; v < nv; ++v) {
        const int64_t c = v2e_ptr[v + 1] - v2e_ptr[v];
        S.invcnt[v] = c > 0 ? 1.0 / (double)c : 0.0;
    }

    // ---- subdomains: grow, select R_p, invert A_p -------------------------
    std::vector<int64_t> part_ptr(n_sub + 1, 0);
    std::vector<int32_t> part_el(ne);
    for (int64_t e = 0; e < ne; ++e) part_ptr[(elem_part ? elem_part[e] : 0) + 1]++;
    for (int64_t p = 0; p < n_sub; ++p) part_ptr[p + 1] += part_ptr[p];
    {
        std::vector<int64_t> fill(part_ptr.begin(), part_ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e) part_el[fill[elem_part ? elem_part[e] : 0]++] = (int32_t)e;
    }
    std::vector<std::vector<int32_t>> sub_sets(n_sub);
    std::vector<std::vector<double>> sub_inv(n_sub);
    std::vector<std::vector<double>> sub_ap(prm.local_cg_steps > 0 ? n_sub : 0);   // A_p, cyclic diagonals
    // subdomains of at most kLaneMaxM dofs (kLaneMaxMixed in the mixed forms)
    // are solved one per lane: always in the mixed forms, and in the FP64 form
    // when there are enough of them to fill the GPU one lane each (otherwise
    // a warp per subdomain)
    // (inexact local solves run CG on A_p itself, one warp per subdomain)
    const bool inexact = prm.local_cg_steps > 0;
    const bool lane_packs = !inexact && (prm.prec != CGS_FP64 || n_sub >= kRowPackMaxSubs);
    const int lane_max = prm.prec == CGS_FP64 ? kLaneMaxM : kLaneMaxMixed;
    bool not_spd = false, too_big = false;
#pragma omp parallel
    {
        std::vector<int32_t> estamp(ne, -1), vcount(nv, 0), vpos(nv, -1);
        std::vector<int32_t> grown, frontier, touched;
        std::vector<double> Ap;
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n_sub; ++p) {
            grown.assign(part_el.begin() + part_ptr[p], part_el.begin() + part_ptr[p + 1]);
            for (int32_t e : grown) estamp[e] = (int32_t)p;
            size_t layer_begin = 0;
            for (int layer = 0; layer < prm.overlap_layers; ++layer) {
                const size_t layer_end = grown.size();
                for (size_t i = layer_begin; i < layer_end; ++i) {
                    const int32_t e = grown[i];
                    for (int k = 0; k < 8; ++k) {
                        const int32_t v = conn[(int64_t)e * 8 + k];
                        for (int64_t t = v2e_ptr[v]; t < v2e_ptr[v + 1]; ++t) {
                            const int32_t f = v2e[t];
                            if (estamp[f] != (int32_t)p) {
                                estamp[f] = (int32_t)p;
                                grown.push_back(f);
                            }
                        }
                    }
                }
                layer_begin = layer_end;
            }
            // vertices all of whose elements are in the grown set
            touched.clear();
            for (int32_t e : grown)
                for (int k = 0; k < 8; ++k) {
                    const int32_t v = conn[(int64_t)e * 8 + k];
                    if (vcount[v]++ == 0) touched.push_back(v);
                }
            std::vector<int32_t>& R = sub_sets[p];
            R.clear();
            for (int32_t v : touched)
                if (!S.dir[v] && vcount[v] == v2e_ptr[v + 1] - v2e_ptr[v]) R.push_back(v);
            for (int32_t v : touched) vcount[v] = 0;
            std::sort(R.begin(), R.end());
            const int m = (int)R.size();
            if (m > kMaxSubDofs) {
#pragma omp atomic write
                too_big = true;
                continue;
            }
            if (m == 0) continue;
            for (int i = 0; i < m; ++i) vpos[R[i]] = i;
            Ap.assign((size_t)m * m, 0.0);
            for (int32_t e : grown) {
                const double* A = &Ae[(size_t)e * 64];
                int loc[8];
                for (int k = 0; k < 8; ++k) loc[k] = vpos[conn[(int64_t)e * 8 + k]];
                for (int k = 0; k < 8; ++k) {
                    if (loc[k] < 0) continue;
                    for (int l = 0; l < 8; ++l)
                        if (loc[l] >= 0) Ap[(size_t)loc[k] * m + loc[l]] += A[k * 8 + l];
                }
            }
            for (int i = 0; i < m; ++i) vpos[R[i]] = -1;
            if (prm.local_cg_steps > 0) {
                // A_p itself for the inexact solves: cyclic diagonals, as the inverse
                const int nd = m / 2 + 1;
                std::vector<double>& ap = sub_ap[p];
                ap.resize((size_t)nd * m);
                for (int d = 0; d < nd; ++d)
                    for (int i = 0; i < m; ++i) ap[(size_t)d * m + i] = Ap[(size_t)i * m + (i + d) % m];
            }
            if (prm.fault_negate_subdomain == (int)p + 1)   // testing aid: a non-SPD block
                for (double& a : Ap) a = -a;
            std::vector<double> full((size_t)m * m);
            if (!spd_inverse(Ap.data(), m, full.data(), 1)) {
#pragma omp atomic write
                not_spd = true;
                continue;
            }
            std::vector<double>& pk = sub_inv[p];
            if (lane_packs && m <= lane_max) {
                // upper triangle, row-major (lane packs)
                pk.resize((size_t)m * (m + 1) / 2);
                size_t e = 0;
                for (int i = 0; i < m; ++i)
                    for (int j = i; j < m; ++j) pk[e++] = full[(size_t)i * m + j];
            } else {
                // cyclic diagonals: entry (i, (i+d) mod m) at d*m + i, d = 0..m/2
                const int nd = m / 2 + 1;
                pk.resize((size_t)nd * m);
                for (int d = 0; d < nd; ++d)
                    for (int i = 0; i < m; ++i) pk[(size_t)d * m + i] = full[(size_t)i * m + (i + d) % m];
            }
        }
    }
    if (too_big) {
        err = "a subdomain has more than 16384 dofs";
        return CGS_ERR_INVALID_ARG;
    }
    if (not_spd) {
        err = "a local matrix A_p is not SPD";
        return CGS_ERR_NOT_SPD;
    }
    // RAS prolongation weights (Sec. 3, R~_p): an entry of R_p keeps its value
    // only if the vertex lies on an element of the original (not grown)
    // Omega_p, divided by the number of original subdomains holding the
    // vertex (continuity of the nodes several subdomains store)
    std::vector<std::vector<double>> sub_ras(n_sub);
    {
        auto part_of = [&](int64_t e) -> int32_t { return elem_part ? elem_part[e] : 0; };
        std::vector<int32_t> own_mult(nv, 0);
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < nv; ++v) {
            int32_t seen[64];
            int ns = 0;
            for (int64_t t = v2e_ptr[v]; t < v2e_ptr[v + 1]; ++t) {
                const int32_t q = part_of(v2e[t]);
                bool dup = false;
                for (int i = 0; i < ns; ++i) dup = dup || seen[i] == q;
                if (!dup && ns < 64) seen[ns++] = q;
            }
            own_mult[v] = ns;
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t p = 0; p < n_sub; ++p) {
            const std::vector<int32_t>& R = sub_sets[p];
            std::vector<double>& w = sub_ras[p];
            w.assign(R.size(), 0.0);
            for (size_t k = 0; k < R.size(); ++k) {
                const int32_t v = R[k];
                bool own = false;
                for (int64_t t = v2e_ptr[v]; t < v2e_ptr[v + 1] && !own; ++t) own = part_of(v2e[t]) == (int32_t)p;
                w[k] = own && own_mult[v] > 0 ? 1.0 / own_mult[v] : 0.0;
            }
        }
    }
    S.sub_ptr.assign(n_sub + 1, 0);
    S.max_m = 0;
    for (int64_t p = 0; p < n_sub; ++p) {
        const int64_t m = (int64_t)sub_sets[p].size();
        S.sub_ptr[p + 1] = S.sub_ptr[p] + m;
        S.max_m = std::max(S.max_m, m);
    }
    S.sum_m = S.sub_ptr[n_sub];
    if (S.sum_m >= INT32_MAX) {
        err = "too many subdomain dofs for 32-bit offsets";
        return CGS_ERR_INVALID_ARG;
    }
    S.sub_idx.resize(S.sum_m);
    S.wov.assign(nv, 0.0);
    std::vector<int32_t> mult(nv, 0);
    for (int64_t p = 0; p < n_sub; ++p) {
        std::copy(sub_sets[p].begin(), sub_sets[p].end(), S.sub_idx.begin() + S.sub_ptr[p]);
        for (int32_t v : sub_sets[p]) mult[v]++;
    }
    for (int64_t v = 0; v < nv; ++v) S.wov[v] = mult[v] ? 1.0 / mult[v] : 0.0;
    S.ras_w.resize(S.sum_m);
    for (int64_t p = 0; p < n_sub; ++p) std::copy(sub_ras[p].begin(), sub_ras[p].end(), S.ras_w.begin() + S.sub_ptr[p]);
    if (prm.local_cg_steps > 0 && S.max_m > 64) {
        err = "inexact local solves (local_cg_steps > 0) need subdomains of at most 64 dofs";
        return CGS_ERR_INVALID_ARG;
    }
    auto in_lane = [&](int64_t p) {
        const size_t m = sub_sets[p].size();
        return lane_packs && m > 0 && m <= (size_t)lane_max;
    };
    // warp-kernel subdomains, caller order
    S.wsub_ptr.assign(1, 0);
    S.inv_ptr.assign(1, 0);
    S.max_wm = 0;
    for (int64_t p = 0; p < n_sub; ++p) {
        if (in_lane(p)) continue;
        const int64_t m = (int64_t)sub_sets[p].size();
        S.wsub_ptr.push_back(S.wsub_ptr.back() + m);
        const int64_t sz = (m / 2 + 1) * m;
        S.inv_ptr.push_back(S.inv_ptr.back() + (sz + kPackAlign - 1) / kPackAlign * kPackAlign);
        S.max_wm = std::max(S.max_wm, m);
    }
    S.n_wsub = (int64_t)S.wsub_ptr.size() - 1;
    S.wsub_idx.resize(S.wsub_ptr.back());
    S.wsub_ras.resize(S.wsub_ptr.back());
    S.inv.assign(S.inv_ptr.back(), 0.0);
    S.ap.assign(prm.local_cg_steps > 0 ? S.inv_ptr.back() : 0, 0.0);
    for (int64_t p = 0, w = 0; p < n_sub; ++p) {
        if (in_lane(p)) continue;
        std::copy(sub_sets[p].begin(), sub_sets[p].end(), S.wsub_idx.begin() + S.wsub_ptr[w]);
        std::copy(sub_ras[p].begin(), sub_ras[p].end(), S.wsub_ras.begin() + S.wsub_ptr[w]);
        std::copy(sub_inv[p].begin(), sub_inv[p].end(), S.inv.begin() + S.inv_ptr[w]);
        if (prm.local_cg_steps > 0) std::copy(sub_ap[p].begin(), sub_ap[p].end(), S.ap.begin() + S.inv_ptr[w]);
        ++w;
    }
    // lane packs: per size class, the largest class first (blocks start
    // roughly in order, so the last wave holds the cheapest packs), 32
    // subdomains in caller order
    S.pack_m.clear();
    S.pack_idx_off.assign(1, 0);
    S.pack_inv_off.assign(1, 0);
    constexpr int kNumClasses = (int)(sizeof(kLaneClasses) / sizeof(kLaneClasses[0]));
    for (int ci = kNumClasses - 1; ci >= 0; --ci) {
        const int c = kLaneClasses[ci];
        std::vector<int64_t> members;
        for (int64_t p = 0; p < n_sub; ++p)
            if (in_lane(p) && lane_class((int)sub_sets[p].size()) == c) members.push_back(p);
        for (size_t b = 0; b < members.size(); b += 32) {
            S.pack_m.push_back(c);
            S.pack_idx_off.push_back(S.pack_idx_off.back() + (int64_t)32 * c);
            S.pack_inv_off.push_back(S.pack_inv_off.back() + (int64_t)32 * lane_entries(c));
            const int64_t io = S.pack_idx_off[S.pack_idx_off.size() - 2];
            const int64_t ao = S.pack_inv_off[S.pack_inv_off.size() - 2];
            S.pack_idx.resize(S.pack_idx_off.back(), -1);
            S.pack_ras.resize(S.pack_idx_off.back(), 0.0);
            S.pack_inv.resize(S.pack_inv_off.back(), 0.0);
            for (int l = 0; l < 32 && b + l < members.size(); ++l) {
                const int64_t p = members[b + l];
                const std::vector<int32_t>& R = sub_sets[p];
                const int m = (int)R.size();
                for (int k = 0; k < m; ++k) {
                    S.pack_idx[io + (int64_t)k * 32 + l] = R[k];
                    S.pack_ras[io + (int64_t)k * 32 + l] = sub_ras[p][k];
                }
                // the m x m triangle inside the c x c one (zero padding)
                const std::vector<double>& tri = sub_inv[p];
                size_t src = 0;
                int64_t e = 0;
                for (int i = 0; i < c; ++i)
                    for (int j = i; j < c; ++j, ++e)
                        if (i < m && j < m) S.pack_inv[ao + (int64_t)l * lane_entries(c) + e] = tri[src++];
            }
        }
    }
    // row packs for small meshes: per size class, 8 subdomains per pack,
    // lane 4 s + g holds rows g, g + 4, ... of subdomain s in full
    S.rpack_m.clear();
    S.rpack_idx_off.assign(1, 0);
    S.rpack_inv_off.assign(1, 0);
    S.rpack_idx.clear();
    S.rpack_inv.clear();
    int64_t n_lane_subs = 0;
    for (int64_t p = 0; p < n_sub; ++p) n_lane_subs += in_lane(p) ? 1 : 0;
    if (prm.prec != CGS_FP64 && n_lane_subs > 0 && n_lane_subs < kRowPackMaxSubs) {
        for (int c : kLaneClasses) {
            std::vector<int64_t> members;
            for (int64_t p = 0; p < n_sub; ++p)
                if (in_lane(p) && lane_class((int)sub_sets[p].size()) == c) members.push_back(p);
            const int per = 32 / kRowLanes, R = row_pack_rows(c), T = row_entries(c);
            for (size_t b = 0; b < members.size(); b += per) {
                S.rpack_m.push_back(c);
                S.rpack_idx_off.push_back(S.rpack_idx_off.back() + (int64_t)32 * c);
                S.rpack_inv_off.push_back(S.rpack_inv_off.back() + (int64_t)32 * T);
                const int64_t io = S.rpack_idx_off[S.rpack_idx_off.size() - 2];
                const int64_t ao = S.rpack_inv_off[S.rpack_inv_off.size() - 2];
                S.rpack_idx.resize(S.rpack_idx_off.back(), -1);
                S.rpack_ras.resize(S.rpack_idx_off.back(), 0.0);
                S.rpack_inv.resize(S.rpack_inv_off.back(), 0.0);
                for (int sidx = 0; sidx < per && b + sidx < members.size(); ++sidx) {
                    const int64_t p = members[b + sidx];
                    const std::vector<int32_t>& Rp = sub_sets[p];
                    const std::vector<double>& tri = sub_inv[p];   // upper triangle, row-major
                    const int m = (int)Rp.size();
                    auto ainv = [&](int i, int j) {
                        const int a = std::min(i, j), bb = std::max(i, j);
                        return tri[(size_t)a * m - (size_t)a * (a - 1) / 2 + (bb - a)];
                    };
                    for (int g = 0; g < kRowLanes; ++g) {
                        const int l = sidx * kRowLanes + g;
                        for (int k = 0; k < m; ++k) {
                            S.rpack_idx[io + (int64_t)k * 32 + l] = Rp[k];
                            S.rpack_ras[io + (int64_t)k * 32 + l] = sub_ras[p][k];
                        }
                        int64_t e = 0;
                        for (int r = 0; r < R; ++r)
                            for (int j = 0; j < c; ++j, ++e) {
                                const int i = r * kRowLanes + g;
                                if (i < m && j < m) S.rpack_inv[ao + (int64_t)l * T + e] = ainv(i, j);
                            }
                    }
                }
            }
        }
    }
    sub_sets.clear();
    sub_inv.clear();
    sub_ap.clear();
    sub_ras.clear();

    // ---- box grid and centroid cells ----------------------------------------
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = 1e300;
        hi[d] = -1e300;
    }
    for (int64_t v = 0; v < nv; ++v)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], xyz[v * 3 + d]);
            hi[d] = std::max(hi[d], xyz[v * 3 + d]);
        }
    for (int d = 0; d < 3; ++d) {
        const double ext = hi[d] - lo[d];
        lo[d] -= prm.box_margin * ext;
        hi[d] += prm.box_margin * ext;
        S.b[d] = prm.box[d];
        S.lo[d] = lo[d];
        S.H[d] = (hi[d] - lo[d]) / S.b[d];
        if (!(S.H[d] > 0.0)) S.H[d] = 1.0;
    }
    const int bx = S.b[0], by = S.b[1], bz = S.b[2];
    const int64_t ncell = (int64_t)bx * by * bz;
    const int64_t nbv = (int64_t)(bx + 1) * (by + 1) * (bz + 1);
    std::vector<int32_t> ecell(ne);
    for (int64_t e = 0; e < ne; ++e) {
        int c[3];
        for (int d = 0; d < 3; ++d) {
            double s = xyz[(size_t)conn[e * 8] * 3 + d];
            for (int k = 1; k < 8; ++k) s += xyz[(size_t)conn[e * 8 + k] * 3 + d];
            const double cen = s / 8.0;
            const double f = std::floor((cen - S.lo[d]) / S.H[d]);
            c[d] = (int)std::min<double>(std::max<double>(f, 0.0), S.b[d] - 1);
        }
        ecell[e] = c[0] + bx * (c[1] + by * c[2]);
    }
    // trilinear weights of the 8 cell corners at the 8 element vertices
    auto weights = [&](int64_t e, double W[8][8]) {
        const int cid = ecell[e];
        const int ci[3] = {cid % bx, (cid / bx) % by, cid / (bx * by)};
        for (int k = 0; k < 8; ++k) {
            const int32_t v = conn[e * 8 + k];
            double t[3];
            for (int d = 0; d < 3; ++d) t[d] = (xyz[(size_t)v * 3 + d] - (S.lo[d] + ci[d] * S.H[d])) / S.H[d];
            for (int m = 0; m < 8; ++m) {
                double w = 1.0;
                for (int d = 0; d < 3; ++d) w *= ((m >> d) & 1) ? t[d] : (1.0 - t[d]);
                W[k][m] = S.dir[v] ? 0.0 : w;
            }
        }
    };
    auto corner_id = [&](int cid, int m) -> int64_t {
        const int i = cid % bx + (m & 1), j = (cid / bx) % by + ((m >> 1) & 1),
                  k = cid / (bx * by) + ((m >> 2) & 1);
        return i + (int64_t)(bx + 1) * (j + (int64_t)(by + 1) * k);
    };
    // trilinear weight of corner m of cell (ci, cj, ck) at point p
    auto corner_weight = [&](const double* pnt, int ci, int cj, int ck, int m) {
        const int c[3] = {ci, cj, ck};
        double w = 1.0;
        for (int d = 0; d < 3; ++d) {
            const double t = (pnt[d] - (S.lo[d] + c[d] * S.H[d])) / S.H[d];
            w *= ((m >> d) & 1) ? t : (1.0 - t);
        }
        return w;
    };
    // the vertex-based J (Sec. 4): every node in the box cell holding it
    const bool vertex_J = prm.coarse_operator == CGS_COARSE_OP_VERTEX;
    std::vector<int32_t> vcell;
    if (vertex_J) {
        vcell.resize(nv);
        for (int64_t v = 0; v < nv; ++v) {
            int c[3];
            for (int d = 0; d < 3; ++d) {
                const double f = std::floor((xyz[(size_t)v * 3 + d] - S.lo[d]) / S.H[d]);
                c[d] = (int)std::min<double>(std::max<double>(f, 0.0), S.b[d] - 1);
            }
            vcell[v] = c[0] + bx * (c[1] + by * c[2]);
        }
    }
    std::vector<double> colmax(nbv, 0.0);
    std::vector<uint8_t> occupied(nbv, 0);
    if (vertex_J) {
        // columns with an entry above 1e-12 at some free node
        for (int64_t v = 0; v < nv; ++v) {
            if (S.dir[v] || v2e_ptr[v + 1] == v2e_ptr[v]) continue;
            const int cid = vcell[v];
            for (int m = 0; m < 8; ++m) {
                const int64_t g = corner_id(cid, m);
                occupied[g] = 1;
                const double w = corner_weight(&xyz[(size_t)v * 3], cid % bx, (cid / bx) % by, cid / (bx * by), m);
                colmax[g] = std::max(colmax[g], std::fabs(w));
            }
        }
    } else {
        for (int64_t e = 0; e < ne; ++e) {
            double W[8][8];
            weights(e, W);
            for (int m = 0; m < 8; ++m) {
                const int64_t g = corner_id(ecell[e], m);
                occupied[g] = 1;
                for (int k = 0; k < 8; ++k) colmax[g] = std::max(colmax[g], std::fabs(W[k][m]));
            }
        }
    }
    std::vector<int32_t> col(nbv, -1);
    S.box_active.clear();
    for (int64_t g = 0; g < nbv; ++g)
        if (occupied[g] && colmax[g] > 1e-12) {
            col[g] = (int32_t)S.box_active.size();
            S.box_active.push_back(g);
        }
    S.nr = (int64_t)S.box_active.size();
    S.cell_cols.assign(ncell * 8, -1);
    for (int64_t c = 0; c < ncell; ++c)
        for (int m = 0; m < 8; ++m) S.cell_cols[c * 8 + m] = col[corner_id((int)c, m)];

    // ---- per-vertex box lists ----------------------------------------------
    // W Q^T J_L regrouped by vertex: vertex v with cnt_v elements, n_c of
    // them in cell c, takes weight n_c / cnt_v on that cell's trilinear
    // interpolant.  Free vertices with elements, in vertex order (the
    // interpolation reads and writes vertex vectors through this list).
    {
        S.vb_vert.clear();
        for (int64_t v = 0; v < nv; ++v)
            if (!S.dir[v] && v2e_ptr[v + 1] > v2e_ptr[v]) S.vb_vert.push_back((int32_t)v);
        S.vb_ptr.assign(1, 0);
        S.vb_cell.clear();
        S.vb_w.clear();
        std::vector<int32_t> cells;
        for (int32_t v : S.vb_vert) {
            if (vertex_J) {   // one cell per node, weight 1
                S.vb_cell.push_back(pack_cell(vcell[v], bx, by));
                S.vb_w.push_back(1.0);
                S.vb_ptr.push_back((int32_t)S.vb_cell.size());
                continue;
            }
            cells.clear();
            for (int64_t t = v2e_ptr[v]; t < v2e_ptr[v + 1]; ++t) cells.push_back(ecell[v2e[t]]);
            std::sort(cells.begin(), cells.end());
            const double cnt = (double)cells.size();
            for (size_t a = 0; a < cells.size();) {
                size_t b = a;
                while (b < cells.size() && cells[b] == cells[a]) ++b;
                S.vb_cell.push_back(pack_cell(cells[a], bx, by));
                S.vb_w.push_back((double)(b - a) / cnt);
                a = b;
            }
            S.vb_ptr.push_back((int32_t)S.vb_cell.size());
        }
        // the same entries as one list sorted by cell (then vertex order)
        const size_t nnz = S.vb_cell.size();
        std::vector<int64_t> ord(nnz);
        std::vector<int32_t> owner(nnz);
        for (size_t i = 0; i < S.vb_vert.size(); ++i)
            for (int32_t e = S.vb_ptr[i]; e < S.vb_ptr[i + 1]; ++e) owner[e] = S.vb_vert[i];
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return S.vb_cell[a] < S.vb_cell[b]; });
        S.re_vert.resize(nnz);
        S.re_cell.resize(nnz);
        S.re_w.resize(nnz);
        for (size_t i = 0; i < nnz; ++i) {
            S.re_vert[i] = owner[ord[i]];
            S.re_cell[i] = S.vb_cell[ord[i]];
            S.re_w[i] = S.vb_w[ord[i]];
        }
        // restriction work: each cell's entries, in ranges of at most kBoxRange
        S.re_rng.clear();
        for (size_t a = 0; a < nnz;) {
            size_t b = a;
            while (b < nnz && S.re_cell[b] == S.re_cell[a]) ++b;
            for (size_t c = a; c < b; c += kBoxRange) {
                S.re_rng.push_back((int32_t)c);
                S.re_rng.push_back((int32_t)std::min(b, c + kBoxRange));
            }
            a = b;
        }
    }

    // ---- J~ by explicit rows, and the hybrid step's restriction -------------
    // Row v of J~ = W Q^T J_L: sum over the vertex's (cell, n_c / cnt_v)
    // entries of the cell's trilinear weights at x_v, duplicate columns
    // (corners shared by neighbouring cells) merged.
    {
        const size_t nvb = S.vb_vert.size();
        std::vector<std::vector<std::pair<int32_t, double>>> rows(nvb);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)nvb; ++i) {
            const int32_t v = S.vb_vert[i];
            auto& row = rows[i];
            for (int32_t e = S.vb_ptr[i]; e < S.vb_ptr[i + 1]; ++e) {
                const int pc = S.vb_cell[e];
                const int ci = pc & 1023, cj = (pc >> 10) & 1023, ck = pc >> 20;
                const int cid = ci + bx * (cj + by * ck);
                for (int m = 0; m < 8; ++m) {
                    const int32_t c = S.cell_cols[(int64_t)cid * 8 + m];
                    if (c < 0) continue;
                    const double w = S.vb_w[e] * corner_weight(&xyz[(size_t)v * 3], ci, cj, ck, m);
                    bool found = false;
                    for (auto& cv : row)
                        if (cv.first == c) {
                            cv.second += w;
                            found = true;
                            break;
                        }
                    if (!found) row.emplace_back(c, w);
                }
            }
            std::sort(row.begin(), row.end());
        }
        // the device copy (FP64 interpolation): rows padded to a multiple of
        // four entries (weight 0, column 0) for 16-byte loads, and ordered by
        // padded length, then vertex, so that the rows a warp takes have the
        // same length
        {
            std::vector<int32_t> order(nvb);
            std::iota(order.begin(), order.end(), 0);
            auto plen = [&](int32_t i) { return (int32_t)((rows[i].size() + 3) / 4 * 4); };
            std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return plen(a) < plen(b); });
            S.jt_vert.resize(nvb);
            S.jt_ptr.assign(nvb + 1, 0);
            for (size_t q = 0; q < nvb; ++q) {
                S.jt_vert[q] = S.vb_vert[order[q]];
                S.jt_ptr[q + 1] = S.jt_ptr[q] + plen(order[q]);
            }
            S.jt_nnz = 0;
            for (const auto& row : rows) S.jt_nnz += (int64_t)row.size();
            S.jt_col.assign(S.jt_ptr[nvb], 0);
            S.jt_val.assign(S.jt_ptr[nvb], 0.0);
            for (size_t q = 0; q < nvb; ++q) {
                const auto& row = rows[order[q]];
                for (size_t k = 0; k < row.size(); ++k) {
                    S.jt_col[S.jt_ptr[q] + k] = row[k].first;
                    S.jt_val[S.jt_ptr[q] + k] = row[k].second;
                }
            }
        }
        // hybrid: r_r = J~^T (r - A l) = J~^T r - (A J~)^T l, so the step
        // needs J~^T and G = A J~ (A symmetric) but never s = r - A l itself.
        // Row v of G = sum over the elements e at v of sum_k A^e(v, k) J~_k
        // (free k); entries kept where J~ or G is nonzero, then sorted by
        // column (vertex order within a column).
        S.hr_vert.clear();
        S.hr_j.clear();
        S.hr_g.clear();
        S.hr_rng.clear();
        if (prm.form == CGS_HYBRID && S.nr > 0) {
            std::vector<int32_t> row_of(nv, -1);
            for (size_t i = 0; i < nvb; ++i) row_of[S.vb_vert[i]] = (int32_t)i;
            struct Ent {
                int32_t v, c;
                double j, g;
            };
            const int nth = omp_get_max_threads();
            std::vector<std::vector<Ent>> buf(nth);
#pragma omp parallel
            {
                const int th = omp_get_thread_num();
                std::vector<double> gacc(S.nr, 0.0), jacc(S.nr, 0.0);
                std::vector<uint8_t> mark(S.nr, 0);
                std::vector<int32_t> touched;
#pragma omp for schedule(static)
                for (int64_t i = 0; i < (int64_t)nvb; ++i) {
                    const int32_t v = S.vb_vert[i];
                    touched.clear();
                    auto touch = [&](int32_t c) {
                        if (!mark[c]) {
                            mark[c] = 1;
                            touched.push_back(c);
                        }
                    };
                    for (const auto& cv : rows[i]) {
                        touch(cv.first);
                        jacc[cv.first] += cv.second;
                    }
                    for (int64_t t = v2e_ptr[v]; t < v2e_ptr[v + 1]; ++t) {
                        const int64_t e = v2e[t];
                        int iv = 0;
                        while (conn[e * 8 + iv] != v) ++iv;
                        for (int k = 0; k < 8; ++k) {
                            const int32_t u = conn[e * 8 + k];
                            const int32_t ru = row_of[u];
                            if (S.dir[u] || ru < 0) continue;
                            const double a = Ae[(size_t)e * 64 + iv * 8 + k];
                            for (const auto& cv : rows[ru]) {
                                touch(cv.first);
                                gacc[cv.first] += a * cv.second;
                            }
                        }
                    }
                    std::sort(touched.begin(), touched.end());
                    for (int32_t c : touched) {
                        if (jacc[c] != 0.0 || gacc[c] != 0.0) buf[th].push_back({v, c, jacc[c], gacc[c]});
                        jacc[c] = gacc[c] = 0.0;
                        mark[c] = 0;
                    }
                }
            }
            // counting sort by column; the buffers hold increasing vertex
            // ranges in thread order, so vertex order within a column stays
            std::vector<int64_t> cptr(S.nr + 1, 0);
            for (auto& b : buf)
                for (const Ent& x : b) cptr[x.c + 1]++;
            for (int64_t c = 0; c < S.nr; ++c) cptr[c + 1] += cptr[c];
            const int64_t nh = cptr[S.nr];
            S.hr_vert.resize(nh);
            S.hr_j.resize(nh);
            S.hr_g.resize(nh);
            std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
            for (auto& b : buf)
                for (const Ent& x : b) {
                    const int64_t at = fill[x.c]++;
                    S.hr_vert[at] = x.v;
                    S.hr_j[at] = x.j;
                    S.hr_g[at] = x.g;
                }
            for (int64_t c = 0; c < S.nr; ++c)
                for (int64_t a = cptr[c]; a < cptr[c + 1]; a += kHybRange) {
                    S.hr_rng.push_back((int32_t)a);
                    S.hr_rng.push_back((int32_t)std::min<int64_t>(cptr[c + 1], a + kHybRange));
                    S.hr_rng.push_back((int32_t)c);
                    S.hr_rng.push_back(0);
                }
        }
    }

    // ---- element order on the device: by cell, then subdomain, then id -----
    S.elem_order.resize(ne);
    std::iota(S.elem_order.begin(), S.elem_order.end(), 0);
    std::stable_sort(S.elem_order.begin(), S.elem_order.end(), [&](int32_t a, int32_t b) {
        if (ecell[a] != ecell[b]) return ecell[a] < ecell[b];
        const int32_t pa = elem_part ? elem_part[a] : 0, pb = elem_part ? elem_part[b] : 0;
        return pa < pb;
    });

    // ---- A_r = sum over cells of sum_e J_e^T A^e J_e  (Eq. (12)) --------------
    // or, for the full-support operators, A_r = J^T A J assembled element by
    // element from the rows of J at the element's nodes
    if (S.nr > 0) {
        std::vector<int64_t> cell_ptr(ncell + 1, 0);
        for (int64_t i = 0; i < ne; ++i) cell_ptr[ecell[S.elem_order[i]] + 1]++;
        for (int64_t c = 0; c < ncell; ++c) cell_ptr[c + 1] += cell_ptr[c];
        const int64_t nr = S.nr;
        std::vector<double> Ar((size_t)nr * nr, 0.0);
        if (prm.coarse_operator != CGS_COARSE_OP_CELLWISE) {
            // rows of J (J~ = W Q^T J_L, or the vertex-based J) by node: from the
            // box lists, each (cell, weight) times the cell's 8 trilinear weights
            std::vector<int64_t> jr_ptr(nv + 1, 0);
            std::vector<int32_t> jr_col;
            std::vector<double> jr_val;
            {
                std::vector<int64_t> cnt(nv, 0);
                for (size_t i = 0; i < S.vb_vert.size(); ++i) cnt[S.vb_vert[i]] = 8 * (S.vb_ptr[i + 1] - S.vb_ptr[i]);
                for (int64_t v = 0; v < nv; ++v) jr_ptr[v + 1] = jr_ptr[v] + cnt[v];
                jr_col.assign(jr_ptr[nv], -1);
                jr_val.assign(jr_ptr[nv], 0.0);
                for (size_t i = 0; i < S.vb_vert.size(); ++i) {
                    const int32_t v = S.vb_vert[i];
                    int64_t o = jr_ptr[v];
                    for (int32_t e = S.vb_ptr[i]; e < S.vb_ptr[i + 1]; ++e) {
                        const int32_t pc = S.vb_cell[e];
                        const int ci = pc & 1023, cj = (pc >> 10) & 1023, ck = pc >> 20;
                        const int64_t cid = ci + (int64_t)bx * (cj + (int64_t)by * ck);
                        for (int m = 0; m < 8; ++m, ++o) {
                            jr_col[o] = S.cell_cols[cid * 8 + m];
                            jr_val[o] = S.vb_w[e] * corner_weight(&xyz[(size_t)v * 3], ci, cj, ck, m);
                        }
                    }
                }
            }
            // cells in chunks: each chunk's cells assembled in parallel into
            // their own blocks, then added into A_r in cell order (the sums do
            // not depend on the thread count)
            constexpr int64_t kChunk = 64;
            std::vector<std::vector<int32_t>> Uc(kChunk);
            std::vector<std::vector<double>> Kc(kChunk);
            for (int64_t c0 = 0; c0 < ncell; c0 += kChunk) {
                const int64_t c1 = std::min(ncell, c0 + kChunk);
#pragma omp parallel
                {
                    std::vector<std::pair<int32_t, double>> rows[8];
#pragma omp for schedule(dynamic, 1)
                    for (int64_t c = c0; c < c1; ++c) {
                        // the cell's columns, then its elements' J^T A^e J on them
                        std::vector<int32_t>& U = Uc[c - c0];
                        std::vector<double>& KL = Kc[c - c0];
                        U.clear();
                        for (int64_t i = cell_ptr[c]; i < cell_ptr[c + 1]; ++i) {
                            const int64_t e = S.elem_order[i];
                            for (int k = 0; k < 8; ++k) {
                                const int32_t v = conn[e * 8 + k];
                                for (int64_t o = jr_ptr[v]; o < jr_ptr[v + 1]; ++o)
                                    if (jr_col[o] >= 0) U.push_back(jr_col[o]);
                            }
                        }
                        std::sort(U.begin(), U.end());
                        U.erase(std::unique(U.begin(), U.end()), U.end());
                        const size_t L = U.size();
                        KL.assign(L * L, 0.0);
                        for (int64_t i = cell_ptr[c]; i < cell_ptr[c + 1]; ++i) {
                            const int64_t e = S.elem_order[i];
                            for (int k = 0; k < 8; ++k) {
                                rows[k].clear();
                                const int32_t v = conn[e * 8 + k];
                                for (int64_t o = jr_ptr[v]; o < jr_ptr[v + 1]; ++o)
                                    if (jr_col[o] >= 0 && jr_val[o] != 0.0)
                                        rows[k].emplace_back(
                                            (int32_t)(std::lower_bound(U.begin(), U.end(), jr_col[o]) - U.begin()),
                                            jr_val[o]);
                            }
                            const double* A = &Ae[(size_t)e * 64];
                            for (int k = 0; k < 8; ++k)
                                for (int l = 0; l < 8; ++l) {
                                    const double a = A[k * 8 + l];
                                    if (a == 0.0) continue;
                                    for (const auto& ri : rows[k])
                                        for (const auto& rj : rows[l])
                                            KL[(size_t)ri.first * L + rj.first] += a * ri.second * rj.second;
                                }
                        }
                    }
                }
                for (int64_t c = c0; c < c1; ++c) {
                    const std::vector<int32_t>& U = Uc[c - c0];
                    const std::vector<double>& KL = Kc[c - c0];
                    const size_t L = U.size();
                    for (size_t i = 0; i < L; ++i)
                        for (size_t j = 0; j < L; ++j) Ar[(size_t)U[i] * nr + U[j]] += KL[i * L + j];
                }
            }
        } else {
        std::vector<double> Kc((size_t)ncell * 64, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t c = 0; c < ncell; ++c) {
            double* K = &Kc[(size_t)c * 64];
            for (int64_t i = cell_ptr[c]; i < cell_ptr[c + 1]; ++i) {
                const int64_t e = S.elem_order[i];
                double W[8][8];
                weights(e, W);
                for (int m = 0; m < 8; ++m)
                    if (S.cell_cols[c * 8 + m] < 0)
                        for (int k = 0; k < 8; ++k) W[k][m] = 0.0;
                const double* A = &Ae[(size_t)e * 64];
                double AW[8][8];  // A^e J_e
                for (int k = 0; k < 8; ++k)
                    for (int m = 0; m < 8; ++m) {
                        double s = 0.0;
                        for (int l = 0; l < 8; ++l) s += A[k * 8 + l] * W[l][m];
                        AW[k][m] = s;
                    }
                for (int m = 0; m < 8; ++m)
                    for (int n = 0; n < 8; ++n) {
                        double s = 0.0;
                        for (int k = 0; k < 8; ++k) s += W[k][m] * AW[k][n];
                        K[m * 8 + n] += s;
                    }
            }
        }
        for (int64_t c = 0; c < ncell; ++c)
            for (int m = 0; m < 8; ++m) {
                const int32_t a = S.cell_cols[c * 8 + m];
                if (a < 0) continue;
                for (int n = 0; n < 8; ++n) {
                    const int32_t b = S.cell_cols[c * 8 + n];
                    if (b >= 0) Ar[(size_t)a * nr + b] += Kc[(size_t)c * 64 + m * 8 + n];
                }
            }
        }
        S.ar_nnz = 0;
        for (size_t i = 0; i < Ar.size(); ++i) S.ar_nnz += Ar[i] != 0.0;
        const int want = prm.coarse_solver == CGS_COARSE_AUTO
                             ? (nr > CGS_COARSE_AUTO_XXT_NR ? CGS_COARSE_XXT : CGS_COARSE_DENSE)
                             : (int)prm.coarse_solver;
        if (want == CGS_COARSE_XXT) {
            if (nr > 65535) {
                err = "XX^T reduced solver needs n_r <= 65535 (16-bit indices)";
                return CGS_ERR_INVALID_ARG;
            }
            // lattice coordinates of the active box vertices
            const int64_t nbx = bx + 1, nby = by + 1;
            std::vector<std::array<int, 3>> lc(nr);
            for (int64_t a = 0; a < nr; ++a) {
                const int64_t g = S.box_active[a];
                lc[a] = {(int)(g % nbx), (int)((g / nbx) % nby), (int)(g / (nbx * nby))};
            }
            std::vector<int32_t> all(nr);
            std::iota(all.begin(), all.end(), 0);
            S.nd_perm.clear();
            nd_order(lc, std::move(all), S.nd_perm);
            if (!xxt_factor(Ar.data(), nr, S.nd_perm, nthreads, S)) {
                err = "reduced matrix A_r is not SPD";
                return CGS_ERR_NOT_SPD;
            }
            S.coarse = CGS_COARSE_XXT;
        } else {
            S.ar_inv.assign((size_t)nr * nr, 0.0);
            if (!spd_inverse(Ar.data(), (int)nr, S.ar_inv.data(), nthreads)) {
                err = "reduced matrix A_r is not SPD";
                return CGS_ERR_NOT_SPD;
            }
            S.coarse = CGS_COARSE_DENSE;
        }
    }

    // ---- device-order element data ------------------------------------------
    S.conn.resize((size_t)ne * 8);
    S.cell.resize(ne);
    S.a36.resize((size_t)kUpper * ne);
    S.a28.resize((size_t)kOff * ne);
    S.a28lo.resize((size_t)kOff * ne);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; ++i) {
        const int64_t e = S.elem_order[i];
        for (int k = 0; k < 8; ++k) {
            const int32_t v = conn[e * 8 + k];
            S.conn[(size_t)i * 8 + k] = S.dir[v] ? ~v : v;
        }
        S.cell[i] = ecell[e];
        const double* A = &Ae[(size_t)e * 64];
        for (int r = 0; r < 8; ++r)
            for (int c = r; c < 8; ++c) {
                S.a36[(size_t)upper_slot(r, c) * ne + i] = A[r * 8 + c];
                if (c > r) {
                    const float hi = (float)A[r * 8 + c];
                    S.a28[(size_t)off_slot(r, c) * ne + i] = hi;
                    S.a28lo[(size_t)off_slot(r, c) * ne + i] = (float)(A[r * 8 + c] - (double)hi);
                }
            }
    }
    // ---- the assembled free block of A, sliced ELL --------------------------
    // B300 issues two FP64 multiply-adds per clock per SM, and the element
    // form of q = A p spends 64 of them per element against about 27 per row
    // of the assembled operator on hexahedral meshes: the FP64 form applies
    // A row by row.  The mixed forms keep the rows as float pairs (hi + lo,
    // about 48 bits) for the outer apply: 27 pair products per row instead of
    // 28 difference-form pair updates of two rows per element.  Each row sums
    // its elements' contributions in float64, in v2e order.
    {
        constexpr int kMaxRow = 64;
        // the entries of row v (caller vertex ids), ascending columns; false
        // if the row has more than kMaxRow
        auto row_of = [&](int64_t v, int32_t* cols, double* vals, int& cnt) {
            cnt = 0;
            if (S.dir[v]) return true;
            for (int64_t t = v2e_ptr[v]; t < v2e_ptr[v + 1]; ++t) {
                const int64_t e = v2e[t];
                int a = 0;
                while (a < 8 && conn[e * 8 + a] != v) ++a;
                const double* A = &Ae[(size_t)e * 64];
                for (int b = 0; b < 8; ++b) {
                    const int32_t u = conn[e * 8 + b];
                    if (S.dir[u]) continue;
                    int q = 0;
                    while (q < cnt && cols[q] != u) ++q;
                    if (q == cnt) {
                        if (cnt == kMaxRow) return false;
                        cols[cnt] = u;
                        vals[cnt] = 0.0;
                        ++cnt;
                    }
                    vals[q] += A[a * 8 + b];
                }
            }
            for (int i = 1; i < cnt; ++i)   // insertion sort by column
                for (int j = i; j > 0 && cols[j - 1] > cols[j]; --j) {
                    std::swap(cols[j - 1], cols[j]);
                    std::swap(vals[j - 1], vals[j]);
                }
            return true;
        };
        const int64_t nsl = (nv + 31) / 32;
        std::vector<int32_t> width(nsl, 0);
        bool fits = true;
#pragma omp parallel for schedule(static) reduction(&& : fits)
        for (int64_t sl = 0; sl < nsl; ++sl) {
            int32_t cols[kMaxRow];
            double vals[kMaxRow];
            int w = 0;
            for (int64_t v = sl * 32; v < std::min<int64_t>(nv, sl * 32 + 32); ++v) {
                int cnt = 0;
                fits = fits && row_of(v, cols, vals, cnt);
                w = std::max(w, cnt);
            }
            width[sl] = w;
        }
        if (fits) {
            // one width for every slice (the widest row; shorter rows are
            // padded), so that entry k of row i sits at a computable place
            const int32_t wmax = nsl ? *std::max_element(width.begin(), width.end()) : 0;
            S.ell_w = wmax;
            S.ell_ptr.assign(nsl + 1, 0);
            for (int64_t sl = 0; sl < nsl; ++sl) S.ell_ptr[sl + 1] = S.ell_ptr[sl] + 32 * (int64_t)wmax;
            S.ell_col.assign(S.ell_ptr[nsl], -1);
            S.ell_val.assign(S.ell_ptr[nsl], 0.0);
            const bool pairs = prm.prec != CGS_FP64;
#pragma omp parallel for schedule(static)
            for (int64_t sl = 0; sl < nsl; ++sl) {
                int32_t cols[kMaxRow];
                double vals[kMaxRow];
                for (int64_t v = sl * 32; v < std::min<int64_t>(nv, sl * 32 + 32); ++v) {
                    int cnt = 0;
                    row_of(v, cols, vals, cnt);
                    for (int k = 0; k < cnt; ++k) {
                        const int64_t o = S.ell_ptr[sl] + 32 * (int64_t)k + (v - sl * 32);
                        S.ell_col[o] = cols[k];
                        S.ell_val[o] = vals[k];
                    }
                }
            }
            if (pairs) {   // float pairs instead of float64 values
                S.ell_pair.assign(2 * S.ell_val.size(), 0.0f);
#pragma omp parallel for schedule(static)
                for (int64_t o = 0; o < (int64_t)S.ell_val.size(); ++o) {
                    const float hi = (float)S.ell_val[o];
                    S.ell_pair[2 * o] = hi;
                    S.ell_pair[2 * o + 1] = (float)(S.ell_val[o] - (double)hi);
                }
                std::vector<double>().swap(S.ell_val);
            }
        }
    }
    // ---- element tiles for block-local assembly --------------------------
    {
        std::vector<int32_t> stamp(nv, -1), loc(nv, 0), in_tile(nv, 0);
        S.tile_ptr.assign(1, 0);
        S.tile_vptr.assign(1, 0);
        S.tile_verts.clear();
        S.eloc.assign((size_t)ne * 8, 0xFFFF);
        int32_t tile = 0, tile_begin = 0;
        std::vector<int32_t> verts;
        auto close_tile = [&](int32_t end) {
            for (int32_t v : verts) {
                const int64_t c = v2e_ptr[v + 1] - v2e_ptr[v];
                S.tile_verts.push_back((uint32_t)v | (in_tile[v] == c ? 0u : kSharedBit));
                in_tile[v] = 0;
            }
            S.tile_ptr.push_back(end);
            S.tile_vptr.push_back((int32_t)S.tile_verts.size());
            verts.clear();
            ++tile;
            tile_begin = end;
        };
        for (int64_t i = 0; i < ne; ++i) {
            int fresh = 0;
            for (int k = 0; k < 8; ++k) {
                const int32_t v = S.conn[(size_t)i * 8 + k];
                if (v >= 0 && stamp[v] != tile) ++fresh;
            }
            if (i - tile_begin >= kTileElems || (int)verts.size() + fresh > kTileVerts) close_tile((int32_t)i);
            for (int k = 0; k < 8; ++k) {
                const int32_t v = S.conn[(size_t)i * 8 + k];
                if (v < 0) continue;
                if (stamp[v] != tile) {
                    stamp[v] = tile;
                    loc[v] = (int32_t)verts.size();
                    verts.push_back(v);
                }
                in_tile[v]++;
                S.eloc[(size_t)i * 8 + k] = (uint16_t)loc[v];
            }
        }
        close_tile((int32_t)ne);
        // tile-major copies of the off-diagonals, zero-padded to kTileElems:
        // [tile][slot / 4][element][slot % 4], so one 16-byte load gives an
        // element four consecutive slots and a warp's load is contiguous
        const int64_t nt = (int64_t)S.tile_ptr.size() - 1;
        S.at_hi.assign((size_t)nt * kOff * kTileElems, 0.0f);
        S.at_lo.assign((size_t)nt * kOff * kTileElems, 0.0f);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < nt; ++t)
            for (int32_t i = S.tile_ptr[t]; i < S.tile_ptr[t + 1]; ++i)
                for (int sl = 0; sl < kOff; ++sl) {
                    const size_t dst =
                        (((size_t)t * (kOff / 4) + sl / 4) * kTileElems + (i - S.tile_ptr[t])) * 4 + sl % 4;
                    S.at_hi[dst] = S.a28[(size_t)sl * ne + i];
                    S.at_lo[dst] = S.a28lo[(size_t)sl * ne + i];
                }
    }
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return CGS_OK;
}

}  // namespace cgs
