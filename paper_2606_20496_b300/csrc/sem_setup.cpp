// Host set-up of the spectral-element levels of the p-multigrid wrap (Sec. 1,
// Sec. 5, Eqs. (13) and (14)): GLL rules, global node numbering, geometric
// factors, Dirichlet nodes and the fast-diagonalisation factors of the
// element-local Schwarz smoother.
//
// Readings (the paper defers the smoother to its references): the element is
// the trilinear image of its 8 vertices; the Dirichlet nodes are the nodes of
// boundary faces; the local problem of Eq. (14) is the separable operator
// B_z (x) B_y (x) A_x + B_z (x) A_y (x) B_x + A_z (x) B_y (x) B_x whose 1D
// factors are the element's 1D GLL stiffness and mass for the mean edge
// length of that direction, plus the corner entry of an equal neighbour at
// each shared end (the neighbour's first interior node held at zero), or with
// the end node dropped on a Dirichlet face.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sem.h"

namespace cgs {

namespace {

// P_n(x) and P_n'(x) by the three-term recurrence and the derivative
// recurrence P_k' = P_{k-2}' + (2k - 1) P_{k-1}
void legendre_pd(int n, double x, double& p, double& dp) {
    double pm2 = 1.0, pm1 = x, dpm2 = 0.0, dpm1 = 1.0;
    if (n == 0) {
        p = 1.0;
        dp = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * x * pm1 - (k - 1.0) * pm2) / k;
        const double dpk = dpm2 + (2.0 * k - 1.0) * pm1;
        pm2 = pm1;
        pm1 = pk;
        dpm2 = dpm1;
        dpm1 = dpk;
    }
    p = pm1;
    dp = dpm1;
}

// cyclic Jacobi rotations on the symmetric m x m matrix C (row-major),
// eigenvectors in the columns of V
void jacobi_eigen(int m, std::vector<double>& C, std::vector<double>& V) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double c2 = C[(size_t)i * m + j] * C[(size_t)i * m + j];
                tot += c2;
                if (i != j) off += c2;
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = C[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double tau = (C[(size_t)q * m + q] - C[(size_t)p * m + p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                // C <- R^T C R with R the rotation in the (p, q) plane
                for (int k = 0; k < m; ++k) {
                    const double ckp = C[(size_t)k * m + p], ckq = C[(size_t)k * m + q];
                    C[(size_t)k * m + p] = c * ckp - s * ckq;
                    C[(size_t)k * m + q] = s * ckp + c * ckq;
                }
                for (int k = 0; k < m; ++k) {
                    const double cpk = C[(size_t)p * m + k], cqk = C[(size_t)q * m + k];
                    C[(size_t)p * m + k] = c * cpk - s * cqk;
                    C[(size_t)q * m + k] = s * cpk + c * cqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
                    V[(size_t)k * m + p] = c * vkp - s * vkq;
                    V[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
    }
}

// trilinear shape function v and its reference gradient at (r, s, t)
inline void trilinear(int v, double r, double s, double t, double& phi, double g[3]) {
    const double xi[3] = {r, s, t};
    double f[3], df[3];
    for (int d = 0; d < 3; ++d) {
        const int bit = (v >> d) & 1;
        f[d] = bit ? 0.5 * (1.0 + xi[d]) : 0.5 * (1.0 - xi[d]);
        df[d] = bit ? 0.5 : -0.5;
    }
    phi = f[0] * f[1] * f[2];
    g[0] = df[0] * f[1] * f[2];
    g[1] = f[0] * df[1] * f[2];
    g[2] = f[0] * f[1] * df[2];
}

// the 4 local vertices of face (d, side), in the order (ca, cb) = (0,0), (1,0),
// (0,1), (1,1) over the two other directions da < db
inline void face_vertices(int d, int side, int out[4], int& da, int& db) {
    da = d == 0 ? 1 : 0;
    db = d == 2 ? 1 : 2;
    for (int cb = 0; cb < 2; ++cb)
        for (int ca = 0; ca < 2; ++ca) out[ca + 2 * cb] = (side << d) | (ca << da) | (cb << db);
}

using Face = std::array<int32_t, 4>;

// face ids (sorted vertex quadruples) of every element face, and the number
// of elements holding each face
void number_faces(const int32_t* conn, int64_t ne, std::vector<int64_t>& fid, std::vector<int>& owners,
                  int64_t& nfaces) {
    std::vector<std::pair<Face, int64_t>> all((size_t)ne * 6);
    for (int64_t e = 0; e < ne; ++e)
        for (int f = 0; f < 6; ++f) {
            int v[4], da, db;
            face_vertices(f / 2, f % 2, v, da, db);
            Face k{conn[e * 8 + v[0]], conn[e * 8 + v[1]], conn[e * 8 + v[2]], conn[e * 8 + v[3]]};
            std::sort(k.begin(), k.end());
            all[(size_t)e * 6 + f] = {k, e * 6 + f};
        }
    std::sort(all.begin(), all.end());
    fid.assign((size_t)ne * 6, -1);
    owners.clear();
    nfaces = 0;
    for (size_t i = 0; i < all.size();) {
        size_t j = i;
        while (j < all.size() && all[j].first == all[i].first) ++j;
        for (size_t k = i; k < j; ++k) fid[all[k].second] = nfaces;
        owners.push_back((int)(j - i));
        ++nfaces;
        i = j;
    }
}

}  // namespace

void gll_rule(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n + 1, 0.0);
    w.assign(n + 1, 0.0);
    x[0] = -1.0;
    x[n] = 1.0;
    // interior nodes: roots of P_n', Newton from the Chebyshev-Lobatto points
    // with P_n'' from the Legendre equation
    for (int i = 1; i < n; ++i) {
        double t = -std::cos(M_PI * i / n);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre_pd(n, t, p, dp);
            const double d2p = (2.0 * t * dp - n * (n + 1.0) * p) / (1.0 - t * t);
            const double step = dp / d2p;
            t -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[i] = t;
    }
    for (int i = 0; i <= n / 2; ++i) {     // exact symmetry x_{n-i} = -x_i
        const double s = 0.5 * (x[n - i] - x[i]);
        x[n - i] = s;
        x[i] = -s;
    }
    if (n % 2 == 0) x[n / 2] = 0.0;
    for (int i = 0; i <= n; ++i) {
        double p, dp;
        legendre_pd(n, x[i], p, dp);
        w[i] = 2.0 / (n * (n + 1.0) * p * p);
    }
}

void gll_derivative(int n, const std::vector<double>& x, std::vector<double>& D) {
    // l_j'(x_i) = P_n(x_i) / (P_n(x_j) (x_i - x_j)) off the diagonal; the
    // diagonal is -n(n+1)/4 at x_0, n(n+1)/4 at x_n and 0 inside
    const int p = n + 1;
    std::vector<double> P(p);
    for (int i = 0; i < p; ++i) {
        double dp;
        legendre_pd(n, x[i], P[i], dp);
    }
    D.assign((size_t)p * p, 0.0);
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            if (i != j) D[(size_t)i * p + j] = P[i] / (P[j] * (x[i] - x[j]));
    D[0] = -0.25 * n * (n + 1.0);
    D[(size_t)n * p + n] = 0.25 * n * (n + 1.0);
}

void lagrange_interp(const std::vector<double>& xc, const std::vector<double>& xf, std::vector<double>& I) {
    const int pc = (int)xc.size(), pf = (int)xf.size();
    I.assign((size_t)pf * pc, 1.0);
    for (int i = 0; i < pf; ++i)
        for (int j = 0; j < pc; ++j)
            for (int k = 0; k < pc; ++k)
                if (k != j) I[(size_t)i * pc + j] *= (xf[i] - xc[k]) / (xc[j] - xc[k]);
}

std::vector<uint8_t> sem_boundary_vertices(const int32_t* conn, int64_t ne, int64_t nv) {
    std::vector<int64_t> fid;
    std::vector<int> owners;
    int64_t nf = 0;
    number_faces(conn, ne, fid, owners, nf);
    std::vector<uint8_t> dir((size_t)nv, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int f = 0; f < 6; ++f)
            if (owners[fid[(size_t)e * 6 + f]] == 1) {
                int v[4], da, db;
                face_vertices(f / 2, f % 2, v, da, db);
                for (int k = 0; k < 4; ++k) dir[conn[e * 8 + v[k]]] = 1;
            }
    return dir;
}

std::string sem_build_level(int n, const double* xyz, int64_t nv, const int32_t* conn, int64_t ne,
                            SemHostLevel& L) {
    if (n < kSemMinOrder || n > kSemMaxOrder) return "order out of range";
    const int p = n + 1, p3 = p * p * p, m = n - 1;
    L.n = n;
    L.p = p;
    std::vector<double> w;
    gll_rule(n, L.x, w);
    gll_derivative(n, L.x, L.D);

    // ---- edges: sorted vertex pairs -> edge id
    std::vector<std::pair<uint64_t, int64_t>> ekeys((size_t)ne * 12);
    for (int64_t e = 0; e < ne; ++e) {
        int c = 0;
        for (int d = 0; d < 3; ++d)
            for (int v = 0; v < 8; ++v)
                if (!((v >> d) & 1)) {
                    const uint32_t a = (uint32_t)conn[e * 8 + v], b = (uint32_t)conn[e * 8 + (v | (1 << d))];
                    ekeys[(size_t)e * 12 + c] = {((uint64_t)std::min(a, b) << 32) | std::max(a, b), e * 12 + c};
                    ++c;
                }
    }
    std::sort(ekeys.begin(), ekeys.end());
    std::vector<int64_t> eid((size_t)ne * 12);
    int64_t nedges = 0;
    for (size_t i = 0; i < ekeys.size();) {
        size_t j = i;
        while (j < ekeys.size() && ekeys[j].first == ekeys[i].first) ++j;
        for (size_t k = i; k < j; ++k) eid[ekeys[k].second] = nedges;
        ++nedges;
        i = j;
    }
    // ---- faces
    std::vector<int64_t> fid;
    std::vector<int> owners;
    int64_t nfaces = 0;
    number_faces(conn, ne, fid, owners, nfaces);

    const int64_t off_e = nv, off_f = off_e + nedges * m, off_i = off_f + nfaces * (int64_t)m * m;
    L.ng = off_i + ne * (int64_t)m * m * m;
    if (L.ng >= (int64_t)INT32_MAX) return "too many nodes for 32-bit indices";
    L.l2g.assign((size_t)ne * p3, 0);
    bool bad = false;
#pragma omp parallel for schedule(static) reduction(|| : bad)
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* cv = conn + e * 8;
        // the edge slot of (direction d, fixed bits) in the order ekeys used
        auto edge_slot = [&](int d, int v0) {
            int c = 0;
            for (int dd = 0; dd < 3; ++dd)
                for (int v = 0; v < 8; ++v)
                    if (!((v >> dd) & 1)) {
                        if (dd == d && v == v0) return c;
                        ++c;
                    }
            return -1;
        };
        for (int k = 0; k < p; ++k)
            for (int j = 0; j < p; ++j)
                for (int i = 0; i < p; ++i) {
                    const int idx[3] = {i, j, k};
                    int at_end = 0;
                    for (int d = 0; d < 3; ++d) at_end += (idx[d] == 0 || idx[d] == n);
                    int64_t g = -1;
                    if (at_end == 3) {
                        g = cv[(i / n) | ((j / n) << 1) | ((k / n) << 2)];
                    } else if (at_end == 2) {
                        int d = 0;
                        for (int dd = 0; dd < 3; ++dd)
                            if (idx[dd] != 0 && idx[dd] != n) d = dd;   // the free direction
                        int v0 = 0;
                        for (int dd = 0; dd < 3; ++dd)
                            if (dd != d && idx[dd] == n) v0 |= 1 << dd;
                        const int v1 = v0 | (1 << d);
                        const int t = idx[d];
                        const int pos = cv[v0] < cv[v1] ? t : n - t;
                        const int slot = edge_slot(d, v0);
                        g = off_e + eid[(size_t)e * 12 + slot] * m + (pos - 1);
                    } else if (at_end == 1) {
                        int d0 = 0;
                        for (int dd = 0; dd < 3; ++dd)
                            if (idx[dd] == 0 || idx[dd] == n) d0 = dd;
                        const int side = idx[d0] == n;
                        int fv[4], da, db;
                        face_vertices(d0, side, fv, da, db);
                        int cmin = 0;
                        for (int c = 1; c < 4; ++c)
                            if (cv[fv[c]] < cv[fv[cmin]]) cmin = c;
                        const int ca0 = cmin & 1, cb0 = cmin >> 1;
                        const int ia = idx[da], ib = idx[db];
                        const int dist_a = ca0 ? n - ia : ia, dist_b = cb0 ? n - ib : ib;
                        const int nb_a = fv[(1 - ca0) + 2 * cb0], nb_b = fv[ca0 + 2 * (1 - cb0)];
                        int u, v;
                        if (cv[nb_a] < cv[nb_b]) {
                            u = dist_a;
                            v = dist_b;
                        } else {
                            u = dist_b;
                            v = dist_a;
                        }
                        g = off_f + fid[(size_t)e * 6 + 2 * d0 + side] * m * m + (int64_t)(u - 1) * m + (v - 1);
                    } else {
                        g = off_i + e * (int64_t)m * m * m + ((int64_t)(k - 1) * m + (j - 1)) * m + (i - 1);
                    }
                    if (g < 0 || g >= L.ng) bad = true;
                    L.l2g[(size_t)e * p3 + (k * p + j) * p + i] = (int32_t)g;
                }
    }
    if (bad) return "node numbering out of range";

    // ---- Dirichlet nodes: every node of a boundary face
    L.dir.assign((size_t)L.ng, 0);
    std::vector<uint8_t> fbd((size_t)ne * 6, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int f = 0; f < 6; ++f) {
            if (owners[fid[(size_t)e * 6 + f]] != 1) continue;
            fbd[(size_t)e * 6 + f] = 1;
            const int d = f / 2, side = f % 2;
            for (int a = 0; a < p; ++a)
                for (int b = 0; b < p; ++b) {
                    int idx[3];
                    idx[d] = side ? n : 0;
                    idx[d == 0 ? 1 : 0] = a;
                    idx[d == 2 ? 1 : 2] = b;
                    L.dir[L.l2g[(size_t)e * p3 + (idx[2] * p + idx[1]) * p + idx[0]]] = 1;
                }
        }
    L.nfree = 0;
    for (int64_t g = 0; g < L.ng; ++g) L.nfree += !L.dir[g];
    // ---- multiplicities
    std::vector<int32_t> cnt((size_t)L.ng, 0);
    for (size_t q = 0; q < L.l2g.size(); ++q) ++cnt[L.l2g[q]];
    L.inv_mult.resize((size_t)L.ng);
    for (int64_t g = 0; g < L.ng; ++g) L.inv_mult[g] = cnt[g] ? 1.0 / cnt[g] : 0.0;

    // ---- geometric factors w det J (J^-1 J^-T) at the GLL nodes
    L.G.assign((size_t)ne * 6 * p3, 0.0);
    bool nonpos = false;
#pragma omp parallel for schedule(static) reduction(|| : nonpos)
    for (int64_t e = 0; e < ne; ++e) {
        double X[8][3];
        for (int v = 0; v < 8; ++v)
            for (int c = 0; c < 3; ++c) X[v][c] = xyz[(size_t)conn[e * 8 + v] * 3 + c];
        for (int k = 0; k < p; ++k)
            for (int j = 0; j < p; ++j)
                for (int i = 0; i < p; ++i) {
                    double J[3][3] = {{0}};   // J[c][a] = dx_c / dxi_a
                    for (int v = 0; v < 8; ++v) {
                        double phi, gr[3];
                        trilinear(v, L.x[i], L.x[j], L.x[k], phi, gr);
                        for (int c = 0; c < 3; ++c)
                            for (int a = 0; a < 3; ++a) J[c][a] += X[v][c] * gr[a];
                    }
                    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                    if (!(det > 0.0)) nonpos = true;
                    // inverse: Ji[a][c] = dxi_a / dx_c = cofactor(J)[c][a] / det
                    double Ji[3][3];
                    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
                    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
                    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
                    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
                    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
                    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
                    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
                    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
                    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
                    const double s = w[i] * w[j] * w[k] * det;
                    const int ab[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
                    const int node = (k * p + j) * p + i;
                    for (int q = 0; q < 6; ++q) {
                        const int a = ab[q][0], b = ab[q][1];
                        L.G[((size_t)e * 6 + q) * p3 + node] =
                            s * (Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2]);
                    }
                }
    }
    if (nonpos) return "element with a non-positive Jacobian at a GLL node";

    // ---- fast diagonalisation of the element-local Schwarz problems
    std::vector<double> Ahat((size_t)p * p, 0.0);
    for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b)
            for (int q = 0; q < p; ++q) Ahat[(size_t)a * p + b] += L.D[(size_t)q * p + a] * w[q] * L.D[(size_t)q * p + b];
    L.S.assign((size_t)ne * 3 * p * p, 0.0);
    L.lam.assign((size_t)ne * 3 * p, 1.0);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
        for (int d = 0; d < 3; ++d) {
            // mean length of the element's four edges along d
            double len = 0.0;
            for (int v = 0; v < 8; ++v)
                if (!((v >> d) & 1)) {
                    const int32_t a = conn[e * 8 + v], b = conn[e * 8 + (v | (1 << d))];
                    double s2 = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        const double t = xyz[(size_t)b * 3 + c] - xyz[(size_t)a * 3 + c];
                        s2 += t * t;
                    }
                    len += 0.25 * std::sqrt(s2);
                }
            std::vector<double> A((size_t)p * p), B(p);
            for (int q = 0; q < p * p; ++q) A[q] = (2.0 / len) * Ahat[q];
            for (int q = 0; q < p; ++q) B[q] = 0.5 * len * w[q];
            const bool lo_dir = fbd[(size_t)e * 6 + 2 * d], hi_dir = fbd[(size_t)e * 6 + 2 * d + 1];
            if (!lo_dir) {
                A[0] += (2.0 / len) * Ahat[(size_t)n * p + n];
                B[0] += 0.5 * len * w[n];
            }
            if (!hi_dir) {
                A[(size_t)n * p + n] += (2.0 / len) * Ahat[0];
                B[n] += 0.5 * len * w[0];
            }
            std::vector<int> keep;
            for (int q = 0; q < p; ++q)
                if (!((q == 0 && lo_dir) || (q == n && hi_dir))) keep.push_back(q);
            const int mk = (int)keep.size();
            // A s = lam B s with B diagonal: C = B^-1/2 A B^-1/2, S = B^-1/2 V
            std::vector<double> C((size_t)mk * mk), V;
            for (int a = 0; a < mk; ++a)
                for (int b = 0; b < mk; ++b)
                    C[(size_t)a * mk + b] =
                        A[(size_t)keep[a] * p + keep[b]] / std::sqrt(B[keep[a]] * B[keep[b]]);
            jacobi_eigen(mk, C, V);
            double* S = &L.S[((size_t)e * 3 + d) * p * p];
            double* lam = &L.lam[((size_t)e * 3 + d) * p];
            for (int md = 0; md < mk; ++md) {
                lam[md] = C[(size_t)md * mk + md];
                for (int a = 0; a < mk; ++a) S[(size_t)keep[a] * p + md] = V[(size_t)a * mk + md] / std::sqrt(B[keep[a]]);
            }
        }
    }
    return "";
}

void sem_node_coords(int n, const double* xyz, const int32_t* conn, int64_t ne, const std::vector<int32_t>& l2g,
                     int64_t ng, double* out) {
    const int p = n + 1, p3 = p * p * p;
    std::vector<double> x, w;
    gll_rule(n, x, w);
    (void)ng;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e)
        for (int k = 0; k < p; ++k)
            for (int j = 0; j < p; ++j)
                for (int i = 0; i < p; ++i) {
                    double pos[3] = {0, 0, 0};
                    for (int v = 0; v < 8; ++v) {
                        double phi, gr[3];
                        trilinear(v, x[i], x[j], x[k], phi, gr);
                        for (int c = 0; c < 3; ++c) pos[c] += phi * xyz[(size_t)conn[e * 8 + v] * 3 + c];
                    }
                    int32_t g = l2g[(size_t)e * p3 + (k * p + j) * p + i];
                    if (g < 0) g = -g - 1;
                    for (int c = 0; c < 3; ++c) out[(size_t)g * 3 + c] = pos[c];
                }
}

}  // namespace cgs
