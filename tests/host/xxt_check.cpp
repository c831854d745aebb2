// Host-side check of the reduced-solver set-up (no GPU): runs the library's
// host set-up twice on a perturbed structured cube, once with the dense
// explicit inverse and once with XX^T, and checks that
//   * X X^T equals the dense A_r^{-1} on 64 sampled columns (relative max
//     norm printed),
//   * the column-major and row-major copies of X hold the same entries, with
//     rows ascending within each column,
//   * the pass-1 segments tile every column in pieces of at most kXxtSeg.
// Prints one line; exit status 0 when every structural check holds.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <string>
#include <vector>
#include "internal.h"
using namespace cgs;
int main(int argc, char** argv) {
    const int n = argc > 1 ? atoi(argv[1]) : 12, B = argc > 2 ? atoi(argv[2]) : 6;
    const int nv = (n + 1) * (n + 1) * (n + 1), ne = n * n * n;
    std::vector<double> xyz(3 * (size_t)nv);
    for (int k = 0; k <= n; ++k) for (int j = 0; j <= n; ++j) for (int i = 0; i <= n; ++i) {
        const int v = i + (n + 1) * (j + (n + 1) * k);
        xyz[3 * v] = i + 0.1 * std::sin(1.3 * j + k); xyz[3 * v + 1] = j + 0.1 * std::cos(i + 0.7 * k); xyz[3 * v + 2] = k;
    }
    std::vector<int32_t> conn(8 * (size_t)ne), part(ne);
    for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
        const int e = i + n * (j + n * k);
        for (int m = 0; m < 8; ++m) {
            const int a = i + (m & 1), b = j + ((m >> 1) & 1), c = k + ((m >> 2) & 1);
            conn[8 * e + m] = a + (n + 1) * (b + (n + 1) * c);
        }
        part[e] = (i / 2) + (n / 2) * ((j / 2) + (n / 2) * (k / 2));
    }
    cgs_params prm{};
    prm.box[0] = prm.box[1] = prm.box[2] = B; prm.overlap_layers = 1; prm.prec = CGS_FP64; prm.form = CGS_HYBRID;
    HostSetup D, X; std::string err;
    prm.coarse_solver = CGS_COARSE_DENSE;
    if (host_setup(xyz.data(), nv, conn.data(), ne, nullptr, part.data(), prm, D, err) != CGS_OK) { printf("dense: %s\n", err.c_str()); return 1; }
    prm.coarse_solver = CGS_COARSE_XXT;
    if (host_setup(xyz.data(), nv, conn.data(), ne, nullptr, part.data(), prm, X, err) != CGS_OK) { printf("xxt: %s\n", err.c_str()); return 1; }
    const int nr = (int)X.nr;
    // X from the row-major copy, dense
    std::vector<double> Xd((size_t)nr * nr, 0.0);
    for (int i = 0; i < nr; ++i) for (int e = X.xr_ptr[i]; e < X.xr_ptr[i + 1]; ++e) Xd[(size_t)i * nr + X.xr_idx[e]] = X.xr_val[e];
    // the column-major copy holds the same entries, rows ascending
    long bad = 0;
    for (int k = 0; k < nr; ++k) for (int e = X.xc_ptr[k]; e < X.xc_ptr[k + 1]; ++e) {
        if (Xd[(size_t)X.xc_idx[e] * nr + k] != X.xc_val[e]) ++bad;
        if (e > X.xc_ptr[k] && X.xc_idx[e] <= X.xc_idx[e - 1]) ++bad;
    }
    // segments tile the columns
    long segn = 0; int prevk = -1, prevend = 0;
    for (size_t s = 0; s < X.xs_seg.size(); s += 4) {
        const int k = X.xs_seg[s], b = X.xs_seg[s + 1], e = X.xs_seg[s + 2];
        if (k != prevk) { if (b != X.xc_ptr[k]) ++bad; } else if (b != prevend) ++bad;
        if (e - b > kXxtSeg || e <= b) ++bad;
        prevk = k; prevend = e; ++segn;
    }
    // X X^T e_j = X (row j of X)^T for 64 sampled columns j, sparse
    double md = 0, mx = 0;
    std::vector<double> y(nr), col(nr);
    for (int smp = 0; smp < 64 && smp < nr; ++smp) {
        const int j = (int)(((long long)smp * 7919) % nr);
        std::fill(col.begin(), col.end(), 0.0);
        for (int e = X.xr_ptr[j]; e < X.xr_ptr[j + 1]; ++e) col[X.xr_idx[e]] = X.xr_val[e];
        for (int i = 0; i < nr; ++i) {
            double s = 0;
            for (int e = X.xr_ptr[i]; e < X.xr_ptr[i + 1]; ++e) s += X.xr_val[e] * col[X.xr_idx[e]];
            y[i] = s;
        }
        for (int i = 0; i < nr; ++i) {
            md = std::max(md, std::fabs(y[i] - D.ar_inv[(size_t)i * nr + j]));
            mx = std::max(mx, std::fabs(D.ar_inv[(size_t)i * nr + j]));
        }
    }
    printf("n=%d boxes=%d nr=%d nnz=%zu (%.3f of dense) segments=%ld consistency errors=%ld |XX^T - inv|/|inv| = %.2e\n",
           n, B, nr, X.xc_idx.size(), (double)X.xc_idx.size() / ((double)nr * nr), segn, bad, md / mx);
    return bad ? 2 : 0;
}
