// Host-side check of the three coarse operators (no GPU): runs the library's
// host set-up on a perturbed 8^3 cube with 4^3 boxes for the cell-wise,
// Galerkin and vertex-based operators and writes, for the test to compare
// with the oracle: the vertex coordinates, then per operator n_r, nnz(A_r),
// the active box-vertex ids and the dense A_r^{-1}.
#include <cstdio>
#include <cmath>
#include <string>
#include <vector>
#include "internal.h"
using namespace cgs;
int main(int argc, char** argv) {
    const int n = 8, B = 4;
    const int nv = (n + 1) * (n + 1) * (n + 1), ne = n * n * n;
    std::vector<double> xyz(3 * (size_t)nv);
    for (int k = 0; k <= n; ++k) for (int j = 0; j <= n; ++j) for (int i = 0; i <= n; ++i) {
        const int v = i + (n + 1) * (j + (n + 1) * k);
        xyz[3 * v] = i + 0.2 * std::sin(1.3 * j + k); xyz[3 * v + 1] = j + 0.2 * std::cos(i + 0.7 * k); xyz[3 * v + 2] = k + 0.1 * std::sin(i + j);
    }
    std::vector<int32_t> conn(8 * (size_t)ne), part(ne);
    for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
        const int e = i + n * (j + n * k);
        for (int m = 0; m < 8; ++m) conn[8 * e + m] = (i + (m & 1)) + (n + 1) * ((j + ((m >> 1) & 1)) + (n + 1) * (k + ((m >> 2) & 1)));
        part[e] = (i / 2) + (n / 2) * ((j / 2) + (n / 2) * (k / 2));
    }
    FILE* f = fopen(argv[1], "w");
    fprintf(f, "%d\n", nv);
    for (int v = 0; v < nv; ++v) fprintf(f, "%.17g %.17g %.17g\n", xyz[3*v], xyz[3*v+1], xyz[3*v+2]);
    for (int op = 0; op < 3; ++op) {
        cgs_params prm{};
        prm.box[0] = prm.box[1] = prm.box[2] = B; prm.overlap_layers = 1; prm.prec = CGS_FP64; prm.form = CGS_HYBRID;
        prm.coarse_solver = CGS_COARSE_DENSE; prm.coarse_operator = (cgs_coarse_operator)op;
        HostSetup S; std::string err;
        if (host_setup(xyz.data(), nv, conn.data(), ne, nullptr, part.data(), prm, S, err) != CGS_OK) { printf("%s\n", err.c_str()); return 1; }
        // A_r from its inverse is not kept; dump the inverse and the active ids
        fprintf(f, "%ld %ld\n", (long)S.nr, (long)S.ar_nnz);
        for (int64_t a = 0; a < S.nr; ++a) fprintf(f, "%ld ", (long)S.box_active[a]);
        fprintf(f, "\n");
        for (size_t i = 0; i < S.ar_inv.size(); ++i) fprintf(f, "%.17g\n", S.ar_inv[i]);
    }
    fclose(f);
    return 0;
}
