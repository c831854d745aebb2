// Host-side check of the spectral-element set-up (no GPU): reads a mesh
// written by the test (order n, nv ne, then xyz and conn), builds the level
// of order n with the library's host set-up (csrc/sem_setup.cpp) and writes,
// for the test to compare with the oracle: p, the node counts, the GLL
// nodes, D, and per element its global node numbers, metric (six entries per
// node), smoother factors S and eigenvalues; then the Dirichlet flag and
// 1 / multiplicity of every global node.
#include <cstdio>
#include <string>
#include <vector>
#include "sem.h"
using namespace cgs;
int main(int argc, char** argv) {
    if (argc < 3) return 2;
    FILE* in = fopen(argv[1], "r");
    if (!in) return 2;
    int n = 0;
    long nv = 0, ne = 0;
    if (fscanf(in, "%d %ld %ld", &n, &nv, &ne) != 3) return 2;
    std::vector<double> xyz(3 * (size_t)nv);
    std::vector<int32_t> conn(8 * (size_t)ne);
    for (auto& v : xyz)
        if (fscanf(in, "%lf", &v) != 1) return 2;
    for (auto& v : conn)
        if (fscanf(in, "%d", &v) != 1) return 2;
    fclose(in);
    SemHostLevel L;
    const std::string err = sem_build_level(n, xyz.data(), nv, conn.data(), ne, L);
    if (!err.empty()) {
        printf("%s\n", err.c_str());
        return 1;
    }
    const int p = L.p, p3 = p * p * p;
    FILE* f = fopen(argv[2], "w");
    fprintf(f, "%d %ld %ld\n", p, (long)L.ng, (long)L.nfree);
    for (double v : L.x) fprintf(f, "%.17g ", v);
    fprintf(f, "\n");
    for (double v : L.D) fprintf(f, "%.17g ", v);
    fprintf(f, "\n");
    for (long e = 0; e < ne; ++e) {
        for (int q = 0; q < p3; ++q) fprintf(f, "%d ", L.l2g[(size_t)e * p3 + q]);
        fprintf(f, "\n");
        for (int q = 0; q < 6 * p3; ++q) fprintf(f, "%.17g ", L.G[(size_t)e * 6 * p3 + q]);
        fprintf(f, "\n");
        for (int q = 0; q < 3 * p * p; ++q) fprintf(f, "%.17g ", L.S[(size_t)e * 3 * p * p + q]);
        fprintf(f, "\n");
        for (int q = 0; q < 3 * p; ++q) fprintf(f, "%.17g ", L.lam[(size_t)e * 3 * p + q]);
        fprintf(f, "\n");
    }
    for (long g = 0; g < L.ng; ++g) fprintf(f, "%d %.17g\n", (int)L.dir[g], L.inv_mult[g]);
    fclose(f);
    return 0;
}
