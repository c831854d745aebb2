// Host-side check of the explicit interpolation rows and hybrid-restriction
// entries (no GPU): reads a mesh written by the test (nv ne b0 b1 b2, then
// xyz, conn and part), runs the library's host set-up in the FP64 hybrid
// form and writes n_r, then the rows of J~ (vertex, then its (column,
// weight) pairs, padding left out) and the entries (vertex, column, J~_vc,
// (A J~)_vc) of the hybrid restriction, column by column.
#include <cstdio>
#include <string>
#include <vector>
#include "internal.h"
using namespace cgs;
int main(int argc, char** argv) {
    if (argc < 3) return 2;
    FILE* in = fopen(argv[1], "r");
    if (!in) return 2;
    long nv = 0, ne = 0;
    int b[3];
    if (fscanf(in, "%ld %ld %d %d %d", &nv, &ne, &b[0], &b[1], &b[2]) != 5) return 2;
    std::vector<double> xyz(3 * (size_t)nv);
    std::vector<int32_t> conn(8 * (size_t)ne), part(ne);
    for (auto& v : xyz)
        if (fscanf(in, "%lf", &v) != 1) return 2;
    for (auto& v : conn)
        if (fscanf(in, "%d", &v) != 1) return 2;
    for (auto& v : part)
        if (fscanf(in, "%d", &v) != 1) return 2;
    fclose(in);
    cgs_params prm{};
    for (int d = 0; d < 3; ++d) prm.box[d] = b[d];
    prm.overlap_layers = 1;
    prm.prec = CGS_FP64;
    prm.form = CGS_HYBRID;
    prm.coarse_solver = CGS_COARSE_DENSE;
    HostSetup S;
    std::string err;
    if (host_setup(xyz.data(), nv, conn.data(), ne, nullptr, part.data(), prm, S, err) != CGS_OK) {
        printf("%s\n", err.c_str());
        return 1;
    }
    FILE* f = fopen(argv[2], "w");
    fprintf(f, "%ld %ld %ld\n", (long)S.nr, (long)S.jt_vert.size(), (long)(S.hr_rng.size() / 4));
    for (size_t q = 0; q < S.jt_vert.size(); ++q) {
        fprintf(f, "%d", S.jt_vert[q]);
        for (int32_t e = S.jt_ptr[q]; e < S.jt_ptr[q + 1]; ++e)
            if (S.jt_val[e] != 0.0) fprintf(f, " %d %.17g", S.jt_col[e], S.jt_val[e]);
        fprintf(f, "\n");
    }
    for (size_t g = 0; g + 3 < S.hr_rng.size(); g += 4)
        for (int32_t i = S.hr_rng[g]; i < S.hr_rng[g + 1]; ++i)
            fprintf(f, "%d %d %.17g %.17g\n", S.hr_vert[i], S.hr_rng[g + 2], S.hr_j[i], S.hr_g[i]);
    fclose(f);
    return 0;
}
