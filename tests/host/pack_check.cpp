// Host-side check of the lane packs (no GPU): reads a mesh written by the
// test (nv ne, then xyz, conn and part per line), runs the library's host
// set-up in the FP32-bulk form and writes, for the test to compare with the
// oracle: the number of subdomains left to the warp kernels, then per lane
// pack its size class M and, per lane, the M vertex ids (-1 = padding) and
// the M (M + 1) / 2 entries of the packed upper triangle of A_p^{-1}.
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
    prm.prec = CGS_FP32_BULK;
    prm.form = CGS_HYBRID;
    prm.coarse_solver = CGS_COARSE_DENSE;
    HostSetup S;
    std::string err;
    if (host_setup(xyz.data(), nv, conn.data(), ne, nullptr, part.data(), prm, S, err) != CGS_OK) {
        printf("%s\n", err.c_str());
        return 1;
    }
    FILE* f = fopen(argv[2], "w");
    fprintf(f, "%ld %ld\n", (long)S.n_wsub, (long)S.pack_m.size());
    for (size_t P = 0; P < S.pack_m.size(); ++P) {
        const int c = S.pack_m[P];
        const int64_t io = S.pack_idx_off[P], ao = S.pack_inv_off[P], T = lane_entries(c);
        fprintf(f, "%d\n", c);
        for (int l = 0; l < 32; ++l) {
            for (int k = 0; k < c; ++k) fprintf(f, "%d ", S.pack_idx[io + (int64_t)k * 32 + l]);
            fprintf(f, "\n");
            for (int e = 0; e < c * (c + 1) / 2; ++e) fprintf(f, "%.17g ", S.pack_inv[ao + l * T + e]);
            fprintf(f, "\n");
        }
    }
    fclose(f);
    return 0;
}
