// Host-side check of the assembled rows (no GPU): reads a mesh written by the
// test (nv ne b0 b1 b2 has_dirichlet, then xyz, conn, part and, if given, the
// Dirichlet mask), runs the library's host set-up in the FP64 and the
// FP32-bulk forms and writes, per form, the sliced-ELL width and, per vertex
// row, its (column, value) entries: float64 values, or the float pair's hi
// and lo.
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
    int b[3], has_dir = 0;
    if (fscanf(in, "%ld %ld %d %d %d %d", &nv, &ne, &b[0], &b[1], &b[2], &has_dir) != 6) return 2;
    std::vector<double> xyz(3 * (size_t)nv);
    std::vector<int32_t> conn(8 * (size_t)ne), part(ne);
    std::vector<uint8_t> dir(has_dir ? nv : 0);
    for (auto& v : xyz)
        if (fscanf(in, "%lf", &v) != 1) return 2;
    for (auto& v : conn)
        if (fscanf(in, "%d", &v) != 1) return 2;
    for (auto& v : part)
        if (fscanf(in, "%d", &v) != 1) return 2;
    for (auto& v : dir) {
        int t = 0;
        if (fscanf(in, "%d", &t) != 1) return 2;
        v = (uint8_t)t;
    }
    fclose(in);
    FILE* f = fopen(argv[2], "w");
    for (cgs_precision prec : {CGS_FP64, CGS_FP32_BULK}) {
        cgs_params prm{};
        for (int d = 0; d < 3; ++d) prm.box[d] = b[d];
        prm.overlap_layers = 1;
        prm.prec = prec;
        prm.form = CGS_HYBRID;
        prm.coarse_solver = CGS_COARSE_DENSE;
        HostSetup S;
        std::string err;
        if (host_setup(xyz.data(), nv, conn.data(), ne, has_dir ? dir.data() : nullptr, part.data(), prm, S,
                       err) != CGS_OK) {
            printf("%s\n", err.c_str());
            return 1;
        }
        const bool pairs = prec != CGS_FP64;
        fprintf(f, "%d %ld\n", S.ell_w, (long)(S.ell_ptr.empty() ? 0 : S.ell_ptr.size() - 1));
        if (S.ell_ptr.empty()) continue;
        for (long v = 0; v < nv; ++v) {
            const long sl = v / 32, lane = v % 32;
            for (int k = 0; k < S.ell_w; ++k) {
                const int64_t o = S.ell_ptr[sl] + 32 * (int64_t)k + lane;
                if (S.ell_col[o] < 0) continue;
                if (pairs)
                    fprintf(f, "%d %.9g %.9g ", S.ell_col[o], (double)S.ell_pair[2 * o], (double)S.ell_pair[2 * o + 1]);
                else
                    fprintf(f, "%d %.17g ", S.ell_col[o], S.ell_val[o]);
            }
            fprintf(f, "\n");
        }
    }
    fclose(f);
    return 0;
}
