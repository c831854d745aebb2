// Internal declarations shared by the host setup, the CUDA kernels and the
// C ABI.  Not installed; the public interface is include/cgs.h.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/cgs.h"

namespace cgs {

// Number of stored entries of a symmetric 8x8 element matrix.
constexpr int kUpper = 36;   // upper triangle including the diagonal, (i <= j)
constexpr int kOff = 28;     // strict upper triangle (i < j); diagonal = -row sum
constexpr int kPackAlign = 8;  // packed inverses start on multiples of 8 entries
// Element tiles for block-local assembly: consecutive device-order elements
// with at most kTileElems elements and kTileVerts distinct free vertices.
constexpr int kTileElems = 256;
constexpr int kTileVerts = 1024;
constexpr uint32_t kSharedBit = 0x80000000u;  // tile vertex also touched by another tile

// Everything the host setup produces, in the layout the device uses.
struct HostSetup {
    int64_t nv = 0, ne = 0, n_free = 0, n_sub = 0, nr = 0;
    int64_t max_m = 0, sum_m = 0;
    // elements in device order (sorted by centroid cell, then subdomain, then id)
    std::vector<int32_t> elem_order;   // device slot -> caller element id
    std::vector<int32_t> conn;         // ne*8, vertex id, or ~v for a Dirichlet vertex
    std::vector<double> a36;           // SoA [kUpper][ne] element matrices, float64
    // the assembled free block of A (float64 form), sliced ELL: rows in
    // slices of 32, every slice ell_w entries wide, entry k of row 32 s + lane
    // at ell_ptr[s] + 32 k + lane = 32 ell_w s + 32 k + lane (column -1 and
    // value 0 pad the shorter rows; Dirichlet rows are all padding)
    int32_t ell_w = 0;
    std::vector<int64_t> ell_ptr;      // nslice+1 (empty: element form only)
    std::vector<int32_t> ell_col;
    std::vector<double> ell_val;       // float64 form
    std::vector<float> ell_pair;       // mixed forms: (hi, lo) per entry
    std::vector<float> a28;            // SoA [kOff][ne] off-diagonals rounded to float32
    std::vector<float> a28lo;          // SoA [kOff][ne] float32 remainders a - (double)a28
    std::vector<uint8_t> dir;          // nv, 1 = Dirichlet
    std::vector<double> invcnt;        // nv, 1 / (elements at the vertex)
    std::vector<double> wov;           // nv, 1 / (subdomains holding the vertex), 0 if none
    std::vector<double> ras_w;         // sum_m, RAS prolongation weight of each entry of sub_idx
    // subdomains, in caller order
    std::vector<int64_t> sub_ptr;      // n_sub+1
    std::vector<int32_t> sub_idx;      // sum_m, ascending vertex ids per subdomain
    // subdomains solved by the warp kernels (all of them in the FP64 form on
    // small meshes, else those with more than kLaneMaxM dofs in the FP64 form
    // and more than kLaneMaxMixed in the mixed forms), caller order
    int64_t n_wsub = 0, max_wm = 0;
    std::vector<int64_t> wsub_ptr;     // n_wsub+1
    std::vector<int32_t> wsub_idx;
    std::vector<int64_t> inv_ptr;      // n_wsub+1, offsets (entries) of the inverses
    std::vector<double> inv;           // cyclic diagonals (i, (i+d) mod m) at d*m + i, float64
    std::vector<double> wsub_ras;      // RAS weights aligned with wsub_idx
    std::vector<double> ap;            // A_p in the same layout (inexact local solves only)
    // lane packs (mixed forms; FP64 form on large meshes): 32 subdomains of
    // one size class, one per lane
    std::vector<int32_t> pack_m;       // n_pack, class size
    std::vector<int64_t> pack_idx_off; // n_pack+1, offsets into pack_idx (32*M per pack)
    std::vector<int64_t> pack_inv_off; // n_pack+1, offsets into pack_inv (32*lane_entries(M) per pack)
    std::vector<int32_t> pack_idx;     // [pack][k][lane] vertex id, -1 = padding
    std::vector<double> pack_inv;      // [pack][lane][lane_entries(M)] upper triangle, row-major, float64
    std::vector<double> pack_ras;      // RAS weights aligned with pack_idx
    // row packs (small meshes): the same subdomains, 8 per pack, full rows
    std::vector<int32_t> rpack_m;
    std::vector<int64_t> rpack_idx_off, rpack_inv_off;
    std::vector<int32_t> rpack_idx;    // [pack][k][lane] vertex id of row k of lane's subdomain, -1 = padding
    std::vector<double> rpack_inv;     // [pack][lane][row_entries(M)] rows g, g+4, ... of the inverse
    std::vector<double> rpack_ras;     // RAS weights aligned with rpack_idx
    // box coarse space
    int b[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, H[3] = {1, 1, 1};
    std::vector<int32_t> cell;         // ne (device order), lexicographic cell id
    std::vector<int32_t> tile_ptr;     // ntiles+1, element ranges (device order)
    std::vector<int32_t> tile_vptr;    // ntiles+1, ranges in tile_verts
    std::vector<uint32_t> tile_verts;  // distinct free vertices of each tile, | kSharedBit if shared
    std::vector<uint16_t> eloc;        // ne*8, tile-local vertex index, 0xFFFF = Dirichlet
    std::vector<float> at_hi, at_lo;   // [ntiles][kOff/4][kTileElems][4] tile-major off-diagonals (float, remainder)
    std::vector<int32_t> cell_cols;    // ncell*8, active column of each cell corner or -1
    // per-vertex box lists (restriction and interpolation by vertex)
    std::vector<int32_t> vb_vert;      // free vertices with elements, in vertex order
    std::vector<int32_t> vb_ptr;       // +1, ranges in vb_cell / vb_w
    std::vector<int32_t> vb_cell;      // cells of the vertex's elements, ascending (packed coordinates)
    std::vector<double> vb_w;          // elements of the vertex in that cell / elements of the vertex
    std::vector<int32_t> re_vert, re_cell;   // the same entries sorted by cell (restriction)
    std::vector<double> re_w;
    std::vector<int32_t> re_rng;       // (begin, end) entry ranges within one cell, <= kBoxRange each
    // J~ = W Q^T J_L as explicit rows (the same interpolant as the box
    // lists, the weights formed once in float64), padded to multiples of 4
    // entries and ordered by padded length, then vertex
    std::vector<int32_t> jt_vert;      // nvb, the vertex of each row
    std::vector<int32_t> jt_ptr;       // nvb+1
    std::vector<int32_t> jt_col;       // reduced columns, ascending per row (padding: column 0)
    std::vector<double> jt_val;        // weights (padding: 0)
    int64_t jt_nnz = 0;                // entries without the padding
    // restriction of the hybrid step, r_r = J~^T r - (A J~)^T l, as explicit
    // entries sorted by reduced column, then vertex (hybrid set-ups only)
    std::vector<int32_t> hr_vert;
    std::vector<double> hr_j, hr_g;    // J~_vc and (A J~)_vc
    std::vector<int32_t> hr_rng;       // 4 per range: begin, end, column, 0 (<= kHybRange entries)
    std::vector<int64_t> box_active;   // nr, lexicographic box-vertex ids
    int coarse = 1;                    // reduced solver: 1 dense A_r^{-1}, 2 XX^T
    int64_t ar_nnz = 0;                // nonzeros of A_r
    std::vector<double> ar_inv;        // nr*nr, A_r^{-1}, full symmetric, float64 (dense)
    // XX^T (Sec. 2): A_r^{-1} = X X^T, column k of X the k-th A_r-conjugate
    // vector in nested-dissection order; rows are reduced indices
    std::vector<int32_t> nd_perm;      // nr, nested-dissection position -> reduced index
    std::vector<int32_t> xc_ptr;       // nr + 1, column starts (pass t = X^T r_r)
    std::vector<uint16_t> xc_idx;      // rows of each column, ascending
    std::vector<double> xc_val;
    std::vector<int32_t> xr_ptr;       // nr + 1, row starts (pass u_r = X t)
    std::vector<uint16_t> xr_idx;      // columns of each row, ascending
    std::vector<double> xr_val;
    std::vector<int32_t> xs_seg;       // 4 per segment: column, begin, end, 0 (<= kXxtSeg entries)
    double seconds = 0.0;
};

// Host setup (setup.cpp).  Returns CGS_OK or an error with a message in err.
cgs_status host_setup(const double* xyz, int64_t nv, const int32_t* conn, int64_t ne,
                      const uint8_t* dirichlet, const int32_t* elem_part,
                      const cgs_params& prm, HostSetup& out, std::string& err);

// Device-resident mesh data (api.cu allocates, kernels.cu reads).
struct DevMesh {
    int64_t nv = 0, ne = 0, n_sub = 0, nr = 0;
    int b[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, H[3] = {1, 1, 1}, iH[3] = {1, 1, 1};
    float Hf[3] = {1, 1, 1}, iHf[3] = {1, 1, 1};   // the same, rounded to float
    const int32_t* conn = nullptr;     // ne*8 (int4 x2 per element)
    const uint8_t* dir = nullptr;      // nv, 1 = Dirichlet
    const double* a36 = nullptr;       // [36][ne]
    int max_pack_m = 0;                // largest lane- or row-pack class
    int64_t nslice = 0;                // sliced-ELL rows of the assembled A (0: none)
    int32_t ell_w = 0;                 // entries per row (every slice as wide)
    const int64_t* ell_ptr = nullptr;
    const int32_t* ell_col = nullptr;
    const double* ell_val = nullptr;   // float64 form
    const float2* ell_pair = nullptr;  // mixed forms
    const double2* xyzw = nullptr;     // 2*nv: (x, y), (z, 1/count) per vertex, float64
    const float4* xyzwf = nullptr;     // nv: same, float32
    const int32_t* cell = nullptr;     // ne
    int64_t ntiles = 0;
    const int32_t* tile_ptr = nullptr;
    const int32_t* tile_vptr = nullptr;
    const uint32_t* tile_verts = nullptr;
    const uint16_t* eloc = nullptr;
    const float* at_hi = nullptr;      // [ntiles][7][256][4] off-diagonals rounded to float, tile-major
    const float* at_lo = nullptr;      // same layout, float remainders (outer operator only)
    const int32_t* cell_cols = nullptr;// ncell*8
    // per-vertex box lists: vertex, its (cell, weight) entries
    int64_t nvb = 0;
    const int32_t* vb_vert = nullptr;  // nvb
    const int32_t* vb_ptr = nullptr;   // nvb+1
    const int32_t* vb_cell = nullptr;  // packed cell coordinates ci | cj << 10 | ck << 20
    const double* vb_w64 = nullptr;    // FP64 form
    const float* vb_w32 = nullptr;     // mixed forms
    // the same (vertex, cell, weight) entries sorted by cell
    int64_t nre = 0;
    const int32_t* re_vert = nullptr;
    const int32_t* re_cell = nullptr;  // packed, as vb_cell
    const double* re_w64 = nullptr;
    const float* re_w32 = nullptr;
    int64_t nrng = 0;
    const int2* re_rng = nullptr;      // nrng (begin, end) ranges of one cell's entries
    // subdomains of the warp kernels (n_sub of them: all in the FP64 form on
    // small meshes, else those above the lane packs' size limit)
    const int32_t* sub_ptr = nullptr;  // n_sub+1 (int32 offsets into sub_idx)
    const int32_t* sub_idx = nullptr;
    const int64_t* inv_ptr = nullptr;  // n_sub+1
    const double* inv64 = nullptr;
    const float* inv32 = nullptr;
    const __half* inv16 = nullptr;
    const float* inv16_scale = nullptr;// n_sub
    // RAS prolongation weight of each entry of sub_idx (Sec. 3, R~_p)
    const double* went64 = nullptr;
    const float* went32 = nullptr;
    // inexact local solves (cg_steps > 0): A_p in the layout of the inverses
    int32_t cg_steps = 0;
    const double* ap64 = nullptr;
    const float* ap32 = nullptr;
    // lane packs (mixed forms): 32 subdomains of one size class M per pack,
    // lane l of the pack solves one; idx [k][32], entries float4 groups
    // [e/4][32][4] (float) or 8-entry groups [e/8][32][8] (half, per-lane scale)
    int64_t n_pack = 0;
    const int32_t* pack_m = nullptr;       // n_pack
    const int64_t* pack_idx_off = nullptr; // n_pack
    const int64_t* pack_inv_off = nullptr; // n_pack (entries)
    const int32_t* pack_idx = nullptr;
    const double* pack_inv64 = nullptr;    // FP64 form: groups [e/2][32][2]
    const double* pack_went64 = nullptr;   // RAS weights [k][32], aligned with pack_idx
    const float* pack_went32 = nullptr;
    const float* pack_inv32 = nullptr;
    const __half* pack_inv16 = nullptr;
    const float* pack_scale = nullptr;     // n_pack*32 (half entries)
    // row packs (small meshes): 8 subdomains per pack, 4 lanes each holding
    // rows g, g + 4, ... in full; same group layouts and per-lane scales
    int64_t n_rpack = 0;
    const int32_t* rpack_m = nullptr;
    const int64_t* rpack_idx_off = nullptr;
    const int64_t* rpack_inv_off = nullptr;
    const int32_t* rpack_idx = nullptr;
    const float* rpack_inv32 = nullptr;
    const __half* rpack_inv16 = nullptr;
    const float* rpack_scale = nullptr;
    const float* rpack_went32 = nullptr;   // RAS weights, aligned with rpack_idx
    const double* wov64 = nullptr;     // nv
    const float* wov32 = nullptr;      // nv
    // explicit rows of J~ (FP64 form): row vertices, offsets (multiples of 4)
    const int32_t* jt_vert = nullptr;  // nvb
    const int32_t* jt_ptr = nullptr;   // nvb + 1
    const int32_t* jt_col = nullptr;
    const double* jt_val = nullptr;
    // restriction of the hybrid step r_r = J~^T r - (A J~)^T l (hybrid set-ups)
    int64_t nhr = 0;                   // ranges
    const int4* hr_rng = nullptr;      // (begin, end, column, 0), <= kHybRange entries of one column
    const int32_t* hr_vert = nullptr;
    const double2* hr_jg64 = nullptr;  // (J~_vc, (A J~)_vc), FP64 form
    const float2* hr_jg32 = nullptr;   // the same rounded to float, mixed forms
    int32_t xxt = 0;                   // 1: reduced solve by XX^T (the fields below), else dense
    int64_t nxseg = 0;                 // pass-1 segments
    const int4* xs_seg = nullptr;      // (column, begin, end, 0) of each segment of X's columns
    const uint16_t* xc_idx = nullptr;  // column-major rows of X
    const void* xc_val = nullptr;      // column-major values: double (FP64 form) or float pair
    const int32_t* xr_ptr = nullptr;   // nr + 1 row starts of X
    const uint16_t* xr_idx = nullptr;  // row-major columns of X
    const void* xr_val = nullptr;      // row-major values: double or float pair
    const double* ar_inv = nullptr;    // nr*nr (FP64 form)
    const float2* ar_inv2 = nullptr;   // nr rows of nr2 float pairs (mixed forms; nr2 = nr rounded up to even)
    int64_t nr2 = 0;
    int max_m = 0;
};

// Work tables: element ranges, element tiles, vertex ranges, warp-kernel
// subdomain ranges, reduced-row ranges, lane-pack ranges, ranges of the
// per-vertex box lists (interpolation) and of their cell-sorted entries
// (restriction), row-pack ranges.
enum WorkKind {
    kWorkElem = 0,
    kWorkTile,
    kWorkVert,
    kWorkSub,
    kWorkRow,
    kWorkPack,
    kWorkBox,
    kWorkBoxEnt,
    kWorkRowPack,
    kWorkXSeg,
    kWorkHybR,
    kWorkEll,
    kWorkKinds
};

// Mesh descriptors and work tables of one set of solve slots (launchers).
struct Work;
struct Plan {
    const DevMesh* meshes = nullptr;       // device array of mesh descriptors
    const Work* work[kWorkKinds] = {};     // device work tables, one per WorkKind
    unsigned int nwork[kWorkKinds] = {};
    int nslots = 0;
    int max_m = 0;                         // largest warp-kernel subdomain over the meshes
    bool any_nr = false;                   // some mesh has a reduced space
    int wait_limit = 1 << 20;              // iteration limit of the element-tile (TMA) waits
    int bar_limit = 1 << 22;               // iteration limit of the persistent loop's grid-barrier waits
    bool tile_tma = false;                 // element tiles staged by TMA (else streamed by the threads)
    int pack_chunk = 8;                    // lane packs per kWorkPack item (the schedule's)
    bool pdl = true;                       // launch with programmatic stream serialization
    bool interp_cells = false;             // interpolation by cell-sorted entries (dots left to the caller)
    bool any_xxt = false;                  // some mesh solves its reduced system by XX^T
    bool hyb_restrict = false;             // every mesh with a reduced space has the hybrid
                                           // restriction entries (no s = r - A l needed)
    bool lane_big = false;                 // some mesh has lane or row packs of more than 32 dofs
    bool ell = false;                      // every mesh has the assembled A in float64:
                                           // the FP64 applies run by rows
    bool ell_pair = false;                 // every mesh has it in float pairs: the PCG's
                                           // outer apply runs by rows (unless tile_tma)
};

// Grid-wide barrier of the persistent PCG kernel (device memory, zeroed
// before each launch): arrival count, generation, error flag.
struct GridBar {
    unsigned int count;
    unsigned int gen;
    int error;
    int pad;
};

// Device scalars of one PCG solve (kernels.cu).
struct SolveScalars {
    double bnorm2;     // ||b||^2
    double tol2;       // (rtol ||b||)^2
    double rho;        // r.z of the current iterate
    double pq;         // p.A p
    double alpha, beta;
    float2 alpha2, beta2;  // alpha and beta as float pairs (mixed forms)
    double rr;         // ||r||^2 after the update
    double zr, zq;     // z.r and z.q for the next direction
    int iters;
    int maxit;
    int loops;         // executions of the device-side loop body
    int done;          // 1 = stop (converged, failed or maxit)
    int status;        // cgs_status of the solve
    unsigned int ticket[4];  // block-completion counters of the fused reductions
    int timeouts;            // bounded device-side waits that expired
    double res2, b2;         // ||b - A x||^2 and ||b||^2 over free entries (final check)
};

// One block's share of work: a range of elements, tiles, vertices,
// subdomains or reduced rows of one solve slot (one mesh and one right-hand
// side).  A slot's vectors live in pooled arrays at the given offsets; its
// blocks of one kind are numbered idx = 0..count-1 for the per-slot
// reductions.
struct Work {
    int32_t mesh;          // index into the mesh descriptor array
    int32_t slot;          // index into the SolveScalars array
    int64_t voff;          // offset of the slot's vertex vectors (nv entries)
    int32_t roff;          // offset of the slot's reduced-space vectors (n_r entries)
    int32_t poff;          // offset of the slot's partial sums (2 * count entries)
    int32_t begin, end;    // the range
    int32_t idx, count;    // this block among the slot's blocks of this kind
};

// Lane packs of the mixed-form local solves: subdomains with at most
// kLaneMaxM dofs, padded to the next size class, 32 of one class per pack.
constexpr int kLaneMaxM = 32;        // FP64 form (a lane keeps 2M doubles in registers)
constexpr int kLaneMaxMixed = 64;    // mixed forms: classes above 32 run in kernels of their own
constexpr int kLaneClasses[] = {8, 12, 16, 18, 20, 24, 27, 32, 40, 48, 56, 64};
inline int lane_class(int m) {
    for (int c : kLaneClasses)
        if (m <= c) return c;
    return 0;
}
// entries stored per lane: the upper triangle, padded to a multiple of 8
constexpr int lane_entries(int M) { return (M * (M + 1) / 2 + 7) / 8 * 8; }
// Row packs (small meshes): 8 subdomains per warp, 4 lanes each; lane g of
// a subdomain holds the full rows g, g + 4, ... (ceil(M / 4) rows of M).
constexpr int kRowLanes = 4;
constexpr int row_pack_rows(int M) { return (M + kRowLanes - 1) / kRowLanes; }
constexpr int row_entries(int M) { return (row_pack_rows(M) * M + 7) / 8 * 8; }
// meshes with fewer lane subdomains than this also get row packs
constexpr int64_t kRowPackMaxSubs = 9472;
constexpr int kElemChunk = 256;   // elements per block
constexpr int kEllChunk = 1024;   // rows of the assembled A per block (four per thread)
// Box cells per axis, at most kMaxBoxes; the box lists store a cell as its
// packed coordinates ci | cj << 10 | ck << 20.
constexpr int kMaxBoxes = 1023;
inline int32_t pack_cell(int32_t c, int bx, int by) {
    return (c % bx) | (((c / bx) % by) << 10) | ((c / (bx * by)) << 20);
}
constexpr int kRowChunk = 4;      // reduced rows per block (one warp each)
constexpr int kXxtSeg = 256;      // entries of one column of X per pass-1 warp
constexpr int kBoxRange = 256;    // restriction entries (of one cell) per warp
// hybrid-restriction entries (of one reduced column) per warp: long ranges,
// so the warp's closing sum (five float64 additions on all 32 lanes) is
// small against its two FMAs per entry
constexpr int kHybRange = 1024;

// Vector pools of a set of slots, passed by value to every kernel.  A slot's
// vector is pool + work.voff (vertex vectors) or pool + work.roff (reduced).
// In the mixed forms the outer iterates
// x, r and p are float pairs stored in the 8-byte entries of x, r and p
// (p2 aliases p); x is turned back into float64 in place before the final
// residual.
struct Vecs {
    double *x = nullptr, *r = nullptr, *p = nullptr, *y = nullptr, *q = nullptr;
    float2 *p2 = nullptr, *q2 = nullptr;   // float-pair p and A p (mixed forms)
    void *z = nullptr, *s = nullptr;       // bulk precision (double or float)
    double *rr = nullptr, *ur = nullptr;
    double* rt = nullptr;                  // t = X^T r_r of the XX^T solve (float pair or double), n_r per slot
    float* ur32 = nullptr;
    double* partials = nullptr;
    SolveScalars* S = nullptr;             // nullptr: no early exit and no wait status (timing runs)
    int step = 0;                          // 1: a single-step call; S then only carries the status of
                                           // bounded waits (no PCG scalar is read or written)
    const double* b = nullptr;             // right-hand sides (pool), or
    const double* const* bptr = nullptr;   // per-slot right-hand side pointers
    double* const* xptr = nullptr;         // per-slot solution pointers (copy-out)
};

}  // namespace cgs
