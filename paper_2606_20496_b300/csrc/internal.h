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
    std::vector<float> a28;            // SoA [kOff][ne] off-diagonals rounded to float32
    std::vector<float> a28lo;          // SoA [kOff][ne] float32 remainders a - (double)a28
    std::vector<uint8_t> dir;          // nv, 1 = Dirichlet
    std::vector<double> invcnt;        // nv, 1 / (elements at the vertex)
    std::vector<double> wov;           // nv, 1 / (subdomains holding the vertex), 0 if none
    // subdomains, in caller order
    std::vector<int64_t> sub_ptr;      // n_sub+1
    std::vector<int32_t> sub_idx;      // sum_m, ascending vertex ids per subdomain
    std::vector<int64_t> inv_ptr;      // n_sub+1, offsets (entries) of packed inverses
    std::vector<double> inv;           // packed lower triangle, row-major, float64
    // box coarse space
    int b[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, H[3] = {1, 1, 1};
    std::vector<int32_t> cell;         // ne (device order), lexicographic cell id
    std::vector<int32_t> tile_ptr;     // ntiles+1, element ranges (device order)
    std::vector<int32_t> tile_vptr;    // ntiles+1, ranges in tile_verts
    std::vector<uint32_t> tile_verts;  // distinct free vertices of each tile, | kSharedBit if shared
    std::vector<uint16_t> eloc;        // ne*8, tile-local vertex index, 0xFFFF = Dirichlet
    std::vector<float> at_hi, at_lo;   // [ntiles][kOff][kTileElems] tile-major off-diagonals (float, remainder)
    std::vector<int32_t> cell_cols;    // ncell*8, active column of each cell corner or -1
    std::vector<int64_t> box_active;   // nr, lexicographic box-vertex ids
    std::vector<double> ar_inv;        // nr*nr, A_r^{-1}, full symmetric, float64
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
    const int32_t* conn = nullptr;     // ne*8 (int4 x2 per element)
    const uint8_t* dir = nullptr;      // nv, 1 = Dirichlet
    const double* a36 = nullptr;       // [36][ne]
    const double2* xyzw = nullptr;     // 2*nv: (x, y), (z, 1/count) per vertex, float64
    const float4* xyzwf = nullptr;     // nv: same, float32
    const int32_t* cell = nullptr;     // ne
    int64_t ntiles = 0;
    const int32_t* tile_ptr = nullptr;
    const int32_t* tile_vptr = nullptr;
    const uint32_t* tile_verts = nullptr;
    const uint16_t* eloc = nullptr;
    const float* at_hi = nullptr;      // [ntiles][28][256] off-diagonals rounded to float, tile-major
    const float* at_lo = nullptr;      // same layout, float remainders (outer operator only)
    const int32_t* cell_cols = nullptr;// ncell*8
    // subdomains grouped by size class for the warp kernels
    const int32_t* sub_ptr = nullptr;  // n_sub+1 (int32 offsets into sub_idx)
    const int32_t* sub_idx = nullptr;
    const int64_t* inv_ptr = nullptr;  // n_sub+1
    const double* inv64 = nullptr;
    const float* inv32 = nullptr;
    const __half* inv16 = nullptr;
    const float* inv16_scale = nullptr;// n_sub
    const double* wov64 = nullptr;     // nv
    const float* wov32 = nullptr;      // nv
    const double* ar_inv = nullptr;    // nr*nr
    int max_m = 0;
};

// Mesh descriptors and work tables of one set of solve slots (launchers).
struct Work;
struct Plan {
    const DevMesh* meshes = nullptr;       // device array of mesh descriptors
    const Work* work[5] = {};              // device work tables, one per WorkKind
    unsigned int nwork[5] = {};
    int nslots = 0;
    int max_m = 0;                         // largest subdomain over the meshes
    bool any_nr = false;                   // some mesh has a reduced space
    int wait_limit = 1 << 20;              // iteration limit of bounded device waits
};

// Device scalars of one PCG solve (kernels.cu).
struct SolveScalars {
    double bnorm2;     // ||b||^2
    double tol2;       // (rtol ||b||)^2
    double rho;        // r.z of the current iterate
    double pq;         // p.A p
    double alpha, beta;
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

enum WorkKind { kWorkElem = 0, kWorkTile, kWorkVert, kWorkSub, kWorkRow, kWorkKinds };
constexpr int kElemChunk = 256;   // elements per block
constexpr int kRowChunk = 8;      // reduced rows per block (one warp each)

// Vector pools of a set of slots, passed by value to every kernel.  A slot's
// vector is pool + work.voff (vertex vectors) or pool + work.roff (reduced).
struct Vecs {
    double *x = nullptr, *r = nullptr, *p = nullptr, *y = nullptr, *q = nullptr;
    float2 *p2 = nullptr, *q2 = nullptr;   // float-pair p and A p (mixed forms)
    void *z = nullptr, *s = nullptr;       // bulk precision (double or float)
    double *rr = nullptr, *ur = nullptr;
    float* ur32 = nullptr;
    double* partials = nullptr;
    SolveScalars* S = nullptr;             // nullptr: no early exit (single steps)
    const double* b = nullptr;             // right-hand sides (pool), or
    const double* const* bptr = nullptr;   // per-slot right-hand side pointers
    double* const* xptr = nullptr;         // per-slot solution pointers (copy-out)
};

}  // namespace cgs
