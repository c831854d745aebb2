// Launchers of the CUDA kernels (kernels.cu), called by the C ABI (api.cu,
// noalloc.cu).  Every launcher runs over the work tables of a Plan; vectors
// are pools addressed per slot through the work items' offsets.
#pragma once

#include <string>
#include <vector>

#include "internal.h"

namespace cgs {

// Projection onto prior solutions (projection.cu), float64 vectors of length
// n; X and Y hold k rows of n.  launch_proj_dots: out[j] = X_j . v (j < k),
// out[k] = v . v, Dirichlet entries of v (dir != 0) taken as zero; `partial`
// holds proj_partial_entries(k) doubles.  Two kernels.
int proj_partial_entries(int max_k);
void launch_proj_dots(const double* X, int k, int64_t n, const double* v, const uint8_t* dir, double* partial,
                      double* out, cudaStream_t st);
// out = base (Dirichlet entries zeroed; nullptr = 0) + s sum_{j<k} coef[j] Y_j
void launch_proj_combine(int64_t n, const double* base, const uint8_t* dir, double s, const double* coef, int k,
                         const double* Y, double* out, cudaStream_t st);
// w -= sum_{j<k} coef[j] X_j (coef on the device), Dirichlet entries of w
// zero; then, with dots, out[j] = X_j . w (j < k) and out[k] = w . w of the
// updated w (false, nothing launched, for k > 32), without dots out[0] =
// w . w.  `partial` holds proj_partial_entries(k) doubles.  Two kernels.
bool launch_gs_update(const double* X, int k, int64_t n, const double* coef, const uint8_t* dir, double* w,
                      double* partial, double* out, bool dots, cudaStream_t st);
void launch_vec_scale(int64_t n, double* a, double alpha, cudaStream_t st);
void launch_vec_add(int64_t n, const double* a, const double* b, double* out, cudaStream_t st);

void launch_apply64(const Plan& P, const Vecs& V, const double* x, double* y, double alpha, bool dot,
                    cudaStream_t st);
void launch_apply_pair_tiled(const Plan& P, const Vecs& V, cudaStream_t st);
// the PCG's outer apply of the mixed forms: by rows of the assembled A when
// every mesh has them and the schedule does not ask for TMA-staged tiles
bool rows_outer(const Plan& P);
void launch_apply_outer(const Plan& P, const Vecs& V, cudaStream_t st);
void launch_apply28f_tiled(const Plan& P, const Vecs& V, const float* x, float* y, float alpha, cudaStream_t st);
// out += sum_p R~_p^T A_p^{-1} R_p r, weighted: 0 none (additive), 1 W_ov per
// vertex (hybrid), 2 the RAS weight per entry
void launch_local(const Plan& P, const Vecs& V, cgs_precision prec, const void* r, void* out, int weighted,
                  cudaStream_t st);
// Additive form, mixed precision: z += local solves of s and r_r += J^T W s
// (float pairs) in one launch; false (nothing launched) unless every
// subdomain is in packs and there is a reduced space.
bool launch_local_restrict(const Plan& P, const Vecs& V, cgs_precision prec, const float* s, float* z, void* rr,
                           cudaStream_t st);
// Hybrid step without s = r - A l: r_r += J~^T r - (A J~)^T l over the
// mesh's explicit entries (float64, or float with a float-pair r_r in the
// mixed forms); r and l in the bulk precision.  Needs P.hyb_restrict.
void launch_restrict_hybrid(const Plan& P, const Vecs& V, bool fp64, const void* r, const void* l, void* rr,
                            cudaStream_t st);
// r_r += J^T W s.  pair_out: rr holds float pairs (mixed forms, float s)
void launch_restrict(const Plan& P, const Vecs& V, bool fp64, const void* s, bool s_is_double, void* rr,
                     bool pair_out, cudaStream_t st);
// z += W Q^T J_L u_r.  dots: also z.r and z.q with beta and rho (fused PCG
// dots; r and q of the engine's slots; mixed forms then zero q).  cond:
// block 0 also sets the device-side loop condition.  With P.interp_cells the
// interpolation runs over the cell-sorted entries and fuses nothing.
// Returns whether the dots (and the loop condition) were fused.
bool launch_interp_add(const Plan& P, const Vecs& V, bool fp64, const double* ur, const float* ur32, void* z,
                       bool dots, const cudaGraphConditionalHandle* cond, cudaStream_t st);
void launch_coarse(const Plan& P, const Vecs& V, const double* rr, double* ur, float* ur32, cudaStream_t st);
// First pass of the XX^T reduced solve for the plan's XX^T meshes: V.rt =
// X^T r_r (zero on entry; float pairs when `pair`).  Returns whether it
// launched (no XX^T mesh: nothing to do).  launch_coarse / launch_coarse_pair
// then finish every mesh: the dense product, or u_r = X V.rt.
bool launch_xxt_pass1(const Plan& P, const Vecs& V, bool pair, const double* rr, cudaStream_t st);
void launch_coarse_pair(const Plan& P, const Vecs& V, const float2* rr2, double* ur, float* ur32, cudaStream_t st);
void launch_split_pair(int64_t n, const double* a, float2* b, cudaStream_t st);
void launch_pair_to_double(int64_t n, const float2* a, double* b, cudaStream_t st);

// Outer iteration of the mixed forms (float-pair x, r, p, q).
void launch_pcg_init_pair(const Plan& P, const Vecs& V, double rtol, int maxit, cudaStream_t st);
void launch_precond_prep_pair(const Plan& P, const Vecs& V, cudaStream_t st);
void launch_pcg_first_dir_pair(const Plan& P, const Vecs& V, cudaStream_t st);
void launch_pcg_update_xr_pair(const Plan& P, const Vecs& V, cudaStream_t st, bool form_p = true);
// p = z + beta p in float pairs; sets the loop condition when cond is given
void launch_pcg_update_p_pair(const Plan& P, const Vecs& V, const cudaGraphConditionalHandle* cond,
                              cudaStream_t st);
void launch_pcg_dots_pair(const Plan& P, const Vecs& V, const cudaGraphConditionalHandle* cond, cudaStream_t st);
void launch_finalize_x_pair(const Plan& P, const Vecs& V, cudaStream_t st);

template <typename Tq>
void launch_pcg_init(const Plan& P, const Vecs& V, Tq* q, double rtol, int maxit, cudaStream_t st);
template <typename Tz>
void launch_precond_prep(const Plan& P, const Vecs& V, const double* r, cudaStream_t st);
template <typename Tz>
void launch_pcg_first_dir(const Plan& P, const Vecs& V, cudaStream_t st);
template <typename Tz, typename Tq>
void launch_pcg_update_xr(const Plan& P, const Vecs& V, const Tq* q, cudaStream_t st);
template <typename Tz, typename Tq>
void launch_pcg_dots(const Plan& P, const Vecs& V, const Tq* q, cudaStream_t st);
// p = z + beta p, q = 0; with cond, block 0 also sets the device-side loop
// condition (the iteration's last kernel)
template <typename Tz, typename Tq>
void launch_pcg_update_p(const Plan& P, const Vecs& V, Tq* q, const cudaGraphConditionalHandle* cond,
                         cudaStream_t st);
// Persistent PCG loop of the mixed forms: up to max_iters iterations over
// every slot of the plan in one cooperative launch of `blocks` blocks (at
// most persistent_blocks(prec, P.lane_big)); bar must be zero on entry.
int persistent_blocks(cgs_precision prec, bool big);
cudaError_t launch_pcg_persistent(const Plan& P, const Vecs& V, cgs_precision prec, bool hybrid, GridBar* bar,
                                  int max_iters, int blocks, cudaStream_t st);
void launch_resid_norm(const Plan& P, const Vecs& V, cudaStream_t st);

void launch_convert_f2d(const Plan& P, const float* a, double* b, bool mask, cudaStream_t st);
void launch_convert_d2f(const Plan& P, const double* a, float* b, bool mask, cudaStream_t st);
void launch_copy_d(const Plan& P, const double* a, double* b, bool mask, cudaStream_t st);
void launch_fill_d(int64_t n, double* a, double v, cudaStream_t st);
void launch_fill_f(int64_t n, float* a, float v, cudaStream_t st);

// Work tables of one mesh as slot `slot` (host side, appended to tabs).
struct MeshSizes {
    int64_t nv, ne, ntiles, n_sub, nr, n_pack, nvb, nrng, n_rpack;   // n_sub: warp-kernel subdomains
    int64_t nxseg;                                                   // XX^T pass-1 segments (0: dense)
    int64_t nhr;                                                     // hybrid restriction ranges
};
// Block sizes of the range-parallel kernels: vertices per block (vector
// kernels) and subdomains per block (local solves), and how the tiled
// applies load their element matrices.  Elements (256) and reduced rows (8)
// per block are fixed by the thread mapping.
struct Schedule {
    int vert_chunk = 1024;
    int sub_chunk = 64;
    int pack_chunk = 8;  // lane packs per block (a multiple of the 8 warps)
    int box_chunk = 1024;// box-list vertices per block of the interpolation (multiple of 256)
    int tile_tma = 0;    // 1: element tiles of the mixed-form applies staged by TMA
    int persistent = -1; // mixed-form iterations in one persistent cooperative launch:
                         // 1 yes; 0 or -1 (default) no
    int pdl = 1;         // programmatic stream serialization of the launches
    int row_packs = 1;   // lane subdomains of meshes that have row packs solved 4 lanes each
    int interp_cells = 0;// 1: interpolation by cell-sorted entries with atomic adds (the PCG
                         // dots in their own kernel); 0: by vertex with the dots fused
};
// Default schedule: enough blocks to fill the GPU (about four per SM) for
// `total` work of each kind, chunks within the kernels' ranges.
Schedule default_schedule(int64_t total_nv, int64_t total_sub, int64_t total_pack, int64_t total_lane_subs);
void append_mesh_work(std::vector<Work> (&tabs)[kWorkKinds], int mesh, int slot, int64_t voff, int64_t roff,
                      int64_t poff, const MeshSizes& z, const Schedule& sch);
int64_t mesh_partial_slots(const MeshSizes& z, const Schedule& sch);   // partial sums one slot needs

// Mesh accessors (api.cu).
const DevMesh& mesh_dev(const cgs_mesh* m);
const Plan& mesh_plan(const cgs_mesh* m);
cgs_precision mesh_prec(const cgs_mesh* m);
cgs_form mesh_form(const cgs_mesh* m);
const uint8_t* mesh_dir(const cgs_mesh* m);
// the mesh's single-step status word (device), its stop flag cleared on `st`
SolveScalars* mesh_step_status_word(cgs_mesh* m, cudaStream_t st);
int mesh_device(const cgs_mesh* m);
void set_last_error(const std::string& msg);

}  // namespace cgs
