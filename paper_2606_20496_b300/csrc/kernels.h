// Launchers of the CUDA kernels (kernels.cu), called by the C ABI (api.cu).
#pragma once

#include "internal.h"

namespace cgs {

unsigned int partial_slots(const DevMesh& m);

void launch_apply64(const DevMesh& m, const double* x, double* y, double alpha, double* partials,
                    SolveScalars* S, bool dot, cudaStream_t st);
void launch_local(const DevMesh& m, cgs_precision prec, const void* r, void* out, bool weighted,
                  const SolveScalars* S, cudaStream_t st);
void launch_restrict(const DevMesh& m, bool fp64, const void* s, bool s_is_double, double* rr,
                     const SolveScalars* S, cudaStream_t st);
void launch_interp_add(const DevMesh& m, bool fp64, const double* ur, const float* ur32, void* z,
                       const SolveScalars* S, cudaStream_t st);
void launch_coarse(const DevMesh& m, const double* rr, double* ur, float* ur32, const SolveScalars* S,
                   cudaStream_t st);
void launch_apply_pair_tiled(const DevMesh& m, const float2* p2, float2* q2, double* partials, SolveScalars* S,
                             cudaStream_t st);
void launch_apply28f_tiled(const DevMesh& m, const float* x, float* y, float alpha, SolveScalars* S,
                           cudaStream_t st);


template <typename Tq>
void launch_pcg_init(const DevMesh& m, const double* b, const uint8_t* dir, double* x, double* r, Tq* q,
                     double rtol, int maxit, double* partials, SolveScalars* S, cudaStream_t st);
template <typename Tz>
void launch_pcg_first_dir(const DevMesh& m, const Tz* z, const double* r, double* p, float2* p2, double* partials,
                          SolveScalars* S, cudaStream_t st);
template <typename Tz, typename Tq>
void launch_pcg_update_xr(const DevMesh& m, double* x, double* r, const double* p, const Tq* q, Tz* z, Tz* s,
                          double* rr_vec, double* partials, SolveScalars* S, cudaStream_t st);
template <typename Tz, typename Tq>
void launch_pcg_dots(const DevMesh& m, const Tz* z, const double* r, const Tq* q, double* partials, SolveScalars* S,
                     cudaStream_t st);
template <typename Tz, typename Tq>
void launch_pcg_update_p(const DevMesh& m, const Tz* z, double* p, float2* p2, Tq* q, SolveScalars* S,
                         cudaGraphConditionalHandle cond, bool use_cond, cudaStream_t st);
void launch_resid_norm(const DevMesh& m, const double* b, const double* y, const uint8_t* dir, double* partials,
                       unsigned int* ticket, double* out2, cudaStream_t st);

void launch_convert_f2d(int64_t n, const float* a, double* b, const uint8_t* dir, cudaStream_t st);
void launch_convert_d2f(int64_t n, const double* a, float* b, const uint8_t* dir, cudaStream_t st);
void launch_copy_d(int64_t n, const double* a, double* b, const uint8_t* dir, cudaStream_t st);
void launch_fill_d(int64_t n, double* a, double v, cudaStream_t st);
void launch_fill_f(int64_t n, float* a, float v, cudaStream_t st);

// Mesh accessors (api.cu).
const DevMesh& mesh_dev(const cgs_mesh* m);
cgs_precision mesh_prec(const cgs_mesh* m);
cgs_form mesh_form(const cgs_mesh* m);
const uint8_t* mesh_dir(const cgs_mesh* m);
int mesh_device(const cgs_mesh* m);
void set_last_error(const std::string& msg);

}  // namespace cgs
