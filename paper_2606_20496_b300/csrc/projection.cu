// Vector kernels of the projection onto prior solutions (Sec. 5: for
// repeated right-hand sides, solve for the change from the A-orthogonal best
// fit onto l earlier solutions).  Float64, one mesh, vectors of length n
// (the mesh's vertices); the kept vectors are the rows of an l x n array.
//
//   launch_proj_dots     out[j] = X_j . v (j < k) and out[k] = v . v, v with
//                        its Dirichlet entries taken as zero: block partials
//                        in a fixed grid, then one block sums them in a fixed
//                        order (deterministic)
//   launch_proj_combine  out = base (Dirichlet entries zeroed) + s sum_j c_j Y_j
//   launch_vec_scale     a *= alpha
//   launch_vec_add       out = a + b
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace cgs {
namespace {

constexpr int kProjBlock = 256;
constexpr int kProjGrid = 296;   // two blocks per SM of a 148-SM part
constexpr int kProjGroup = 8;    // kept vectors per pass over v

__device__ __forceinline__ double masked(const double* v, const uint8_t* dir, int64_t i) {
    return (dir && dir[i]) ? 0.0 : v[i];
}

__device__ __forceinline__ double block_reduce(double x, double* sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

// partial[b * (k + 1) + j]: block b's share of X_j . v (j < k) or v . v (j = k)
__global__ void __launch_bounds__(kProjBlock) proj_dots_partial(const double* __restrict__ X, int k, int64_t n,
                                                                const double* __restrict__ v,
                                                                const uint8_t* __restrict__ dir,
                                                                double* __restrict__ partial) {
    __shared__ double sh[kProjBlock / 32];
    for (int j0 = 0; j0 <= k; j0 += kProjGroup) {
        double acc[kProjGroup];
#pragma unroll
        for (int g = 0; g < kProjGroup; ++g) acc[g] = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double vi = masked(v, dir, i);
#pragma unroll
            for (int g = 0; g < kProjGroup; ++g) {
                const int j = j0 + g;
                if (j < k)
                    acc[g] = fma(__ldg(&X[(size_t)j * n + i]), vi, acc[g]);
                else if (j == k)
                    acc[g] = fma(vi, vi, acc[g]);
            }
        }
#pragma unroll
        for (int g = 0; g < kProjGroup; ++g) {
            if (j0 + g > k) break;
            const double t = block_reduce(acc[g], sh);
            if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (k + 1) + j0 + g] = t;
        }
    }
}

// out[j] = sum over blocks of partial[b * (k + 1) + j], blocks in order
__global__ void proj_dots_final(const double* __restrict__ partial, int nblocks, int k1, double* __restrict__ out) {
    for (int j = threadIdx.x; j < k1; j += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * k1 + j];
        out[j] = s;
    }
}

__global__ void __launch_bounds__(kProjBlock) proj_combine(int64_t n, const double* __restrict__ base,
                                                           const uint8_t* __restrict__ dir, double s,
                                                           const double* __restrict__ coef, int k,
                                                           const double* __restrict__ Y, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc = fma(__ldg(&coef[j]), __ldg(&Y[(size_t)j * n + i]), acc);
        out[i] = (base ? masked(base, dir, i) : 0.0) + s * acc;
    }
}

__global__ void __launch_bounds__(kProjBlock) vec_scale(int64_t n, double* __restrict__ a, double alpha) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] *= alpha;
}

__global__ void __launch_bounds__(kProjBlock) vec_add(int64_t n, const double* __restrict__ a,
                                                      const double* __restrict__ b, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

unsigned int grid_for(int64_t n) {
    const int64_t g = (n + kProjBlock - 1) / kProjBlock;
    return (unsigned int)(g < kProjGrid ? (g > 0 ? g : 1) : kProjGrid);
}

}  // namespace

int proj_partial_entries(int max_k) { return kProjGrid * (max_k + 1); }

void launch_proj_dots(const double* X, int k, int64_t n, const double* v, const uint8_t* dir, double* partial,
                      double* out, cudaStream_t st) {
    const unsigned int g = grid_for(n);
    proj_dots_partial<<<g, kProjBlock, 0, st>>>(X, k, n, v, dir, partial);
    proj_dots_final<<<1, 64, 0, st>>>(partial, (int)g, k + 1, out);
}

void launch_proj_combine(int64_t n, const double* base, const uint8_t* dir, double s, const double* coef, int k,
                         const double* Y, double* out, cudaStream_t st) {
    proj_combine<<<grid_for(n), kProjBlock, 0, st>>>(n, base, dir, s, coef, k, Y, out);
}

void launch_vec_scale(int64_t n, double* a, double alpha, cudaStream_t st) {
    vec_scale<<<grid_for(n), kProjBlock, 0, st>>>(n, a, alpha);
}

void launch_vec_add(int64_t n, const double* a, const double* b, double* out, cudaStream_t st) {
    vec_add<<<grid_for(n), kProjBlock, 0, st>>>(n, a, b, out);
}

}  // namespace cgs
