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
//   launch_gs_update     w -= sum_j c_j X_j, then out[j] = X_j . w (j < k,
//                        when asked) and the last entry w . w of the
//                        updated w, in one pass over the X_j (the second read
//                        of X_j[i] by the same thread comes from cache)
//
// On B300 these kernels are bound by the float64 pipe (two fused
// multiply-adds per clock per SM, about one per 8 bytes of HBM traffic), not
// by HBM: every loop therefore does exactly the multiply-adds it needs (no
// padded rows), and a row loop stops at k with a uniform branch.  Each thread
// takes two entries per step with all their loads issued first, so that the
// pipe is not left waiting on one entry's loads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace cgs {
namespace {

constexpr int kProjBlock = 256;
constexpr int kProjGrid = 592;   // four blocks per SM of a 148-SM part
constexpr int kProjGroup = 8;    // kept vectors per pass over v
constexpr int kProjU = 2;        // elements per thread and step of the dots and updates

// v[i] with a Dirichlet entry read as zero; both loads are issued together
__device__ __forceinline__ double masked(const double* v, const uint8_t* dir, int64_t i) {
    const double x = __ldg(&v[i]);
    return (dir && __ldg(&dir[i])) ? 0.0 : x;
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
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    for (int j0 = 0; j0 <= k; j0 += kProjGroup) {
        const int G = min(kProjGroup, k + 1 - j0);   // rows of this group (v . v last)
        double acc[kProjGroup];
#pragma unroll
        for (int g = 0; g < kProjGroup; ++g) acc[g] = 0.0;
        // kProjU elements per thread and step: that many loads in flight
        for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kProjU * S) {
            double vi[kProjU];
#pragma unroll
            for (int u = 0; u < kProjU; ++u) {
                const int64_t i = i0 + u * S;
                vi[u] = i < n ? masked(v, dir, i) : 0.0;
            }
#pragma unroll
            for (int g = 0; g < kProjGroup; ++g) {
                if (g >= G) break;
                const int j = j0 + g;
#pragma unroll
                for (int u = 0; u < kProjU; ++u) {
                    const int64_t i = i0 + u * S;
                    const double a = i >= n ? 0.0 : j < k ? __ldg(&X[(size_t)j * n + i]) : vi[u];
                    acc[g] = fma(a, vi[u], acc[g]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < kProjGroup; ++g) {
            if (g >= G) break;
            const double t = block_reduce(acc[g], sh);
            if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (k + 1) + j0 + g] = t;
        }
    }
}

// out[j] = sum over blocks of partial[b * (k + 1) + j]: block j sums its
// column with a fixed stride-and-tree order (deterministic)
__global__ void __launch_bounds__(kProjBlock) proj_dots_final(const double* __restrict__ partial, int nblocks, int k1,
                                                              double* __restrict__ out) {
    __shared__ double sh[kProjBlock / 32];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * k1 + j];
    const double t = block_reduce(s, sh);
    if (threadIdx.x == 0) out[j] = t;
}

// out = base + sum_j (s c_j) Y_j: k multiply-adds per element (the first a
// multiply when there is no base)
__global__ void __launch_bounds__(kProjBlock) proj_combine(int64_t n, const double* __restrict__ base,
                                                           const uint8_t* __restrict__ dir, double s,
                                                           const double* __restrict__ coef, int k,
                                                           const double* __restrict__ Y, double* __restrict__ out) {
    extern __shared__ double sc[];   // s c_j, k entries
    for (int j = threadIdx.x; j < k; j += blockDim.x) sc[j] = s * coef[j];
    __syncthreads();
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += S) {
        double acc;
        int j = 0;
        if (base) {
            acc = masked(base, dir, i);
        } else if (k > 0) {
            acc = sc[0] * __ldg(&Y[i]);
            j = 1;
        } else {
            acc = 0.0;
        }
#pragma unroll 4
        for (; j < k; ++j) acc = fma(sc[j], __ldg(&Y[(size_t)j * n + i]), acc);
        out[i] = acc;
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

// w[i] -= sum_{j<k} coef[j] X_j[i] (a Dirichlet entry of w is written zero);
// then, with DOTS, partial[b * (k + 1) + j] = block b's share of X_j . w
// (j < k) and of w . w (j = k) for the updated w (KMAX >= k accumulators in
// registers); without DOTS only w . w, in partial[b].
template <int KMAX, bool DOTS>
__global__ void __launch_bounds__(kProjBlock) gs_update_partial(const double* __restrict__ X, int k, int64_t n,
                                                                const double* __restrict__ coef,
                                                                const uint8_t* __restrict__ dir, double* w,
                                                                double* __restrict__ partial) {
    extern __shared__ double sc[];   // coef, k entries
    __shared__ double sh[kProjBlock / 32];
    for (int j = threadIdx.x; j < k; j += blockDim.x) sc[j] = coef[j];
    __syncthreads();
    double acc[DOTS ? KMAX : 1];
#pragma unroll
    for (int j = 0; j < (DOTS ? KMAX : 1); ++j) acc[j] = 0.0;
    double nrm = 0.0;
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    // kProjU elements per thread and step: that many loads in flight
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kProjU * S) {
        double wi[kProjU];
#pragma unroll
        for (int u = 0; u < kProjU; ++u) {
            const int64_t i = i0 + u * S;
            wi[u] = i < n ? w[i] : 0.0;
        }
#pragma unroll 2
        for (int j = 0; j < k; ++j) {
            const double c = sc[j];
#pragma unroll
            for (int u = 0; u < kProjU; ++u) {
                const int64_t i = i0 + u * S;
                wi[u] = fma(-c, i < n ? __ldg(&X[(size_t)j * n + i]) : 0.0, wi[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kProjU; ++u) {
            const int64_t i = i0 + u * S;
            if (i >= n) continue;
            if (dir && __ldg(&dir[i])) wi[u] = 0.0;
            w[i] = wi[u];
            if (DOTS) {
#pragma unroll
                for (int j = 0; j < KMAX; ++j) {
                    if (j >= k) break;
                    acc[j] = fma(__ldg(&X[(size_t)j * n + i]), wi[u], acc[j]);
                }
            }
            nrm = fma(wi[u], wi[u], nrm);
        }
    }
    if (DOTS) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j >= k) break;
            const double t = block_reduce(acc[j], sh);
            if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (k + 1) + j] = t;
        }
    }
    const double t = block_reduce(nrm, sh);
    if (threadIdx.x == 0) partial[DOTS ? (size_t)blockIdx.x * (k + 1) + k : (size_t)blockIdx.x] = t;
}

// Grids of the reductions: as many blocks as fit on the GPU at once (one
// wave), at most kProjGrid (the partial sums are laid out for that many) and
// no more than the vector needs.
template <class Kernel>
unsigned int resident_grid(Kernel kernel, int64_t n) {
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kProjBlock, 0);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks = std::max(1, std::min(kProjGrid, std::max(1, per_sm) * std::max(1, sms)));
    }
    const int64_t g = (n + kProjBlock - 1) / kProjBlock;
    return (unsigned int)std::max<int64_t>(1, std::min<int64_t>(g, blocks));
}
// the element-wise kernels: about four elements per thread
unsigned int grid_wide(int64_t n) {
    const int64_t g = (n + 4 * kProjBlock - 1) / (4 * kProjBlock);   // grid-stride over the rest
    return (unsigned int)(g < (1 << 20) ? (g > 0 ? g : 1) : (1 << 20));
}

}  // namespace

int proj_partial_entries(int max_k) { return kProjGrid * (max_k + 1); }

void launch_proj_dots(const double* X, int k, int64_t n, const double* v, const uint8_t* dir, double* partial,
                      double* out, cudaStream_t st) {
    const unsigned int g = resident_grid(proj_dots_partial, n);
    proj_dots_partial<<<g, kProjBlock, 0, st>>>(X, k, n, v, dir, partial);
    proj_dots_final<<<k + 1, kProjBlock, 0, st>>>(partial, (int)g, k + 1, out);
}

bool launch_gs_update(const double* X, int k, int64_t n, const double* coef, const uint8_t* dir, double* w,
                      double* partial, double* out, bool dots, cudaStream_t st) {
    const size_t sm = sizeof(double) * std::max(k, 1);
    unsigned int g;
    if (!dots) {
        g = resident_grid(gs_update_partial<1, false>, n);
        gs_update_partial<1, false><<<g, kProjBlock, sm, st>>>(X, k, n, coef, dir, w, partial);
        proj_dots_final<<<1, kProjBlock, 0, st>>>(partial, (int)g, 1, out);
        return true;
    }
    if (k <= 8) {
        g = resident_grid(gs_update_partial<8, true>, n);
        gs_update_partial<8, true><<<g, kProjBlock, sm, st>>>(X, k, n, coef, dir, w, partial);
    } else if (k <= 16) {
        g = resident_grid(gs_update_partial<16, true>, n);
        gs_update_partial<16, true><<<g, kProjBlock, sm, st>>>(X, k, n, coef, dir, w, partial);
    } else if (k <= 32) {
        g = resident_grid(gs_update_partial<32, true>, n);
        gs_update_partial<32, true><<<g, kProjBlock, sm, st>>>(X, k, n, coef, dir, w, partial);
    } else {
        return false;
    }
    proj_dots_final<<<k + 1, kProjBlock, 0, st>>>(partial, (int)g, k + 1, out);
    return true;
}

void launch_proj_combine(int64_t n, const double* base, const uint8_t* dir, double s, const double* coef, int k,
                         const double* Y, double* out, cudaStream_t st) {
    proj_combine<<<grid_wide(n), kProjBlock, sizeof(double) * std::max(k, 1), st>>>(n, base, dir, s, coef, k, Y, out);
}

void launch_vec_scale(int64_t n, double* a, double alpha, cudaStream_t st) {
    vec_scale<<<grid_wide(n), kProjBlock, 0, st>>>(n, a, alpha);
}

void launch_vec_add(int64_t n, const double* a, const double* b, double* out, cudaStream_t st) {
    vec_add<<<grid_wide(n), kProjBlock, 0, st>>>(n, a, b, out);
}

}  // namespace cgs
