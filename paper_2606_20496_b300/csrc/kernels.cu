// CUDA kernels of the coarse-grid solve (sm_103a).
//
//   apply64 / apply28f  y += alpha * Q^T A_L Q x              (Sec. 3)
//   local_warp          out += W_ov sum_p R_p^T A_p^{-1} R_p r (Eq. asm1)
//   restrict_box        r_r += J_L^T Q W s                    (Sec. 4)
//   coarse_gemv         u_r = A_r^{-1} r_r                    (float64)
//   interp_add          z += W Q^T J_L u_r                    (Sec. 4)
//   pcg_*               vector updates and fused dot products of flexible PCG
//
// Layout: element data is structure-of-arrays in "device order" (elements
// sorted by centroid cell), so a warp reads 32 consecutive entries of each
// element-matrix slot and its 32 elements mostly share one box cell.  The
// connectivity of an element is two int4 loads; a Dirichlet vertex v is
// stored as ~v (negative): reads give 0, writes are skipped.
//
// Reductions are deterministic: each block writes one partial, the last
// block to finish (ticket counter) sums the partials in a fixed order and
// finalises the PCG scalars on the device, so the host never has to read a
// scalar inside the iteration.
#include <algorithm>

#include <cuda_fp16.h>

#include "internal.h"
#include "kernels.h"

namespace cgs {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool is_done(const SolveScalars* S) {
    return S != nullptr && *(volatile const int*)&S->done;
}

// Block-wide sum of NV values; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[i][w] = v[i];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = warp_sum(lane < nw ? sh[i][lane] : 0.0);
    }
}

// Grid-wide deterministic sum: every block calls this with its values; the
// last block to arrive gets true and the totals in tot (all its threads).
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* ticket, double (&tot)[NV]) {
    __shared__ bool last;
    __shared__ double res[NV];
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) partials[(size_t)i * gridDim.x + blockIdx.x] = v[i];
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        s[i] = 0.0;
        for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            s[i] += __ldcg(&partials[(size_t)i * gridDim.x + b]);
    }
    block_sum<NV>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) res[i] = s[i];
        *ticket = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = res[i];
    return true;
}

__device__ __forceinline__ void load_conn(const int32_t* __restrict__ conn, int64_t e, int (&v)[8]) {
    const int4 c0 = __ldg(reinterpret_cast<const int4*>(conn) + 2 * e);
    const int4 c1 = __ldg(reinterpret_cast<const int4*>(conn) + 2 * e + 1);
    v[0] = c0.x; v[1] = c0.y; v[2] = c0.z; v[3] = c0.w;
    v[4] = c1.x; v[5] = c1.y; v[6] = c1.z; v[7] = c1.w;
}

template <typename T>
__device__ __forceinline__ T to(double x) { return static_cast<T>(x); }

// ---------------------------------------------------------------------------
// Operator apply, float64, 36 stored entries (upper triangle with diagonal).
// kDot: also sum the element energies x_e^T A^e x_e = x^T A x (used as p.q in
// PCG; Dirichlet entries of x are zero so this equals p^T A p on free dofs),
// finalise alpha = rho / pq in the last block.
// ---------------------------------------------------------------------------
template <bool kDot>
__global__ void __launch_bounds__(kBlock) apply64_kernel(int64_t ne, const int32_t* __restrict__ conn,
                                                         const double* __restrict__ a36,
                                                         const double* __restrict__ x, double* __restrict__ y,
                                                         double alpha, double* partials, SolveScalars* S) {
    if (is_done(S)) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double energy = 0.0;
    if (e < ne) {
        int v[8];
        load_conn(conn, e, v);
        double xe[8], ye[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            xe[k] = v[k] >= 0 ? __ldg(&x[v[k]]) : 0.0;
            ye[k] = 0.0;
        }
        int s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = i; j < 8; ++j, ++s) {
                const double a = __ldg(&a36[(size_t)s * ne + e]);
                if (i == j) {
                    ye[i] = fma(a, xe[i], ye[i]);
                } else {
                    ye[i] = fma(a, xe[j], ye[i]);
                    ye[j] = fma(a, xe[i], ye[j]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (v[k] >= 0) atomicAdd(&y[v[k]], alpha * ye[k]);
            if (kDot) energy = fma(xe[k], ye[k], energy);
        }
    }
    if (kDot) {
        double val[1] = {energy}, tot[1];
        if (grid_sum<1>(val, partials, &S->ticket[0], tot) && threadIdx.x == 0) {
            const double pq = tot[0];
            S->pq = pq;
            if (!(pq > 0.0) || !isfinite(pq)) {
                S->status = CGS_ERR_BREAKDOWN;
                S->done = 1;
            } else {
                S->alpha = S->rho / pq;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Float-pair ("double-float") arithmetic on the FP32 pipes.  A value is
// hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  B300 runs FP32
// FMA ~60x faster than FP64, so the outer operator of the mixed forms is
// evaluated this way: same iterates as FP64 to ~1e-14, no FP64 instruction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ah + al)(bh + bl) ~= ph + pl (the al*bl term, ~2^-48 relative, is dropped)
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    ph = __fmul_rn(ah, bh);
    pl = __fmaf_rn(ah, bh, -ph);
    pl = __fmaf_rn(ah, bl, pl);
    pl = __fmaf_rn(al, bh, pl);
}
// (yh, yl) += (ph, pl) without renormalising (few terms per accumulator)
__device__ __forceinline__ void pair_acc(float& yh, float& yl, float ph, float pl) {
    float s, e;
    two_sum(yh, ph, s, e);
    yh = s;
    yl = __fadd_rn(yl, __fadd_rn(e, pl));
}

// ---------------------------------------------------------------------------
// Block-local assembly with TMA staging.  One block per element tile (<= 256
// consecutive elements, <= 1024 distinct free vertices).  Thread 0 starts a
// bulk asynchronous copy (cp.async.bulk, completion on an mbarrier) of the
// tile's element matrices, stored tile-major [28 slots][256 elements], into
// shared memory; meanwhile the block gathers the tile's vertex values once.
// Each thread then computes one element from 16-bit tile-local indices,
// outputs are summed in shared memory, and every tile vertex is written once:
// a plain store when no other tile touches it, an atomic otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bytes must be a multiple of 16, src and dst 16-byte aligned
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase 0 of the tile barrier with an iteration limit.  On expiry
// the solve is flagged CGS_ERR_TIMEOUT and stopped, and the block waits once
// more (bounded) for its copy before it may return.
constexpr int kWaitLimit = 1 << 20;
__device__ __forceinline__ bool wait_tile(uint64_t* bar, SolveScalars* S) {
    for (int i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, 0)) return true;
    if (S) {
        atomicAdd(&S->timeouts, 1);
        S->status = CGS_ERR_TIMEOUT;
        S->done = 1;
    }
    for (int i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, 0)) break;
    return false;
}

__device__ __forceinline__ void load_loc(const uint16_t* __restrict__ eloc, int64_t e, int (&L)[8]) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(eloc) + e);
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int lo = (int)(u[k] & 0xFFFFu), hi = (int)(u[k] >> 16);
        L[2 * k] = lo == 0xFFFF ? -1 : lo;
        L[2 * k + 1] = hi == 0xFFFF ? -1 : hi;
    }
}

constexpr uint32_t kTileSlotBytes = kOff * kTileElems * sizeof(float);   // 28 KiB

// q += A p in float-pair arithmetic (outer operator of the mixed forms): the
// difference form y_i = sum_j a_ij (x_j - x_i) keeps the error relative to
// |a||x_j - x_i|; q is summed as pairs with compensated atomics (the exact
// rounding error of each add to q.hi, recovered from the returned old value,
// goes to q.lo).  Also sums p.Ap and finalises alpha in the last block.
__global__ void __launch_bounds__(kBlock) apply_pair_tiled_kernel(
    int64_t ntiles, const int32_t* __restrict__ tile_ptr, const int32_t* __restrict__ tile_vptr,
    const uint32_t* __restrict__ tile_verts, const uint16_t* __restrict__ eloc, const float* __restrict__ at_hi,
    const float* __restrict__ at_lo, const float2* __restrict__ p2, float2* __restrict__ q2, double* partials,
    SolveScalars* S) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sh_hi = reinterpret_cast<float*>(smem);
    float* sh_lo = sh_hi + kOff * kTileElems;
    float2* ps = reinterpret_cast<float2*>(sh_lo + kOff * kTileElems);
    float2* ys = ps + kTileVerts;
    __shared__ uint64_t bar;
    if (is_done(S)) return;
    const int t = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 2 * kTileSlotBytes);
        bulk_copy_g2s(sh_hi, at_hi + (size_t)t * kOff * kTileElems, kTileSlotBytes, &bar);
        bulk_copy_g2s(sh_lo, at_lo + (size_t)t * kOff * kTileElems, kTileSlotBytes, &bar);
    }
    const int e0 = __ldg(&tile_ptr[t]), net = __ldg(&tile_ptr[t + 1]) - e0;
    const int v0 = __ldg(&tile_vptr[t]), nvt = __ldg(&tile_vptr[t + 1]) - v0;
    for (int i = threadIdx.x; i < nvt; i += blockDim.x) {
        ps[i] = __ldg(&p2[__ldg(&tile_verts[v0 + i]) & ~kSharedBit]);
        ys[i] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const bool ok = wait_tile(&bar, S);
    double energy = 0.0;
    if (ok && (int)threadIdx.x < net) {
        int L[8];
        load_loc(eloc, e0 + threadIdx.x, L);
        float xh[8], xl[8], yh[8], yl[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 t2 = L[k] >= 0 ? ps[L[k]] : make_float2(0.0f, 0.0f);
            xh[k] = t2.x;
            xl[k] = t2.y;
            yh[k] = 0.0f;
            yl[k] = 0.0f;
        }
        int s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = i + 1; j < 8; ++j, ++s) {
                const float ah = sh_hi[s * kTileElems + threadIdx.x];
                const float al = sh_lo[s * kTileElems + threadIdx.x];
                float dh, dl, t1, t2;
                two_sum(xh[j], -xh[i], t1, t2);
                t2 = __fadd_rn(t2, __fsub_rn(xl[j], xl[i]));
                fast_two_sum(t1, t2, dh, dl);
                float ph, pl;
                pair_mul(ah, al, dh, dl, ph, pl);
                pair_acc(yh[i], yl[i], ph, pl);
                pair_acc(yh[j], yl[j], -ph, -pl);
            }
        }
        float eh = 0.0f, el = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float h, l;
            fast_two_sum(yh[k], yl[k], h, l);
            float ph, pl;
            pair_mul(xh[k], xl[k], h, l, ph, pl);
            pair_acc(eh, el, ph, pl);
            if (L[k] >= 0) {
                const float old = atomicAdd(&ys[L[k]].x, h);
                float sum, err;
                two_sum(old, h, sum, err);
                atomicAdd(&ys[L[k]].y, __fadd_rn(err, l));
            }
        }
        energy = (double)eh + (double)el;
    }
    __syncthreads();
    if (ok) {
        for (int i = threadIdx.x; i < nvt; i += blockDim.x) {
            const uint32_t raw = __ldg(&tile_verts[v0 + i]);
            const int v = (int)(raw & ~kSharedBit);
            float h, l;
            fast_two_sum(ys[i].x, ys[i].y, h, l);
            if (!(raw & kSharedBit)) {
                q2[v] = make_float2(h, l);
            } else {
                float* q = reinterpret_cast<float*>(&q2[v]);
                const float old = atomicAdd(q, h);
                float sum, err;
                two_sum(old, h, sum, err);
                atomicAdd(q + 1, __fadd_rn(err, l));
            }
        }
    }
    double val[1] = {energy}, tot[1];
    if (grid_sum<1>(val, partials, &S->ticket[0], tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        S->pq = pq;
        if (S->status == CGS_ERR_TIMEOUT) {
            S->done = 1;
        } else if (!(pq > 0.0) || !isfinite(pq)) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        } else {
            S->alpha = S->rho / pq;
        }
    }
}

// y += alpha A x in float32 (inner apply s -= A l of the hybrid step).
__global__ void __launch_bounds__(kBlock) apply28f_tiled_kernel(
    int64_t ntiles, const int32_t* __restrict__ tile_ptr, const int32_t* __restrict__ tile_vptr,
    const uint32_t* __restrict__ tile_verts, const uint16_t* __restrict__ eloc, const float* __restrict__ at_hi,
    const float* __restrict__ x, float* __restrict__ y, float alpha, SolveScalars* S) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sh_a = reinterpret_cast<float*>(smem);
    float* xs = sh_a + kOff * kTileElems;
    float* ys = xs + kTileVerts;
    __shared__ uint64_t bar;
    if (is_done(S)) return;
    const int t = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, kTileSlotBytes);
        bulk_copy_g2s(sh_a, at_hi + (size_t)t * kOff * kTileElems, kTileSlotBytes, &bar);
    }
    const int e0 = __ldg(&tile_ptr[t]), net = __ldg(&tile_ptr[t + 1]) - e0;
    const int v0 = __ldg(&tile_vptr[t]), nvt = __ldg(&tile_vptr[t + 1]) - v0;
    for (int i = threadIdx.x; i < nvt; i += blockDim.x) {
        xs[i] = __ldg(&x[__ldg(&tile_verts[v0 + i]) & ~kSharedBit]);
        ys[i] = 0.0f;
    }
    __syncthreads();
    if (!wait_tile(&bar, S)) return;
    if ((int)threadIdx.x < net) {
        int L[8];
        load_loc(eloc, e0 + threadIdx.x, L);
        float xe[8], ye[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            xe[k] = L[k] >= 0 ? xs[L[k]] : 0.0f;
            ye[k] = 0.0f;
        }
        int s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = i + 1; j < 8; ++j, ++s) {
                const float d = sh_a[s * kTileElems + threadIdx.x] * (xe[j] - xe[i]);
                ye[i] += d;
                ye[j] -= d;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (L[k] >= 0) atomicAdd(&ys[L[k]], ye[k]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nvt; i += blockDim.x) {
        const uint32_t raw = __ldg(&tile_verts[v0 + i]);
        const int v = (int)(raw & ~kSharedBit);
        if (!(raw & kSharedBit))
            y[v] += alpha * ys[i];
        else
            atomicAdd(&y[v], alpha * ys[i]);
    }
}

// ---------------------------------------------------------------------------
// Local solves, one warp per subdomain with m_p <= 64 dofs.  The explicit
// symmetric inverse is stored by cyclic diagonals: entry (i, (i+d) mod m) at
// d*m + i, d = 0..floor(m/2).  Lane i then forms
//   y_i = sum_d inv(i, i+d) x_{i+d} + inv(i-d, i) x_{i-d}
// reading diagonal d at i and at (i-d) mod m: both are contiguous in memory,
// so every load of the warp is coalesced straight from global memory, and
// x_{i +- d} comes by shuffle.  m(m+1)/2 entries, m^2 FMAs, no shared memory.
// ---------------------------------------------------------------------------
template <typename Stor>
__device__ __forceinline__ float load_entry(const Stor* p, size_t i, float scale);
template <>
__device__ __forceinline__ float load_entry<float>(const float* p, size_t i, float) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float load_entry<__half>(const __half* p, size_t i, float scale) {
    return __half2float(__ldg(p + i)) * scale;
}

template <typename T, typename Stor>
__device__ __forceinline__ T stage(const Stor* p, size_t i, float scale) {
    return (T)load_entry<Stor>(p, i, scale);
}
template <>
__device__ __forceinline__ double stage<double, double>(const double* p, size_t i, float) { return __ldg(p + i); }

// inv(i, j) of an m x m symmetric inverse in the cyclic-diagonal layout
template <typename T, typename Stor>
__device__ __forceinline__ T diag_entry(const Stor* inv, size_t io, int m, int i, int j, float sc) {
    int d = j - i;
    if (d < 0) d += m;
    if (2 * d <= m) return stage<T, Stor>(inv, io + (size_t)d * m + i, sc);
    return stage<T, Stor>(inv, io + (size_t)(m - d) * m + j, sc);
}

template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_warp_kernel(int64_t n_sub, const int32_t* __restrict__ sub_ptr,
                                                            const int32_t* __restrict__ sub_idx,
                                                            const int64_t* __restrict__ inv_ptr,
                                                            const Stor* __restrict__ inv,
                                                            const float* __restrict__ scale,
                                                            const T* __restrict__ r,
                                                            const T* __restrict__ wov, T* __restrict__ out,
                                                            const SolveScalars* S) {
    if (is_done(S)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_sub; p += nwt) {
        const int o = __ldg(&sub_ptr[p]);
        const int m = __ldg(&sub_ptr[p + 1]) - o;
        if (m == 0 || m > 64) continue;
        const size_t io = (size_t)__ldg(&inv_ptr[p]);
        const float sc = scale ? __ldg(&scale[p]) : 1.0f;
        const int nd = m / 2 + 1;
        if (m <= 32) {
            // every load of this lane is issued before the first FMA: the
            // entries inv(i, i+d) and inv(i-d, i) for d < nd <= 17
            const bool h = lane < m;
            const int v = h ? __ldg(&sub_idx[o + lane]) : 0;
            T ap[17], am[17];
#pragma unroll
            for (int d = 0; d < 17; ++d) {
                int jm = lane - d;
                if (jm < 0) jm += m;
                const bool ok = h && d < nd;
                ap[d] = ok ? stage<T, Stor>(inv, io + (size_t)d * m + lane, sc) : T(0);
                am[d] = (ok && d > 0 && 2 * d != m) ? stage<T, Stor>(inv, io + (size_t)d * m + jm, sc) : T(0);
            }
            const T x = h ? __ldg(&r[v]) : T(0);
            T y = ap[0] * x;
#pragma unroll
            for (int d = 1; d < 17; ++d) {
                if (d >= nd) break;
                int jp = lane + d;
                if (jp >= m) jp -= m;
                int jm = lane - d;
                if (jm < 0) jm += m;
                const T xp = __shfl_sync(0xffffffffu, x, jp);
                const T xm = __shfl_sync(0xffffffffu, x, jm);
                y += ap[d] * xp + am[d] * xm;
            }
            if (h) atomicAdd(&out[v], wov ? y * __ldg(&wov[v]) : y);
        } else {
            // 33..64 dofs: lane holds rows lane and lane + 32
            const bool h1 = lane + 32 < m;
            const int v0 = __ldg(&sub_idx[o + lane]);
            const int v1 = h1 ? __ldg(&sub_idx[o + lane + 32]) : 0;
            const T x0 = __ldg(&r[v0]);
            const T x1 = h1 ? __ldg(&r[v1]) : T(0);
            T y0 = stage<T, Stor>(inv, io + lane, sc) * x0;
            T y1 = h1 ? stage<T, Stor>(inv, io + lane + 32, sc) * x1 : T(0);
            for (int d = 1; d < nd; ++d) {
                const size_t row = io + (size_t)d * m;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int i = lane + 32 * half;
                    int jp = i + d;
                    if (jp >= m) jp -= m;
                    int jm = i - d;
                    if (jm < 0) jm += m;
                    const T pa = __shfl_sync(0xffffffffu, x0, jp & 31), pb = __shfl_sync(0xffffffffu, x1, jp & 31);
                    const T ma = __shfl_sync(0xffffffffu, x0, jm & 31), mb = __shfl_sync(0xffffffffu, x1, jm & 31);
                    if (i < m) {
                        T acc = stage<T, Stor>(inv, row + i, sc) * (jp < 32 ? pa : pb);
                        if (2 * d != m) acc += stage<T, Stor>(inv, row + jm, sc) * (jm < 32 ? ma : mb);
                        if (half == 0)
                            y0 += acc;
                        else
                            y1 += acc;
                    }
                }
            }
            atomicAdd(&out[v0], wov ? y0 * __ldg(&wov[v0]) : y0);
            if (h1) atomicAdd(&out[v1], wov ? y1 * __ldg(&wov[v1]) : y1);
        }
    }
}

// Subdomains with more than 64 dofs: one block each, rows spread over threads.
template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_block_kernel(int64_t n_sub, const int32_t* __restrict__ sub_ptr,
                                                             const int32_t* __restrict__ sub_idx,
                                                             const int64_t* __restrict__ inv_ptr,
                                                             const Stor* __restrict__ inv,
                                                             const float* __restrict__ scale,
                                                             const T* __restrict__ r,
                                                             const T* __restrict__ wov, T* __restrict__ out,
                                                             const SolveScalars* S) {
    if (is_done(S)) return;
    for (int64_t p = blockIdx.x; p < n_sub; p += gridDim.x) {
        const int o = sub_ptr[p];
        const int m = sub_ptr[p + 1] - o;
        if (m <= 64) continue;
        const size_t io = (size_t)inv_ptr[p];
        const float sc = scale ? scale[p] : 1.0f;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            T y = 0;
            for (int j = 0; j < m; ++j) y += diag_entry<T, Stor>(inv, io, m, i, j, sc) * __ldg(&r[sub_idx[o + j]]);
            const int v = sub_idx[o + i];
            atomicAdd(&out[v], wov ? y * wov[v] : y);
        }
    }
}

// ---------------------------------------------------------------------------
// Box coarse space.  Element e (device order) lies in cell c(e) with lower
// corner lo + (ci,cj,ck) H; its vertex x has local cell coordinates
// t = (x - corner) / H (outside [0,1] = extrapolation) and corner m = (ma,
// mb, mc) has weight prod_d (t_d if m_d else 1 - t_d).  Vertex data holds the
// coordinates and 1/count, so W = diag(1/count) comes with the same load.
// ---------------------------------------------------------------------------
template <typename T>
struct VertexXYZW;
template <>
struct VertexXYZW<double> {
    const double2* p;
    __device__ __forceinline__ void load(int v, double& x, double& y, double& z, double& w) const {
        const double2 a = __ldg(p + 2 * (size_t)v), b = __ldg(p + 2 * (size_t)v + 1);
        x = a.x; y = a.y; z = b.x; w = b.y;
    }
};
template <>
struct VertexXYZW<float> {
    const float4* p;
    __device__ __forceinline__ void load(int v, float& x, float& y, float& z, float& w) const {
        const float4 a = __ldg(p + v);
        x = a.x; y = a.y; z = a.z; w = a.w;
    }
};

template <typename T>
struct BoxGrid {
    int bx, by;
    T lox, loy, loz, hx, hy, hz, ihx, ihy, ihz;
};

template <typename T>
__device__ __forceinline__ void corner_weights(T tx, T ty, T tz, T (&w)[8]) {
    const T fx[2] = {T(1) - tx, tx}, fy[2] = {T(1) - ty, ty}, fz[2] = {T(1) - tz, tz};
#pragma unroll
    for (int m = 0; m < 8; ++m) w[m] = fx[m & 1] * fy[(m >> 1) & 1] * fz[(m >> 2) & 1];
}

// Warp sum of per-element cell contributions in float64 accuracy.  The FP64
// form adds doubles; the float form adds float pairs (hi, lo) with exact
// two-sums, so no FP64 instruction runs per lane (B300 issues FP64 ~60x
// slower than FP32) and the result still carries ~48 significant bits.
struct CellSum64 {
    double v;
    __device__ __forceinline__ double value() const { return v; }
};
struct CellSum32 {
    float h, l;
    __device__ __forceinline__ double value() const { return (double)h + (double)l; }  // leader lane only
};
__device__ __forceinline__ CellSum64 cell_sum(double v) { return {warp_sum(v)}; }
__device__ __forceinline__ CellSum32 cell_sum(float v) {
    float h = v, l = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        float sh, se;
        two_sum(h, oh, sh, se);
        h = sh;
        l = __fadd_rn(l, __fadd_rn(ol, se));
    }
    return {h, l};
}

template <typename T, typename Tin>
__global__ void __launch_bounds__(kBlock) restrict_kernel(int64_t ne, const int32_t* __restrict__ conn,
                                                          const int32_t* __restrict__ cell,
                                                          const int32_t* __restrict__ cell_cols,
                                                          VertexXYZW<T> vx, BoxGrid<T> g,
                                                          const Tin* __restrict__ s, double* __restrict__ rr,
                                                          const SolveScalars* S) {
    if (is_done(S)) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = e < ne;
    T acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = T(0);
    int c = -1;
    if (valid) {
        c = __ldg(&cell[e]);
        const int ci = c % g.bx, cj = (c / g.bx) % g.by, ck = c / (g.bx * g.by);
        const T cx = g.lox + ci * g.hx, cy = g.loy + cj * g.hy, cz = g.loz + ck * g.hz;
        int v[8];
        load_conn(conn, e, v);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (v[k] < 0) continue;
            T x, y, z, ic;
            vx.load(v[k], x, y, z, ic);
            const T sv = (T)__ldg(&s[v[k]]) * ic;
            T w[8];
            corner_weights<T>((x - cx) * g.ihx, (y - cy) * g.ihy, (z - cz) * g.ihz, w);
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] += w[m] * sv;
        }
    }
    // segmented warp reduction over lanes sharing a cell, float64 sums
    const int lane = threadIdx.x & 31;
    unsigned int todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int cc = __shfl_sync(0xffffffffu, c, leader);
        const bool mine = valid && c == cc;
        todo &= ~__ballot_sync(0xffffffffu, mine);
        // corner m's total ends up in lane m (one FP64 conversion and one
        // atomic per corner, issued as a single warp instruction)
        auto mine_sum = cell_sum(mine ? acc[0] : T(0));
#pragma unroll
        for (int m = 1; m < 8; ++m) {
            const auto sum = cell_sum(mine ? acc[m] : T(0));
            if (lane == m) mine_sum = sum;
        }
        if (lane < 8) {
            const int col = __ldg(&cell_cols[(size_t)cc * 8 + lane]);
            if (col >= 0) atomicAdd(&rr[col], mine_sum.value());
        }
    }
}

template <typename T, typename Tu>
__global__ void __launch_bounds__(kBlock) interp_add_kernel(int64_t ne, const int32_t* __restrict__ conn,
                                                            const int32_t* __restrict__ cell,
                                                            const int32_t* __restrict__ cell_cols,
                                                            VertexXYZW<T> vx, BoxGrid<T> g,
                                                            const Tu* __restrict__ ur, T* __restrict__ z,
                                                            const SolveScalars* S) {
    if (is_done(S)) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int c = __ldg(&cell[e]);
    const int ci = c % g.bx, cj = (c / g.bx) % g.by, ck = c / (g.bx * g.by);
    const T cx = g.lox + ci * g.hx, cy = g.loy + cj * g.hy, cz = g.loz + ck * g.hz;
    T u[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int col = __ldg(&cell_cols[(size_t)c * 8 + m]);
        u[m] = col >= 0 ? (T)__ldg(&ur[col]) : T(0);
    }
    int v[8];
    load_conn(conn, e, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (v[k] < 0) continue;
        T x, y, zz, ic;
        vx.load(v[k], x, y, zz, ic);
        T w[8];
        corner_weights<T>((x - cx) * g.ihx, (y - cy) * g.ihy, (zz - cz) * g.ihz, w);
        T val = T(0);
#pragma unroll
        for (int m = 0; m < 8; ++m) val += w[m] * u[m];
        atomicAdd(&z[v[k]], val * ic);
    }
}

// u_r = A_r^{-1} r_r: one warp per row of the full symmetric inverse.
__global__ void __launch_bounds__(kBlock) coarse_gemv_kernel(int64_t nr, const double* __restrict__ Ainv,
                                                             const double* __restrict__ rr,
                                                             double* __restrict__ ur, float* __restrict__ ur32,
                                                             const SolveScalars* S) {
    if (is_done(S)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nr; i += nwt) {
        const double* row = Ainv + (size_t)i * nr;
        double s = 0.0;
        for (int64_t j = lane; j < nr; j += 32) s = fma(__ldg(&row[j]), __ldg(&rr[j]), s);
        s = warp_sum(s);
        if (lane == 0) {
            ur[i] = s;
            if (ur32) ur32[i] = (float)s;
        }
    }
}

// ---------------------------------------------------------------------------
// PCG vector kernels (float64 outer iteration)
// ---------------------------------------------------------------------------

// q is double (FP64 form) or a float pair (mixed forms, written by apply_pair).
__device__ __forceinline__ double qval(const double* q, int64_t i) { return q[i]; }
__device__ __forceinline__ double qval(const float2* q, int64_t i) {
    const float2 t = q[i];
    return (double)t.x + (double)t.y;
}
__device__ __forceinline__ void qzero(double* q, int64_t i) { q[i] = 0.0; }
__device__ __forceinline__ void qzero(float2* q, int64_t i) { q[i] = make_float2(0.0f, 0.0f); }
// x -> (hi, lo) float pair, hi = x rounded to float, lo = rounded remainder
__device__ __forceinline__ float2 split_pair(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// r = b with Dirichlet entries zeroed, x = 0, q = 0; ||b||^2 -> bnorm2, tol2.
template <typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_init_kernel(int64_t nv, const double* __restrict__ b,
                                                          const uint8_t* __restrict__ dir, double* __restrict__ x,
                                                          double* __restrict__ r, Tq* __restrict__ q,
                                                          double rtol, int maxit, double* partials,
                                                          SolveScalars* S) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = dir[i] ? 0.0 : b[i];
        r[i] = bi;
        x[i] = 0.0;
        qzero(q, i);
        acc = fma(bi, bi, acc);
    }
    double val[1] = {acc}, tot[1];
    if (grid_sum<1>(val, partials, &S->ticket[1], tot) && threadIdx.x == 0) {
        S->bnorm2 = tot[0];
        S->tol2 = rtol * rtol * tot[0];
        S->iters = 0;
        S->maxit = maxit;
        S->loops = 0;
        S->status = CGS_OK;
        S->done = (tot[0] == 0.0 || maxit <= 0) ? 1 : 0;
        if (maxit <= 0 && tot[0] != 0.0) S->status = CGS_ERR_NO_CONVERGENCE;
        S->rho = 0.0;
    }
}

// p = z (and its float pair p2 when the mixed operator needs it), rho = r.z.
template <typename Tz>
__global__ void __launch_bounds__(kBlock) pcg_first_dir_kernel(int64_t nv, const Tz* __restrict__ z,
                                                               const double* __restrict__ r, double* __restrict__ p,
                                                               float2* __restrict__ p2, double* partials,
                                                               SolveScalars* S) {
    if (is_done(S)) return;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = (double)z[i];
        p[i] = zi;
        if (p2) p2[i] = split_pair(zi);
        acc = fma(zi, r[i], acc);
    }
    double val[1] = {acc}, tot[1];
    if (grid_sum<1>(val, partials, &S->ticket[1], tot) && threadIdx.x == 0) {
        S->rho = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        }
    }
}

// x += alpha p, r -= alpha q, ||r||^2; prepare the preconditioner buffers
// (zero z, s = r in the bulk precision, zero r_r).  Last block: iteration
// count and the stopping test.
template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_update_xr_kernel(int64_t nv, double* __restrict__ x,
                                                               double* __restrict__ r, const double* __restrict__ p,
                                                               const Tq* __restrict__ q, Tz* __restrict__ z,
                                                               Tz* __restrict__ s, double* __restrict__ rr_vec,
                                                               int64_t nr, double* partials, SolveScalars* S) {
    if (is_done(S)) return;
    const double alpha = S->alpha;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, qval(q, i), r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
        z[i] = Tz(0);
        s[i] = (Tz)ri;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) rr_vec[i] = 0.0;
    double val[1] = {acc}, tot[1];
    if (grid_sum<1>(val, partials, &S->ticket[2], tot) && threadIdx.x == 0) {
        S->rr = tot[0];
        const int it = S->iters + 1;
        S->iters = it;
        if (!isfinite(tot[0])) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        } else if (tot[0] <= S->tol2) {
            S->status = CGS_OK;
            S->done = 1;
        } else if (it >= S->maxit) {
            S->status = CGS_ERR_NO_CONVERGENCE;
            S->done = 1;
        }
    }
}

// z.r and z.q; beta = -alpha (z.q) / rho (Polak-Ribiere, since
// r_new - r_old = -alpha q), rho = z.r.
template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_dots_kernel(int64_t nv, const Tz* __restrict__ z,
                                                          const double* __restrict__ r, const Tq* __restrict__ q,
                                                          double* partials, SolveScalars* S) {
    if (is_done(S)) return;
    double zr = 0.0, zq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = (double)z[i];
        zr = fma(zi, r[i], zr);
        zq = fma(zi, qval(q, i), zq);
    }
    double val[2] = {zr, zq}, tot[2];
    if (grid_sum<2>(val, partials, &S->ticket[3], tot) && threadIdx.x == 0) {
        S->zr = tot[0];
        S->zq = tot[1];
        const double beta = -S->alpha * tot[1] / S->rho;
        S->beta = beta;
        S->rho = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0]) || !isfinite(beta)) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        }
    }
}

// p = z + beta p (and p2), q = 0 for the next product.  Block 0 also sets
// the condition of the device-side loop when the iteration runs inside a
// graph's while node: continue while not done and fewer than maxit loops.
template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_update_p_kernel(int64_t nv, const Tz* __restrict__ z,
                                                              double* __restrict__ p, float2* __restrict__ p2,
                                                              Tq* __restrict__ q, SolveScalars* S,
                                                              cudaGraphConditionalHandle cond, int use_cond) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
        const int loops = ++S->loops;
        const bool go = !*(volatile int*)&S->done && loops < S->maxit + 2;
        cudaGraphSetConditional(cond, go ? 1u : 0u);
    }
    if (is_done(S)) return;
    const double beta = S->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double pi = fma(beta, p[i], (double)z[i]);
        p[i] = pi;
        if (p2) p2[i] = split_pair(pi);
        qzero(q, i);
    }
}

// ||b - y||^2 and ||b||^2 over free entries (true residual at the end).
__global__ void __launch_bounds__(kBlock) resid_norm_kernel(int64_t nv, const double* __restrict__ b,
                                                            const double* __restrict__ y,
                                                            const uint8_t* __restrict__ dir, double* partials,
                                                            unsigned int* ticket, double* out2) {
    double rn = 0.0, bn = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        if (dir[i]) continue;
        const double d = b[i] - y[i];
        rn = fma(d, d, rn);
        bn = fma(b[i], b[i], bn);
    }
    double val[2] = {rn, bn}, tot[2];
    if (grid_sum<2>(val, partials, ticket, tot) && threadIdx.x == 0) {
        out2[0] = tot[0];
        out2[1] = tot[1];
    }
}

template <typename Ta, typename Tb>
__global__ void __launch_bounds__(kBlock) convert_kernel(int64_t n, const Ta* __restrict__ a, Tb* __restrict__ b,
                                                         const uint8_t* __restrict__ dir) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (dir && dir[i]) ? Tb(0) : (Tb)a[i];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) fill_kernel(int64_t n, T* __restrict__ a, T v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

inline unsigned int grid_for(int64_t n, unsigned int cap = 148 * 8) {
    const int64_t b = (n + kBlock - 1) / kBlock;
    return (unsigned int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}
inline unsigned int grid_exact(int64_t n) { return (unsigned int)std::max<int64_t>(1, (n + kBlock - 1) / kBlock); }

template <typename T>
BoxGrid<T> box_grid(const DevMesh& m) {
    BoxGrid<T> g;
    g.bx = m.b[0];
    g.by = m.b[1];
    g.lox = (T)m.lo[0]; g.loy = (T)m.lo[1]; g.loz = (T)m.lo[2];
    g.hx = (T)m.H[0]; g.hy = (T)m.H[1]; g.hz = (T)m.H[2];
    g.ihx = (T)(1.0 / m.H[0]); g.ihy = (T)(1.0 / m.H[1]); g.ihz = (T)(1.0 / m.H[2]);
    return g;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

unsigned int partial_slots(const DevMesh& m) {
    const unsigned int a = std::max(grid_exact(m.ne), grid_for(m.nv));
    return std::max(a, (unsigned int)std::max<int64_t>(m.ntiles, 1));
}

void launch_apply64(const DevMesh& m, const double* x, double* y, double alpha, double* partials,
                    SolveScalars* S, bool dot, cudaStream_t st) {
    if (dot)
        apply64_kernel<true><<<grid_exact(m.ne), kBlock, 0, st>>>(m.ne, m.conn, m.a36, x, y, alpha, partials, S);
    else
        apply64_kernel<false><<<grid_exact(m.ne), kBlock, 0, st>>>(m.ne, m.conn, m.a36, x, y, alpha, partials, S);
}

template <typename T, typename Stor>
static void local_launch(const DevMesh& m, const Stor* inv, const float* scale, const T* r, const T* wov, T* out,
                         const SolveScalars* S, cudaStream_t st) {
    if (m.n_sub == 0) return;
    const unsigned int blocks =
        (unsigned int)std::max<int64_t>(1, std::min<int64_t>((m.n_sub + 7) / 8, 148 * 16));
    local_warp_kernel<T, Stor><<<blocks, kBlock, 0, st>>>(m.n_sub, m.sub_ptr, m.sub_idx, m.inv_ptr, inv, scale, r,
                                                          wov, out, S);
    if (m.max_m > 64)
        local_block_kernel<T, Stor><<<(unsigned int)std::min<int64_t>(m.n_sub, 148 * 8), kBlock, 0, st>>>(
            m.n_sub, m.sub_ptr, m.sub_idx, m.inv_ptr, inv, scale, r, wov, out, S);
}

void launch_local(const DevMesh& m, cgs_precision prec, const void* r, void* out, bool weighted,
                  const SolveScalars* S, cudaStream_t st) {
    // r is float64 in the FP64 form and the float copy of the residual otherwise
    if (prec == CGS_FP64)
        local_launch<double, double>(m, m.inv64, nullptr, static_cast<const double*>(r), weighted ? m.wov64 : nullptr,
                                     static_cast<double*>(out), S, st);
    else if (prec == CGS_FP32_BULK)
        local_launch<float, float>(m, m.inv32, nullptr, static_cast<const float*>(r), weighted ? m.wov32 : nullptr,
                                   static_cast<float*>(out), S, st);
    else
        local_launch<float, __half>(m, m.inv16, m.inv16_scale, static_cast<const float*>(r),
                                    weighted ? m.wov32 : nullptr, static_cast<float*>(out), S, st);
}

void launch_restrict(const DevMesh& m, bool fp64, const void* s, bool s_is_double, double* rr,
                     const SolveScalars* S, cudaStream_t st) {
    if (fp64) {
        VertexXYZW<double> vx{m.xyzw};
        restrict_kernel<double, double><<<grid_exact(m.ne), kBlock, 0, st>>>(
            m.ne, m.conn, m.cell, m.cell_cols, vx, box_grid<double>(m), static_cast<const double*>(s), rr, S);
    } else {
        VertexXYZW<float> vx{m.xyzwf};
        if (s_is_double)
            restrict_kernel<float, double><<<grid_exact(m.ne), kBlock, 0, st>>>(
                m.ne, m.conn, m.cell, m.cell_cols, vx, box_grid<float>(m), static_cast<const double*>(s), rr, S);
        else
            restrict_kernel<float, float><<<grid_exact(m.ne), kBlock, 0, st>>>(
                m.ne, m.conn, m.cell, m.cell_cols, vx, box_grid<float>(m), static_cast<const float*>(s), rr, S);
    }
}

void launch_interp_add(const DevMesh& m, bool fp64, const double* ur, const float* ur32, void* z,
                       const SolveScalars* S, cudaStream_t st) {
    if (fp64) {
        VertexXYZW<double> vx{m.xyzw};
        interp_add_kernel<double, double><<<grid_exact(m.ne), kBlock, 0, st>>>(
            m.ne, m.conn, m.cell, m.cell_cols, vx, box_grid<double>(m), ur, static_cast<double*>(z), S);
    } else {
        VertexXYZW<float> vx{m.xyzwf};
        if (ur32)   // float copy of u_r written by the reduced solve: no conversions per element
            interp_add_kernel<float, float><<<grid_exact(m.ne), kBlock, 0, st>>>(
                m.ne, m.conn, m.cell, m.cell_cols, vx, box_grid<float>(m), ur32, static_cast<float*>(z), S);
        else
            interp_add_kernel<float, double><<<grid_exact(m.ne), kBlock, 0, st>>>(
                m.ne, m.conn, m.cell, m.cell_cols, vx, box_grid<float>(m), ur, static_cast<float*>(z), S);
    }
}

void launch_coarse(const DevMesh& m, const double* rr, double* ur, float* ur32, const SolveScalars* S,
                   cudaStream_t st) {
    if (m.nr == 0) return;
    const unsigned int blocks = (unsigned int)std::min<int64_t>((m.nr + 7) / 8, 148 * 16);
    coarse_gemv_kernel<<<blocks, kBlock, 0, st>>>(m.nr, m.ar_inv, rr, ur, ur32, S);
}

void launch_apply_pair_tiled(const DevMesh& m, const float2* p2, float2* q2, double* partials, SolveScalars* S,
                             cudaStream_t st) {
    const int smem = (int)(2 * kTileSlotBytes + 2 * kTileVerts * sizeof(float2));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(apply_pair_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    apply_pair_tiled_kernel<<<(unsigned int)m.ntiles, kBlock, smem, st>>>(
        m.ntiles, m.tile_ptr, m.tile_vptr, m.tile_verts, m.eloc, m.at_hi, m.at_lo, p2, q2, partials, S);
}
void launch_apply28f_tiled(const DevMesh& m, const float* x, float* y, float alpha, SolveScalars* S,
                           cudaStream_t st) {
    const int smem = (int)(kTileSlotBytes + 2 * kTileVerts * sizeof(float));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(apply28f_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    apply28f_tiled_kernel<<<(unsigned int)m.ntiles, kBlock, smem, st>>>(m.ntiles, m.tile_ptr, m.tile_vptr,
                                                                        m.tile_verts, m.eloc, m.at_hi, x, y, alpha,
                                                                        S);
}

template <typename Tq>
void launch_pcg_init(const DevMesh& m, const double* b, const uint8_t* dir, double* x, double* r, Tq* q,
                     double rtol, int maxit, double* partials, SolveScalars* S, cudaStream_t st) {
    pcg_init_kernel<Tq><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, b, dir, x, r, q, rtol, maxit, partials, S);
}
template <typename Tz>
void launch_pcg_first_dir(const DevMesh& m, const Tz* z, const double* r, double* p, float2* p2, double* partials,
                          SolveScalars* S, cudaStream_t st) {
    pcg_first_dir_kernel<Tz><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, z, r, p, p2, partials, S);
}
template <typename Tz, typename Tq>
void launch_pcg_update_xr(const DevMesh& m, double* x, double* r, const double* p, const Tq* q, Tz* z, Tz* s,
                          double* rr_vec, double* partials, SolveScalars* S, cudaStream_t st) {
    pcg_update_xr_kernel<Tz, Tq><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, x, r, p, q, z, s, rr_vec, m.nr, partials,
                                                                     S);
}
template <typename Tz, typename Tq>
void launch_pcg_dots(const DevMesh& m, const Tz* z, const double* r, const Tq* q, double* partials, SolveScalars* S,
                     cudaStream_t st) {
    pcg_dots_kernel<Tz, Tq><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, z, r, q, partials, S);
}
template <typename Tz, typename Tq>
void launch_pcg_update_p(const DevMesh& m, const Tz* z, double* p, float2* p2, Tq* q, SolveScalars* S,
                         cudaGraphConditionalHandle cond, bool use_cond, cudaStream_t st) {
    pcg_update_p_kernel<Tz, Tq><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, z, p, p2, q, S, cond, use_cond ? 1 : 0);
}
#define CGS_INST(TZ, TQ)                                                                                          \
    template void launch_pcg_update_xr<TZ, TQ>(const DevMesh&, double*, double*, const double*, const TQ*, TZ*,   \
                                               TZ*, double*, double*, SolveScalars*, cudaStream_t);               \
    template void launch_pcg_dots<TZ, TQ>(const DevMesh&, const TZ*, const double*, const TQ*, double*,           \
                                          SolveScalars*, cudaStream_t);                                           \
    template void launch_pcg_update_p<TZ, TQ>(const DevMesh&, const TZ*, double*, float2*, TQ*, SolveScalars*,    \
                                              cudaGraphConditionalHandle, bool, cudaStream_t);
CGS_INST(double, double)
CGS_INST(double, float2)
CGS_INST(float, double)
CGS_INST(float, float2)
#undef CGS_INST
template void launch_pcg_init<double>(const DevMesh&, const double*, const uint8_t*, double*, double*, double*,
                                      double, int, double*, SolveScalars*, cudaStream_t);
template void launch_pcg_init<float2>(const DevMesh&, const double*, const uint8_t*, double*, double*, float2*,
                                      double, int, double*, SolveScalars*, cudaStream_t);
template void launch_pcg_first_dir<double>(const DevMesh&, const double*, const double*, double*, float2*, double*,
                                           SolveScalars*, cudaStream_t);
template void launch_pcg_first_dir<float>(const DevMesh&, const float*, const double*, double*, float2*, double*,
                                          SolveScalars*, cudaStream_t);

void launch_resid_norm(const DevMesh& m, const double* b, const double* y, const uint8_t* dir, double* partials,
                       unsigned int* ticket, double* out2, cudaStream_t st) {
    resid_norm_kernel<<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, b, y, dir, partials, ticket, out2);
}

void launch_convert_f2d(int64_t n, const float* a, double* b, const uint8_t* dir, cudaStream_t st) {
    convert_kernel<float, double><<<grid_for(n), kBlock, 0, st>>>(n, a, b, dir);
}
void launch_convert_d2f(int64_t n, const double* a, float* b, const uint8_t* dir, cudaStream_t st) {
    convert_kernel<double, float><<<grid_for(n), kBlock, 0, st>>>(n, a, b, dir);
}
void launch_copy_d(int64_t n, const double* a, double* b, const uint8_t* dir, cudaStream_t st) {
    convert_kernel<double, double><<<grid_for(n), kBlock, 0, st>>>(n, a, b, dir);
}
void launch_fill_d(int64_t n, double* a, double v, cudaStream_t st) {
    fill_kernel<double><<<grid_for(n), kBlock, 0, st>>>(n, a, v);
}
void launch_fill_f(int64_t n, float* a, float v, cudaStream_t st) {
    fill_kernel<float><<<grid_for(n), kBlock, 0, st>>>(n, a, v);
}

}  // namespace cgs
