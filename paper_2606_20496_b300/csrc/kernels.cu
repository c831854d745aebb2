// CUDA kernels of the coarse-grid solve (sm_103a).
//
//   apply64               y += alpha Q^T A_L Q x, float64          (Sec. 3)
//   apply_pair_tiled      q  = A p, float-pair outer operator      (Sec. 3)
//   apply28f_tiled        s -= A l, float32 inner apply            (Eq. asm2)
//   local_warp            out += W_ov sum_p R_p^T A_p^{-1} R_p r   (Eq. asm1)
//   restrict              r_r += J_L^T Q W s                       (Sec. 4)
//   coarse_gemv           u_r = A_r^{-1} r_r, float64              (Sec. 4)
//   interp_add            z += W Q^T J_L u_r                       (Sec. 4)
//   pcg_*                 flexible-PCG vector updates, fused dots
//
// Every kernel works through a table of Work items, one per block: a range
// of elements, element tiles, vertices, subdomains or reduced rows of one
// solve slot (one mesh and one right-hand side).  A single solve is one slot;
// a batch of meshes and right-hand sides is many slots in the same launch.
// Mesh data comes from a device array of mesh descriptors, so the slots of
// one mesh share it (their blocks are adjacent in the tables, so repeated
// reads of the same tile hit L2).
//
// Per-slot reductions are deterministic: each block writes a partial, the
// last of the slot's blocks (ticket counter) sums them in a fixed order and
// finalises the slot's PCG scalars on the device.
//
// Layout: elements in "device order" (sorted by centroid cell).  A Dirichlet
// vertex v appears in the connectivity as ~v: reads give 0, writes skip it.
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

// Deterministic per-slot sum: every block of the slot calls this with its
// values; the last of the slot's `count` blocks gets true and the totals.
template <int NV>
__device__ bool slot_sum(double (&v)[NV], double* partials, int idx, int count, unsigned int* ticket,
                         double (&tot)[NV]) {
    __shared__ bool last;
    __shared__ double res[NV];
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) partials[(size_t)i * count + idx] = v[i];
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == (unsigned int)count - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        s[i] = 0.0;
        for (int b = threadIdx.x; b < count; b += blockDim.x) s[i] += __ldcg(&partials[(size_t)i * count + b]);
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

// Block prologue: this block's work item, its slot's scalars, and early exit
// once the slot has stopped.
#define CGS_WORK_PROLOGUE()                              \
    const Work w = work[blockIdx.x];                     \
    SolveScalars* S = V.S ? V.S + w.slot : nullptr;      \
    if (is_done(S)) return;                              \
    const DevMesh& M = meshes[w.mesh];                   \
    (void)M;

// ---------------------------------------------------------------------------
// Operator apply, float64 (FP64 form and the final true residual), 36 stored
// entries (upper triangle with diagonal).  kDot: also sum the element
// energies x_e^T A^e x_e = p.Ap (Dirichlet entries of p are 0) and finalise
// alpha = rho / pq in the slot's last block.
// ---------------------------------------------------------------------------
template <bool kDot>
__global__ void __launch_bounds__(kBlock) apply64_kernel(const DevMesh* __restrict__ meshes,
                                                         const Work* __restrict__ work, Vecs V,
                                                         const double* __restrict__ xin, double* __restrict__ yout,
                                                         double alpha) {
    CGS_WORK_PROLOGUE();
    const double* x = xin + w.voff;
    double* y = yout + w.voff;
    const int64_t ne = M.ne;
    const int64_t e = (int64_t)w.begin + threadIdx.x;
    double energy = 0.0;
    if (e < w.end) {
        int v[8];
        load_conn(M.conn, e, v);
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
                const double a = __ldg(&M.a36[(size_t)s * ne + e]);
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
        if (slot_sum<1>(val, V.partials + w.poff, w.idx, w.count, &S->ticket[0], tot) && threadIdx.x == 0) {
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
// FMA ~60x faster than FP64 (and converts between them at the FP64 rate), so
// the outer operator of the mixed forms is evaluated this way: the same
// iterates as FP64 to ~1e-14, no FP64 instruction per element.
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
// the slot is flagged CGS_ERR_TIMEOUT and stopped, and the block waits once
// more (bounded) for its copy before it may return.
constexpr int kWaitLimit = 1 << 20;
__device__ __forceinline__ bool wait_tile(uint64_t* bar, SolveScalars* S, int limit) {
    for (int i = 0; i < limit; ++i)
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

// q = A p in float-pair arithmetic (outer operator of the mixed forms): the
// difference form y_i = sum_j a_ij (x_j - x_i) keeps the error relative to
// |a||x_j - x_i|; q is summed as pairs with compensated atomics (the exact
// rounding error of each add to q.hi, recovered from the returned old value,
// goes to q.lo).  Also sums p.Ap and finalises alpha in the slot's last block.
__global__ void __launch_bounds__(kBlock) apply_pair_tiled_kernel(const DevMesh* __restrict__ meshes,
                                                                  const Work* __restrict__ work, Vecs V,
                                                                  int wait_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sh_hi = reinterpret_cast<float*>(smem);
    float* sh_lo = sh_hi + kOff * kTileElems;
    float2* ps = reinterpret_cast<float2*>(sh_lo + kOff * kTileElems);
    float2* ys = ps + kTileVerts;
    __shared__ uint64_t bar;
    CGS_WORK_PROLOGUE();
    const float2* p2 = V.p2 + w.voff;
    float2* q2 = V.q2 + w.voff;
    const int t = w.begin;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 2 * kTileSlotBytes);
        bulk_copy_g2s(sh_hi, M.at_hi + (size_t)t * kOff * kTileElems, kTileSlotBytes, &bar);
        bulk_copy_g2s(sh_lo, M.at_lo + (size_t)t * kOff * kTileElems, kTileSlotBytes, &bar);
    }
    const int e0 = __ldg(&M.tile_ptr[t]), net = __ldg(&M.tile_ptr[t + 1]) - e0;
    const int v0 = __ldg(&M.tile_vptr[t]), nvt = __ldg(&M.tile_vptr[t + 1]) - v0;
    for (int i = threadIdx.x; i < nvt; i += blockDim.x) {
        ps[i] = __ldg(&p2[__ldg(&M.tile_verts[v0 + i]) & ~kSharedBit]);
        ys[i] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const bool ok = wait_tile(&bar, S, wait_limit);
    double energy = 0.0;
    if (ok && (int)threadIdx.x < net) {
        int L[8];
        load_loc(M.eloc, e0 + threadIdx.x, L);
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
            const uint32_t raw = __ldg(&M.tile_verts[v0 + i]);
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
    if (slot_sum<1>(val, V.partials + w.poff, w.idx, w.count, &S->ticket[0], tot) && threadIdx.x == 0) {
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
__global__ void __launch_bounds__(kBlock) apply28f_tiled_kernel(const DevMesh* __restrict__ meshes,
                                                                const Work* __restrict__ work, Vecs V,
                                                                const float* __restrict__ xin,
                                                                float* __restrict__ yout, float alpha,
                                                                int wait_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sh_a = reinterpret_cast<float*>(smem);
    float* xs = sh_a + kOff * kTileElems;
    float* ys = xs + kTileVerts;
    __shared__ uint64_t bar;
    CGS_WORK_PROLOGUE();
    const float* x = xin + w.voff;
    float* y = yout + w.voff;
    const int t = w.begin;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, kTileSlotBytes);
        bulk_copy_g2s(sh_a, M.at_hi + (size_t)t * kOff * kTileElems, kTileSlotBytes, &bar);
    }
    const int e0 = __ldg(&M.tile_ptr[t]), net = __ldg(&M.tile_ptr[t + 1]) - e0;
    const int v0 = __ldg(&M.tile_vptr[t]), nvt = __ldg(&M.tile_vptr[t + 1]) - v0;
    for (int i = threadIdx.x; i < nvt; i += blockDim.x) {
        xs[i] = __ldg(&x[__ldg(&M.tile_verts[v0 + i]) & ~kSharedBit]);
        ys[i] = 0.0f;
    }
    __syncthreads();
    if (!wait_tile(&bar, S, wait_limit)) return;
    if ((int)threadIdx.x < net) {
        int L[8];
        load_loc(M.eloc, e0 + threadIdx.x, L);
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
        const uint32_t raw = __ldg(&M.tile_verts[v0 + i]);
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

template <typename Stor>
__device__ __forceinline__ const Stor* inverse_store(const DevMesh& M);
template <>
__device__ __forceinline__ const double* inverse_store<double>(const DevMesh& M) { return M.inv64; }
template <>
__device__ __forceinline__ const float* inverse_store<float>(const DevMesh& M) { return M.inv32; }
template <>
__device__ __forceinline__ const __half* inverse_store<__half>(const DevMesh& M) { return M.inv16; }

template <typename T>
__device__ __forceinline__ const T* overlap_weights(const DevMesh& M);
template <>
__device__ __forceinline__ const double* overlap_weights<double>(const DevMesh& M) { return M.wov64; }
template <>
__device__ __forceinline__ const float* overlap_weights<float>(const DevMesh& M) { return M.wov32; }

template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_warp_kernel(const DevMesh* __restrict__ meshes,
                                                            const Work* __restrict__ work, Vecs V,
                                                            const T* __restrict__ rin, T* __restrict__ outv,
                                                            int weighted) {
    CGS_WORK_PROLOGUE();
    const T* r = rin + w.voff;
    T* out = outv + w.voff;
    const Stor* inv = inverse_store<Stor>(M);
    const float* scale = M.inv16_scale;
    const T* wov = weighted ? overlap_weights<T>(M) : nullptr;
    const int lane = threadIdx.x & 31;
    for (int p = w.begin + (int)(threadIdx.x >> 5); p < w.end; p += kBlock / 32) {
        const int o = __ldg(&M.sub_ptr[p]);
        const int m = __ldg(&M.sub_ptr[p + 1]) - o;
        if (m == 0 || m > 64) continue;
        const size_t io = (size_t)__ldg(&M.inv_ptr[p]);
        const float sc = scale ? __ldg(&scale[p]) : 1.0f;
        const int nd = m / 2 + 1;
        if (m <= 32) {
            // every load of this lane is issued before the first FMA: the
            // entries inv(i, i+d) and inv(i-d, i) for d < nd <= 17
            const bool h = lane < m;
            const int v = h ? __ldg(&M.sub_idx[o + lane]) : 0;
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
            const int v0 = __ldg(&M.sub_idx[o + lane]);
            const int v1 = h1 ? __ldg(&M.sub_idx[o + lane + 32]) : 0;
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

// Subdomains with more than 64 dofs: the whole block on one subdomain, rows
// spread over threads.
template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_block_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const T* __restrict__ rin, T* __restrict__ outv,
                                                             int weighted) {
    CGS_WORK_PROLOGUE();
    const T* r = rin + w.voff;
    T* out = outv + w.voff;
    const Stor* inv = inverse_store<Stor>(M);
    const T* wov = weighted ? overlap_weights<T>(M) : nullptr;
    for (int p = w.begin; p < w.end; ++p) {
        const int o = M.sub_ptr[p];
        const int m = M.sub_ptr[p + 1] - o;
        if (m <= 64) continue;
        const size_t io = (size_t)M.inv_ptr[p];
        const float sc = M.inv16_scale ? M.inv16_scale[p] : 1.0f;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            T y = 0;
            for (int j = 0; j < m; ++j) y += diag_entry<T, Stor>(inv, io, m, i, j, sc) * __ldg(&r[M.sub_idx[o + j]]);
            const int v = M.sub_idx[o + i];
            atomicAdd(&out[v], wov ? y * wov[v] : y);
        }
    }
}

// ---------------------------------------------------------------------------
// Box coarse space.  Element e (device order) lies in cell c(e) with lower
// corner (ci,cj,ck) H (coordinates are stored relative to the box origin);
// its vertex x has local cell coordinates t = (x - corner) / H (outside
// [0,1] = extrapolation) and corner m = (ma, mb, mc) has weight
// prod_d (t_d if m_d else 1 - t_d).  Vertex records hold the coordinates and
// 1/count, so W = diag(1/count) comes with the same load.
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
__device__ __forceinline__ VertexXYZW<double> vertex_data(const DevMesh& M, double) { return {M.xyzw}; }
__device__ __forceinline__ VertexXYZW<float> vertex_data(const DevMesh& M, float) { return {M.xyzwf}; }

template <typename T>
struct BoxGrid {
    int bx, by;
    T hx, hy, hz, ihx, ihy, ihz;
    __device__ __forceinline__ explicit BoxGrid(const DevMesh& M)
        : bx(M.b[0]), by(M.b[1]), hx((T)M.H[0]), hy((T)M.H[1]), hz((T)M.H[2]), ihx((T)M.iH[0]),
          ihy((T)M.iH[1]), ihz((T)M.iH[2]) {}
};

template <typename T>
__device__ __forceinline__ void corner_weights(T tx, T ty, T tz, T (&w)[8]) {
    const T fx[2] = {T(1) - tx, tx}, fy[2] = {T(1) - ty, ty}, fz[2] = {T(1) - tz, tz};
#pragma unroll
    for (int m = 0; m < 8; ++m) w[m] = fx[m & 1] * fy[(m >> 1) & 1] * fz[(m >> 2) & 1];
}

// Warp sum of per-element cell contributions in float64 accuracy.  The FP64
// form adds doubles; the float form adds float pairs (hi, lo) with exact
// two-sums, so no FP64 instruction runs per lane and the result still
// carries ~48 significant bits.
struct CellSum64 {
    double v;
    __device__ __forceinline__ double value() const { return v; }
};
struct CellSum32 {
    float h, l;
    __device__ __forceinline__ double value() const { return (double)h + (double)l; }
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
__global__ void __launch_bounds__(kBlock) restrict_kernel(const DevMesh* __restrict__ meshes,
                                                          const Work* __restrict__ work, Vecs V,
                                                          const Tin* __restrict__ sin, double* __restrict__ rrv) {
    CGS_WORK_PROLOGUE();
    const Tin* s = sin + w.voff;
    double* rr = rrv + w.roff;
    const BoxGrid<T> g(M);
    const auto vx = vertex_data(M, T(0));
    const int64_t e = (int64_t)w.begin + threadIdx.x;
    const bool valid = e < w.end;
    T acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = T(0);
    int c = -1;
    if (valid) {
        c = __ldg(&M.cell[e]);
        const int ci = c % g.bx, cj = (c / g.bx) % g.by, ck = c / (g.bx * g.by);
        const T cx = ci * g.hx, cy = cj * g.hy, cz = ck * g.hz;
        int v[8];
        load_conn(M.conn, e, v);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (v[k] < 0) continue;
            T x, y, z, ic;
            vx.load(v[k], x, y, z, ic);
            const T sv = (T)__ldg(&s[v[k]]) * ic;
            T wt[8];
            corner_weights<T>((x - cx) * g.ihx, (y - cy) * g.ihy, (z - cz) * g.ihz, wt);
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] += wt[m] * sv;
        }
    }
    // segmented warp reduction over lanes sharing a cell
    const int lane = threadIdx.x & 31;
    unsigned int todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int cc = __shfl_sync(0xffffffffu, c, leader);
        const bool mine = valid && c == cc;
        todo &= ~__ballot_sync(0xffffffffu, mine);
        // corner m's total ends up in lane m: one FP64 conversion and one
        // atomic per corner, issued as a single warp instruction
        auto mine_sum = cell_sum(mine ? acc[0] : T(0));
#pragma unroll
        for (int m = 1; m < 8; ++m) {
            const auto sum = cell_sum(mine ? acc[m] : T(0));
            if (lane == m) mine_sum = sum;
        }
        if (lane < 8) {
            const int col = __ldg(&M.cell_cols[(size_t)cc * 8 + lane]);
            if (col >= 0) atomicAdd(&rr[col], mine_sum.value());
        }
    }
}

template <typename T, typename Tu>
__global__ void __launch_bounds__(kBlock) interp_add_kernel(const DevMesh* __restrict__ meshes,
                                                            const Work* __restrict__ work, Vecs V,
                                                            const Tu* __restrict__ urv, T* __restrict__ zv) {
    CGS_WORK_PROLOGUE();
    const Tu* ur = urv + w.roff;
    T* z = zv + w.voff;
    const int64_t e = (int64_t)w.begin + threadIdx.x;
    if (e >= w.end) return;
    const BoxGrid<T> g(M);
    const auto vx = vertex_data(M, T(0));
    const int c = __ldg(&M.cell[e]);
    const int ci = c % g.bx, cj = (c / g.bx) % g.by, ck = c / (g.bx * g.by);
    const T cx = ci * g.hx, cy = cj * g.hy, cz = ck * g.hz;
    T u[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int col = __ldg(&M.cell_cols[(size_t)c * 8 + m]);
        u[m] = col >= 0 ? (T)__ldg(&ur[col]) : T(0);
    }
    int v[8];
    load_conn(M.conn, e, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (v[k] < 0) continue;
        T x, y, zz, ic;
        vx.load(v[k], x, y, zz, ic);
        T wt[8];
        corner_weights<T>((x - cx) * g.ihx, (y - cy) * g.ihy, (zz - cz) * g.ihz, wt);
        T val = T(0);
#pragma unroll
        for (int m = 0; m < 8; ++m) val += wt[m] * u[m];
        atomicAdd(&z[v[k]], val * ic);
    }
}

// u_r = A_r^{-1} r_r: one warp per row of the full symmetric inverse; also a
// float copy of u_r for the float interpolation (no conversions per element).
__global__ void __launch_bounds__(kBlock) coarse_gemv_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const double* __restrict__ rrv,
                                                             double* __restrict__ urv, float* __restrict__ ur32v) {
    CGS_WORK_PROLOGUE();
    const int64_t nr = M.nr;
    const double* rr = rrv + w.roff;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)w.begin + (threadIdx.x >> 5);
    if (i >= w.end) return;
    const double* row = M.ar_inv + (size_t)i * nr;
    double s = 0.0;
    for (int64_t j = lane; j < nr; j += 32) s = fma(__ldg(&row[j]), __ldg(&rr[j]), s);
    s = warp_sum(s);
    if (lane == 0) {
        urv[w.roff + i] = s;
        if (ur32v) ur32v[w.roff + i] = (float)s;
    }
}

// ---------------------------------------------------------------------------
// PCG vector kernels (float64 outer iteration), over vertex ranges.
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

#define CGS_VERT_LOOP(i) for (int64_t i = (int64_t)w.begin + threadIdx.x; i < w.end; i += blockDim.x)

// r = b with Dirichlet entries zeroed, x = 0, q = 0; ||b||^2 -> bnorm2, tol2.
template <typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_init_kernel(const DevMesh* __restrict__ meshes,
                                                          const Work* __restrict__ work, Vecs V, Tq* qv,
                                                          double rtol, int maxit) {
    const Work w = work[blockIdx.x];
    SolveScalars* S = V.S + w.slot;
    const DevMesh& M = meshes[w.mesh];
    const double* b = V.bptr ? V.bptr[w.slot] : V.b + w.voff;
    double* x = V.x + w.voff;
    double* r = V.r + w.voff;
    Tq* q = qv + w.voff;
    double acc = 0.0;
    CGS_VERT_LOOP(i) {
        const double bi = M.dir[i] ? 0.0 : b[i];
        r[i] = bi;
        x[i] = 0.0;
        qzero(q, i);
        acc = fma(bi, bi, acc);
    }
    double val[1] = {acc}, tot[1];
    if (slot_sum<1>(val, V.partials + w.poff, w.idx, w.count, &S->ticket[1], tot) && threadIdx.x == 0) {
        S->bnorm2 = tot[0];
        S->tol2 = rtol * rtol * tot[0];
        S->iters = 0;
        S->maxit = maxit;
        S->loops = 0;
        S->timeouts = 0;
        S->status = CGS_OK;
        S->done = (tot[0] == 0.0 || maxit <= 0) ? 1 : 0;
        if (maxit <= 0 && tot[0] != 0.0) S->status = CGS_ERR_NO_CONVERGENCE;
        S->rho = 0.0;
    }
}

// z = 0, s = r in the bulk precision, r_r = 0 (before a preconditioner apply).
template <typename Tz>
__global__ void __launch_bounds__(kBlock) precond_prep_kernel(const DevMesh* __restrict__ meshes,
                                                              const Work* __restrict__ work, Vecs V,
                                                              const double* __restrict__ rin) {
    CGS_WORK_PROLOGUE();
    const double* r = rin + w.voff;
    Tz* z = static_cast<Tz*>(V.z) + w.voff;
    Tz* s = static_cast<Tz*>(V.s) + w.voff;
    CGS_VERT_LOOP(i) {
        z[i] = Tz(0);
        s[i] = (Tz)r[i];
    }
    // this block's share of r_r
    const int64_t chunk = (M.nr + w.count - 1) / w.count;
    const int64_t r0 = (int64_t)w.idx * chunk, r1 = min((int64_t)M.nr, r0 + chunk);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) V.rr[w.roff + i] = 0.0;
}

// p = z (and its float pair p2 when the mixed operator needs it), rho = r.z.
template <typename Tz>
__global__ void __launch_bounds__(kBlock) pcg_first_dir_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V) {
    CGS_WORK_PROLOGUE();
    const Tz* z = static_cast<const Tz*>(V.z) + w.voff;
    const double* r = V.r + w.voff;
    double* p = V.p + w.voff;
    float2* p2 = V.p2 ? V.p2 + w.voff : nullptr;
    double acc = 0.0;
    CGS_VERT_LOOP(i) {
        const double zi = (double)z[i];
        p[i] = zi;
        if (p2) p2[i] = split_pair(zi);
        acc = fma(zi, r[i], acc);
    }
    double val[1] = {acc}, tot[1];
    if (slot_sum<1>(val, V.partials + w.poff, w.idx, w.count, &S->ticket[1], tot) && threadIdx.x == 0) {
        S->rho = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        }
    }
}

// x += alpha p, r -= alpha q, ||r||^2; prepare the preconditioner buffers
// (zero z, s = r in the bulk precision, zero r_r).  The slot's last block
// counts the iteration and applies the stopping test.
template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_update_xr_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V,
                                                               const Tq* __restrict__ qv) {
    CGS_WORK_PROLOGUE();
    double* x = V.x + w.voff;
    double* r = V.r + w.voff;
    const double* p = V.p + w.voff;
    const Tq* q = qv + w.voff;
    Tz* z = static_cast<Tz*>(V.z) + w.voff;
    Tz* s = static_cast<Tz*>(V.s) + w.voff;
    const double alpha = S->alpha;
    double acc = 0.0;
    CGS_VERT_LOOP(i) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, qval(q, i), r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
        z[i] = Tz(0);
        s[i] = (Tz)ri;
    }
    const int64_t chunk = (M.nr + w.count - 1) / w.count;
    const int64_t r0 = (int64_t)w.idx * chunk, r1 = min((int64_t)M.nr, r0 + chunk);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) V.rr[w.roff + i] = 0.0;
    double val[1] = {acc}, tot[1];
    if (slot_sum<1>(val, V.partials + w.poff, w.idx, w.count, &S->ticket[2], tot) && threadIdx.x == 0) {
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
__global__ void __launch_bounds__(kBlock) pcg_dots_kernel(const DevMesh* __restrict__ meshes,
                                                          const Work* __restrict__ work, Vecs V,
                                                          const Tq* __restrict__ qv) {
    CGS_WORK_PROLOGUE();
    const Tz* z = static_cast<const Tz*>(V.z) + w.voff;
    const double* r = V.r + w.voff;
    const Tq* q = qv + w.voff;
    double zr = 0.0, zq = 0.0;
    CGS_VERT_LOOP(i) {
        const double zi = (double)z[i];
        zr = fma(zi, r[i], zr);
        zq = fma(zi, qval(q, i), zq);
    }
    double val[2] = {zr, zq}, tot[2];
    if (slot_sum<2>(val, V.partials + w.poff, w.idx, w.count, &S->ticket[3], tot) && threadIdx.x == 0) {
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

// p = z + beta p (and p2), q = 0 for the next product.
template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_update_p_kernel(const DevMesh* __restrict__ meshes,
                                                              const Work* __restrict__ work, Vecs V, Tq* qv) {
    CGS_WORK_PROLOGUE();
    const Tz* z = static_cast<const Tz*>(V.z) + w.voff;
    double* p = V.p + w.voff;
    float2* p2 = V.p2 ? V.p2 + w.voff : nullptr;
    Tq* q = qv + w.voff;
    const double beta = S->beta;
    CGS_VERT_LOOP(i) {
        const double pi = fma(beta, p[i], (double)z[i]);
        p[i] = pi;
        if (p2) p2[i] = split_pair(pi);
        qzero(q, i);
    }
}

// Condition of the device-side loop (graph while node): continue while some
// slot is still running and fewer than maxit + 2 bodies have run (slot 0
// counts the bodies; all slots share maxit).
__global__ void __launch_bounds__(kBlock) loop_cond_kernel(SolveScalars* __restrict__ S, int nslots,
                                                           cudaGraphConditionalHandle cond) {
    int running = 0;
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) running |= !*(volatile const int*)&S[i].done;
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) {
        const int loops = ++S[0].loops;
        cudaGraphSetConditional(cond, (running && loops < S[0].maxit + 2) ? 1u : 0u);
    }
}

// x_out = x (copy-out), then ||b - y||^2 and ||b||^2 over free entries.
__global__ void __launch_bounds__(kBlock) resid_norm_kernel(const DevMesh* __restrict__ meshes,
                                                            const Work* __restrict__ work, Vecs V) {
    const Work w = work[blockIdx.x];
    SolveScalars* S = V.S + w.slot;
    const DevMesh& M = meshes[w.mesh];
    const double* b = V.bptr ? V.bptr[w.slot] : V.b + w.voff;
    double* xo = V.xptr ? V.xptr[w.slot] : nullptr;
    const double* x = V.x + w.voff;
    const double* y = V.y + w.voff;
    double rn = 0.0, bn = 0.0;
    CGS_VERT_LOOP(i) {
        if (xo) xo[i] = x[i];
        if (M.dir[i]) continue;
        const double d = b[i] - y[i];
        rn = fma(d, d, rn);
        bn = fma(b[i], b[i], bn);
    }
    double val[2] = {rn, bn}, tot[2];
    if (slot_sum<2>(val, V.partials + w.poff, w.idx, w.count, &S->ticket[1], tot) && threadIdx.x == 0) {
        S->res2 = tot[0];
        S->b2 = tot[1];
    }
}

// dst = src (optionally zero at Dirichlet vertices) over the slot's vertices.
template <typename Ta, typename Tb>
__global__ void __launch_bounds__(kBlock) convert_kernel(const DevMesh* __restrict__ meshes,
                                                         const Work* __restrict__ work, const Ta* __restrict__ a,
                                                         Tb* __restrict__ b, int mask_dirichlet) {
    const Work w = work[blockIdx.x];
    const DevMesh& M = meshes[w.mesh];
    CGS_VERT_LOOP(i) b[w.voff + i] = (mask_dirichlet && M.dir[i]) ? Tb(0) : (Tb)a[w.voff + i];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) fill_kernel(int64_t n, T* __restrict__ a, T v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers.  A Plan names the mesh descriptors and the work tables of one
// set of slots (one mesh with one right-hand side, or a batch).
// ---------------------------------------------------------------------------

void launch_apply64(const Plan& P, const Vecs& V, const double* x, double* y, double alpha, bool dot,
                    cudaStream_t st) {
    if (!P.nwork[kWorkElem]) return;
    if (dot)
        apply64_kernel<true><<<P.nwork[kWorkElem], kBlock, 0, st>>>(P.meshes, P.work[kWorkElem], V, x, y, alpha);
    else
        apply64_kernel<false><<<P.nwork[kWorkElem], kBlock, 0, st>>>(P.meshes, P.work[kWorkElem], V, x, y, alpha);
}

void launch_apply_pair_tiled(const Plan& P, const Vecs& V, cudaStream_t st) {
    if (!P.nwork[kWorkTile]) return;
    const int smem = (int)(2 * kTileSlotBytes + 2 * kTileVerts * sizeof(float2));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(apply_pair_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    apply_pair_tiled_kernel<<<P.nwork[kWorkTile], kBlock, smem, st>>>(P.meshes, P.work[kWorkTile], V,
                                                                      P.wait_limit);
}

void launch_apply28f_tiled(const Plan& P, const Vecs& V, const float* x, float* y, float alpha, cudaStream_t st) {
    if (!P.nwork[kWorkTile]) return;
    const int smem = (int)(kTileSlotBytes + 2 * kTileVerts * sizeof(float));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(apply28f_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    apply28f_tiled_kernel<<<P.nwork[kWorkTile], kBlock, smem, st>>>(P.meshes, P.work[kWorkTile], V, x, y, alpha,
                                                                    P.wait_limit);
}

void launch_local(const Plan& P, const Vecs& V, cgs_precision prec, const void* r, void* out, bool weighted,
                  cudaStream_t st) {
    if (!P.nwork[kWorkSub]) return;
    const unsigned int n = P.nwork[kWorkSub];
    const Work* W = P.work[kWorkSub];
    const int wt = weighted ? 1 : 0;
    // r is float64 in the FP64 form and the float copy of the residual otherwise
    if (prec == CGS_FP64) {
        local_warp_kernel<double, double><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const double*>(r),
                                                                static_cast<double*>(out), wt);
        if (P.max_m > 64)
            local_block_kernel<double, double><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const double*>(r),
                                                                     static_cast<double*>(out), wt);
    } else if (prec == CGS_FP32_BULK) {
        local_warp_kernel<float, float><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const float*>(r),
                                                              static_cast<float*>(out), wt);
        if (P.max_m > 64)
            local_block_kernel<float, float><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const float*>(r),
                                                                   static_cast<float*>(out), wt);
    } else {
        local_warp_kernel<float, __half><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const float*>(r),
                                                               static_cast<float*>(out), wt);
        if (P.max_m > 64)
            local_block_kernel<float, __half><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const float*>(r),
                                                                    static_cast<float*>(out), wt);
    }
}

void launch_restrict(const Plan& P, const Vecs& V, bool fp64, const void* s, bool s_is_double, double* rr,
                     cudaStream_t st) {
    if (!P.nwork[kWorkElem] || !P.any_nr) return;
    const unsigned int n = P.nwork[kWorkElem];
    const Work* W = P.work[kWorkElem];
    if (fp64)
        restrict_kernel<double, double><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const double*>(s), rr);
    else if (s_is_double)
        restrict_kernel<float, double><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const double*>(s), rr);
    else
        restrict_kernel<float, float><<<n, kBlock, 0, st>>>(P.meshes, W, V, static_cast<const float*>(s), rr);
}

void launch_interp_add(const Plan& P, const Vecs& V, bool fp64, const double* ur, const float* ur32, void* z,
                       cudaStream_t st) {
    if (!P.nwork[kWorkElem] || !P.any_nr) return;
    const unsigned int n = P.nwork[kWorkElem];
    const Work* W = P.work[kWorkElem];
    if (fp64)
        interp_add_kernel<double, double><<<n, kBlock, 0, st>>>(P.meshes, W, V, ur, static_cast<double*>(z));
    else if (ur32)   // float copy of u_r written by the reduced solve: no conversions per element
        interp_add_kernel<float, float><<<n, kBlock, 0, st>>>(P.meshes, W, V, ur32, static_cast<float*>(z));
    else
        interp_add_kernel<float, double><<<n, kBlock, 0, st>>>(P.meshes, W, V, ur, static_cast<float*>(z));
}

void launch_coarse(const Plan& P, const Vecs& V, const double* rr, double* ur, float* ur32, cudaStream_t st) {
    if (!P.nwork[kWorkRow]) return;
    coarse_gemv_kernel<<<P.nwork[kWorkRow], kBlock, 0, st>>>(P.meshes, P.work[kWorkRow], V, rr, ur, ur32);
}

template <typename Tq>
void launch_pcg_init(const Plan& P, const Vecs& V, Tq* q, double rtol, int maxit, cudaStream_t st) {
    pcg_init_kernel<Tq><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], V, q, rtol, maxit);
}
template <typename Tz>
void launch_precond_prep(const Plan& P, const Vecs& V, const double* r, cudaStream_t st) {
    precond_prep_kernel<Tz><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], V, r);
}
template <typename Tz>
void launch_pcg_first_dir(const Plan& P, const Vecs& V, cudaStream_t st) {
    pcg_first_dir_kernel<Tz><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], V);
}
template <typename Tz, typename Tq>
void launch_pcg_update_xr(const Plan& P, const Vecs& V, const Tq* q, cudaStream_t st) {
    pcg_update_xr_kernel<Tz, Tq><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], V, q);
}
template <typename Tz, typename Tq>
void launch_pcg_dots(const Plan& P, const Vecs& V, const Tq* q, cudaStream_t st) {
    pcg_dots_kernel<Tz, Tq><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], V, q);
}
template <typename Tz, typename Tq>
void launch_pcg_update_p(const Plan& P, const Vecs& V, Tq* q, cudaStream_t st) {
    pcg_update_p_kernel<Tz, Tq><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], V, q);
}
void launch_loop_cond(const Plan& P, const Vecs& V, cudaGraphConditionalHandle cond, cudaStream_t st) {
    loop_cond_kernel<<<1, kBlock, 0, st>>>(V.S, P.nslots, cond);
}

void launch_resid_norm(const Plan& P, const Vecs& V, cudaStream_t st) {
    resid_norm_kernel<<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], V);
}

Schedule default_schedule(int64_t total_nv, int64_t total_sub) {
    const int64_t target = 4 * 148;
    Schedule s;
    int64_t v = (total_nv + target - 1) / target;
    s.vert_chunk = (int)std::min<int64_t>(2048, std::max<int64_t>(256, (v + 255) / 256 * 256));
    int64_t c = (total_sub + target - 1) / target;
    s.sub_chunk = (int)std::min<int64_t>(64, std::max<int64_t>(8, (c + 7) / 8 * 8));
    return s;
}

// Work tables of one mesh as one slot: element ranges, tiles, vertex ranges,
// subdomain ranges and reduced-row ranges, each numbered within the slot.
void append_mesh_work(std::vector<Work> (&tabs)[kWorkKinds], int mesh, int slot, int64_t voff, int64_t roff,
                      int64_t poff, const MeshSizes& z, const Schedule& sch) {
    auto add = [&](int kind, int64_t n, int64_t chunk) {
        const int64_t count = (n + chunk - 1) / chunk;
        for (int64_t i = 0; i < count; ++i) {
            Work w;
            w.mesh = mesh;
            w.slot = slot;
            w.voff = voff;
            w.roff = (int32_t)roff;
            w.poff = (int32_t)poff;
            w.begin = (int32_t)(i * chunk);
            w.end = (int32_t)std::min(n, (i + 1) * chunk);
            w.idx = (int32_t)i;
            w.count = (int32_t)count;
            tabs[kind].push_back(w);
        }
    };
    add(kWorkElem, z.ne, kElemChunk);
    add(kWorkTile, z.ntiles, 1);
    add(kWorkVert, z.nv, sch.vert_chunk);
    add(kWorkSub, z.n_sub, sch.sub_chunk);
    add(kWorkRow, z.nr, kRowChunk);
}

int64_t mesh_partial_slots(const MeshSizes& z, const Schedule& sch) {
    int64_t c = (z.ne + kElemChunk - 1) / kElemChunk;
    c = std::max(c, z.ntiles);
    c = std::max(c, (z.nv + sch.vert_chunk - 1) / sch.vert_chunk);
    return 2 * std::max<int64_t>(c, 1);
}

#define CGS_INST(TZ, TQ)                                                                                       \
    template void launch_pcg_update_xr<TZ, TQ>(const Plan&, const Vecs&, const TQ*, cudaStream_t);             \
    template void launch_pcg_dots<TZ, TQ>(const Plan&, const Vecs&, const TQ*, cudaStream_t);                  \
    template void launch_pcg_update_p<TZ, TQ>(const Plan&, const Vecs&, TQ*, cudaStream_t);
CGS_INST(double, double)
CGS_INST(double, float2)
CGS_INST(float, double)
CGS_INST(float, float2)
#undef CGS_INST
template void launch_pcg_init<double>(const Plan&, const Vecs&, double*, double, int, cudaStream_t);
template void launch_pcg_init<float2>(const Plan&, const Vecs&, float2*, double, int, cudaStream_t);
template void launch_precond_prep<double>(const Plan&, const Vecs&, const double*, cudaStream_t);
template void launch_precond_prep<float>(const Plan&, const Vecs&, const double*, cudaStream_t);
template void launch_pcg_first_dir<double>(const Plan&, const Vecs&, cudaStream_t);
template void launch_pcg_first_dir<float>(const Plan&, const Vecs&, cudaStream_t);

void launch_convert_f2d(const Plan& P, const float* a, double* b, bool mask, cudaStream_t st) {
    convert_kernel<float, double><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], a, b, mask);
}
void launch_convert_d2f(const Plan& P, const double* a, float* b, bool mask, cudaStream_t st) {
    convert_kernel<double, float><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], a, b, mask);
}
void launch_copy_d(const Plan& P, const double* a, double* b, bool mask, cudaStream_t st) {
    convert_kernel<double, double><<<P.nwork[kWorkVert], kBlock, 0, st>>>(P.meshes, P.work[kWorkVert], a, b, mask);
}
void launch_fill_d(int64_t n, double* a, double v, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t b = std::min<int64_t>((n + kBlock - 1) / kBlock, 148 * 8);
    fill_kernel<double><<<(unsigned int)b, kBlock, 0, st>>>(n, a, v);
}
void launch_fill_f(int64_t n, float* a, float v, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t b = std::min<int64_t>((n + kBlock - 1) / kBlock, 148 * 8);
    fill_kernel<float><<<(unsigned int)b, kBlock, 0, st>>>(n, a, v);
}

}  // namespace cgs
