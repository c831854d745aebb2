// CUDA kernels of the coarse-grid solve (sm_103a).
//
//   apply64               y += alpha Q^T A_L Q x, float64          (Sec. 3)
//   apply_ell64           the same by rows of the assembled A (float64 form)
//   apply_pair_tiled      q  = A p, float-pair outer operator      (Sec. 3)
//   apply_ell_pair        the same by rows of the assembled A (float pairs)
//   apply28f_tiled        s -= A l, float32 inner apply            (Eq. (5))
//   local_warp            out += W_ov sum_p R_p^T A_p^{-1} R_p r   (Eq. (4))
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
#include <type_traits>

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

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool is_done(const SolveScalars* S) {
    return S != nullptr && *(volatile const int*)&S->done;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor runs.
// pdl_wait returns once the predecessor grids have completed and their
// writes are visible, so every kernel calls it before touching data produced
// upstream.  pdl_trigger lets this grid's successor be scheduled; kernels
// call it late, just before their per-slot reduction tail (or implicitly at
// exit), so that waiting successors do not take SM resources from the
// predecessor's main work.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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

// Publish a block's values (valid in thread 0) as partial `idx` of the
// slot's `count` blocks; the last block to arrive sums the partials in a
// fixed order and gets true and the totals (deterministic per-slot sums).
template <int NV>
__device__ bool slot_publish(const double (&v)[NV], double* partials, int idx, int count, unsigned int* ticket,
                             double (&tot)[NV]) {
    __shared__ bool last;
    __shared__ double res[NV];
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
    // four independent loads and sums per thread and round (the order is
    // fixed by count and the block size: deterministic)
    double s[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        const double* pi = partials + (size_t)i * count;
        for (int b = threadIdx.x; b < count; b += 4 * blockDim.x) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int bk = b + k * (int)blockDim.x;
                if (bk < count) a[k] += __ldcg(&pi[bk]);
            }
        }
        s[i] = (a[0] + a[1]) + (a[2] + a[3]);
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

// Condition of the device-side loop (graph while node): continue while some
// slot is still running and fewer than maxit + 2 bodies have run (slot 0
// counts the bodies; all slots share maxit).  Evaluated by block 0 of the
// iteration's last kernel (a slot that breaks down inside that kernel runs
// one more, skipped, body).
__device__ __forceinline__ void loop_condition(SolveScalars* __restrict__ S, int nslots,
                                               cudaGraphConditionalHandle cond) {
    int running = 0;
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) running |= !*(volatile const int*)&S[i].done;
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) {
        const int loops = ++S[0].loops;
        cudaGraphSetConditional(cond, (running && loops < S[0].maxit + 2) ? 1u : 0u);
    }
}

// Deterministic per-slot sum of float64 values.
template <int NV>
__device__ bool slot_sum(double (&v)[NV], double* partials, int idx, int count, unsigned int* ticket,
                         double (&tot)[NV]) {
    block_sum<NV>(v);
    return slot_publish<NV>(v, partials, idx, count, ticket, tot);
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
    pdl_wait();                                          \
    SolveScalars* S = V.S ? V.S + w.slot : nullptr;      \
    if (is_done(S)) return;                              \
    const DevMesh& M = meshes[w.mesh];                   \
    (void)M;
// The same for a per-item device function that gets its work item `w`
// (kernels launched one block per item, or the persistent loop).
#define CGS_ITEM_PROLOGUE()                              \
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
__device__ __forceinline__ void apply64_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                             const double* __restrict__ xin, double* __restrict__ yout, double alpha) {
    CGS_ITEM_PROLOGUE();
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
        // (a product with alpha only when it is not 1: FP64 issue slots are
        // what bounds this kernel on B300)
        const bool scale = alpha != 1.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (v[k] >= 0) atomicAdd(&y[v[k]], scale ? alpha * ye[k] : ye[k]);
            if (kDot) energy = fma(xe[k], ye[k], energy);
        }
    }
    if (kDot) {
        double val[1] = {energy}, tot[1];
        pdl_trigger();   // the successor may launch during the reduction tail
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

// read-once loads that do not allocate in L1
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream_f64(const double* p) {
    double v;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ld_stream_f2(const float2* p) {
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

// y += alpha A x over the rows of the assembled free block (sliced ELL),
// float64: each row's entries are read once, coalesced across the warp that
// holds its slice, about 27 FP64 multiply-adds per row on hexahedral meshes
// (the element form needs 64 per element).  Dirichlet rows are padding and
// add zero to y; Dirichlet columns are not stored.  kDot: p.Ap = sum over
// rows of x_i (A x)_i and alpha for the PCG.
template <bool kDot>
__device__ __forceinline__ void apply_ell64_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                 const double* __restrict__ xin, double* __restrict__ yout,
                                                 double alpha) {
    CGS_ITEM_PROLOGUE();
    const double* x = xin + w.voff;
    double* y = yout + w.voff;
    double energy = 0.0;
    const int W = M.ell_w;
    for (int64_t i = (int64_t)w.begin + threadIdx.x; i < w.end; i += blockDim.x) {
        const int64_t o0 = (i >> 5) * 32 * (int64_t)W + (i & 31);
        double acc = 0.0;
// the entries stream past L1 (read once), which keeps L1 for the gathers
        // of x (each x_j is read by up to 27 rows); the loop unrolled over a
        // hexahedral mesh's 27 entries keeps them all in flight
#pragma unroll 27
        for (int k = 0; k < W; ++k) {
            const int32_t c = ld_stream_i32(&M.ell_col[o0 + 32 * k]);
            const double a = ld_stream_f64(&M.ell_val[o0 + 32 * k]);
            if (c >= 0) acc = fma(a, __ldg(&x[c]), acc);
        }
        y[i] = alpha == 1.0 ? y[i] + acc : fma(alpha, acc, y[i]);
        if (kDot) energy = fma(__ldg(&x[i]), acc, energy);
    }
    if (kDot) {
        double val[1] = {energy}, tot[1];
        pdl_trigger();   // the successor may launch during the reduction tail
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

template <bool kDot>
__global__ void __launch_bounds__(kBlock) apply_ell64_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const double* __restrict__ xin,
                                                             double* __restrict__ yout, double alpha) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    apply_ell64_item<kDot>(meshes, w_, V, xin, yout, alpha);
}

template <bool kDot>
__global__ void __launch_bounds__(kBlock) apply64_kernel(const DevMesh* __restrict__ meshes,
                                                         const Work* __restrict__ work, Vecs V,
                                                         const double* __restrict__ xin, double* __restrict__ yout,
                                                         double alpha) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    apply64_item<kDot>(meshes, w_, V, xin, yout, alpha);
}

// ---------------------------------------------------------------------------
// Float-pair ("double-float") arithmetic on the FP32 pipes.  A value is
// hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  B300 runs FP32
// FMA ~60x faster than FP64 (and converts between them at the FP64 rate), so
// the outer operator of the mixed forms is evaluated this way: the same
// iterates as FP64 to ~1e-14, no FP64 instruction per element.
// ---------------------------------------------------------------------------
// Zero for clearing a value that this thread has just loaded from the same
// address: 0 * x, which the compiler may not fold, so the store waits for the
// load's data.  A constant store issued while the load of its own address is
// still in flight took a slow path on B300 (about 3x the kernel time when the
// line came from DRAM).  The result is +0 or -0, an exact additive identity
// for what accumulates there next; x is finite on every path that runs on.
__device__ __forceinline__ float zero_after(float x) { return __fmul_rn(x, 0.0f); }
__device__ __forceinline__ float2 zero_after(float2 x) { return make_float2(zero_after(x.x), zero_after(x.y)); }

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

// x -> (hi, lo) float pair, hi = x rounded to float, lo = rounded remainder
__device__ __forceinline__ float2 split_pair(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// (yh, yl) += (ph, pl) without renormalising (few terms per accumulator)
__device__ __forceinline__ void pair_acc(float& yh, float& yl, float ph, float pl) {
    float s, e;
    two_sum(yh, ph, s, e);
    yh = s;
    yl = __fadd_rn(yl, __fadd_rn(e, pl));
}

__device__ __forceinline__ float2* as_pair(double* p) { return reinterpret_cast<float2*>(p); }
__device__ __forceinline__ const float2* as_pair(const double* p) { return reinterpret_cast<const float2*>(p); }

// a + b, renormalised (the low words are added once, error ~2^-48 |a + b|
// unless the high words cancel, where it stays ~2^-48 max(|a|, |b|))
__device__ __forceinline__ float2 pr_add(float2 a, float2 b) {
    float s, e, h, l;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
}

// a b + c
__device__ __forceinline__ float2 pr_fma(float2 a, float2 b, float2 c) {
    float ph, pl;
    pair_mul(a.x, a.y, b.x, b.y, ph, pl);
    return pr_add(make_float2(ph, pl), c);
}

// acc += a b (unnormalised accumulator, a few terms per thread)
__device__ __forceinline__ void pr_dot_acc(float& h, float& l, float2 a, float2 b) {
    float ph, pl;
    pair_mul(a.x, a.y, b.x, b.y, ph, pl);
    pair_acc(h, l, ph, pl);
}
__device__ __forceinline__ double pr_value(float h, float l) { return (double)h + (double)l; }

// Block-wide sum of NV float pairs on the FP32 pipes (shuffle trees of
// two-sums); the block totals are converted to float64 once, in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_pair(float (&h)[NV], float (&l)[NV]) {
    __shared__ float2 sh[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h[i], o), ol = __shfl_xor_sync(0xffffffffu, l[i], o);
            pair_acc(h[i], l[i], oh, ol);
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[i][w] = make_float2(h[i], l[i]);
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float2 t = lane < nw ? sh[i][lane] : make_float2(0.0f, 0.0f);
            h[i] = t.x;
            l[i] = t.y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, h[i], o), ol = __shfl_xor_sync(0xffffffffu, l[i], o);
                pair_acc(h[i], l[i], oh, ol);
            }
        }
    }
}

// Deterministic per-slot sum of float-pair values (block sums in pairs,
// partials and the final sum in float64).
template <int NV>
__device__ bool slot_sum_pair(float (&h)[NV], float (&l)[NV], double* partials, int idx, int count,
                              unsigned int* ticket, double (&tot)[NV]) {
    block_sum_pair<NV>(h, l);
    double v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = threadIdx.x == 0 ? pr_value(h[i], l[i]) : 0.0;
    return slot_publish<NV>(v, partials, idx, count, ticket, tot);
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

// tile-local index k (0..7) of an element from its packed 16-bit indices,
// -1 for a Dirichlet vertex
__device__ __forceinline__ int loc_of(const uint4& w, int k) {
    const uint32_t u = k < 2 ? w.x : k < 4 ? w.y : k < 6 ? w.z : w.w;
    const int v = (int)((k & 1) ? (u >> 16) : (u & 0xFFFFu));
    return v == 0xFFFF ? -1 : v;
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
constexpr int kGroups = kOff / 4;                                            // float4 groups per element

// Where a thread finds its element's off-diagonals, four slots per 16-byte
// group g: the tile staged in shared memory by TMA, or read straight from
// global memory (contiguous across the warp, streamed past L1).
struct SmemSlots {
    const float4* hi;
    const float4* lo;
    int e;
    __device__ __forceinline__ float4 h(int g) const { return hi[g * kTileElems + e]; }
    __device__ __forceinline__ float4 l(int g) const { return lo[g * kTileElems + e]; }
};
// read-only streaming load (not volatile: the compiler may hoist it)
__device__ __forceinline__ float4 ld_stream(const float4* p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}
struct GlobalSlots {
    const float4* hi;   // this tile's [7][256] groups
    const float4* lo;
    int e;
    __device__ __forceinline__ float4 h(int g) const { return ld_stream(hi + g * kTileElems + e); }
    __device__ __forceinline__ float4 l(int g) const { return ld_stream(lo + g * kTileElems + e); }
};
__device__ __forceinline__ float comp(const float4& v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

// y_e = A^e x_e in float-pair arithmetic, difference form
// y_i = sum_j a_ij (x_j - x_i): the error stays relative to |a_ij||x_j - x_i|.
// The difference is left unnormalised (hi + lo, |lo| small against the
// product's rounding), the products and sums are error-free transformations.
template <class Slots>
__device__ __forceinline__ void element_pair(const Slots& A, float4 H, float4 L, const float (&xh)[8],
                                             const float (&xl)[8], float (&yh)[8], float (&yl)[8]) {
    // group g + 1 is requested while group g is used
    float4 Hn = A.h(1), Ln = A.l(1);
    int s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = i + 1; j < 8; ++j, ++s) {
            if ((s & 3) == 0 && s > 0) {
                H = Hn;
                L = Ln;
                if ((s >> 2) + 1 < kGroups) {
                    Hn = A.h((s >> 2) + 1);
                    Ln = A.l((s >> 2) + 1);
                }
            }
            const float ah = comp(H, s & 3), al = comp(L, s & 3);
            float dh, dl;
            two_sum(xh[j], -xh[i], dh, dl);
            dl = __fadd_rn(dl, __fsub_rn(xl[j], xl[i]));
            float ph, pl;
            pair_mul(ah, al, dh, dl, ph, pl);
            pair_acc(yh[i], yl[i], ph, pl);
            pair_acc(yh[j], yl[j], -ph, -pl);
        }
    }
}

// y_e = A^e x_e in float32, difference form.
template <class Slots>
__device__ __forceinline__ void element_f32(const Slots& A, float4 H, const float (&xe)[8], float (&ye)[8]) {
    float4 Hn = A.h(1);
    int s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = i + 1; j < 8; ++j, ++s) {
            if ((s & 3) == 0 && s > 0) {
                H = Hn;
                if ((s >> 2) + 1 < kGroups) Hn = A.h((s >> 2) + 1);
            }
            const float d = comp(H, s & 3) * (xe[j] - xe[i]);
            ye[i] += d;
            ye[j] -= d;
        }
    }
}

// Up to kTileVerts / kBlock tile vertices per thread: all index loads first,
// then all value loads (two dependent round trips in total).
constexpr int kVertsPerThread = kTileVerts / kBlock;
__device__ __forceinline__ void tile_vertex_ids(const DevMesh& M, int v0, int nvt, uint32_t (&raw)[kVertsPerThread]) {
#pragma unroll
    for (int k = 0; k < kVertsPerThread; ++k) {
        const int i = (int)threadIdx.x + k * kBlock;
        raw[k] = i < nvt ? __ldg(&M.tile_verts[v0 + i]) : 0u;
    }
}

// q = A p in float-pair arithmetic (outer operator of the mixed forms), one
// block per element tile.  kTma: the tile's matrices (hi and lo, 56 KiB)
// arrive in shared memory by one bulk asynchronous copy while the block
// gathers the tile's vertex values; otherwise every thread streams its
// element's 14 groups from global memory (less shared memory, more blocks
// per SM).  Element outputs are summed in shared memory with compensated
// float atomics and every tile vertex is written once: a plain store when no
// other tile touches it, compensated global atomics otherwise.  Also sums
// p.Ap and finalises alpha in the slot's last block.
template <bool kTma>
__device__ __forceinline__ void apply_pair_tiled_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                      int wait_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    float2* ps = reinterpret_cast<float2*>(smem);
    float2* ys = ps + kTileVerts;
    float4* sh_hi = reinterpret_cast<float4*>(ys + kTileVerts);
    float4* sh_lo = sh_hi + kGroups * kTileElems;
    __shared__ uint64_t bar;
    CGS_ITEM_PROLOGUE();
    const float2* p2 = V.p2 + w.voff;
    const float* zf = static_cast<const float*>(V.z) + w.voff;
    // inside the PCG: this iteration's p is formed from z and beta on the fly
    // and p.Ap is reduced; a single step (or a timing run) applies A to p2
    const bool pcg = S && !V.step;
    const float2 beta2 = pcg ? S->beta2 : make_float2(0.0f, 0.0f);
    float2* q2 = V.q2 + w.voff;
    const int t = w.begin;
    const float4* ghi = reinterpret_cast<const float4*>(M.at_hi) + (size_t)t * kGroups * kTileElems;
    const float4* glo = reinterpret_cast<const float4*>(M.at_lo) + (size_t)t * kGroups * kTileElems;
    if (kTma && threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 2 * kTileSlotBytes);
        bulk_copy_g2s(sh_hi, ghi, kTileSlotBytes, &bar);
        bulk_copy_g2s(sh_lo, glo, kTileSlotBytes, &bar);
    }
    const int e0 = __ldg(&M.tile_ptr[t]), net = __ldg(&M.tile_ptr[t + 1]) - e0;
    const int v0 = __ldg(&M.tile_vptr[t]), nvt = __ldg(&M.tile_vptr[t + 1]) - v0;
    const bool has_e = (int)threadIdx.x < net;
    // the first group of this thread's element is requested before the gather
    float4 H = make_float4(0.f, 0.f, 0.f, 0.f), L = H;
    if (!kTma && has_e) {
        H = ld_stream(ghi + threadIdx.x);
        L = ld_stream(glo + threadIdx.x);
    }
    const uint4 lw = has_e ? __ldg(reinterpret_cast<const uint4*>(M.eloc) + e0 + threadIdx.x)
                           : make_uint4(~0u, ~0u, ~0u, ~0u);
    {
        uint32_t raw[kVertsPerThread];
        tile_vertex_ids(M, v0, nvt, raw);
        // every gather load is issued before the arithmetic and the shared
        // stores, so that the loads of one thread overlap
        float2 pg[kVertsPerThread];
        float zg[kVertsPerThread];
#pragma unroll
        for (int k = 0; k < kVertsPerThread; ++k) {
            const int i = (int)threadIdx.x + k * kBlock;
            const int v = (int)(raw[k] & ~kSharedBit);
            pg[k] = i < nvt ? __ldg(&p2[v]) : make_float2(0.0f, 0.0f);
            zg[k] = (pcg && i < nvt) ? __ldg(&zf[v]) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kVertsPerThread; ++k) {
            const int i = (int)threadIdx.x + k * kBlock;
            if (i < nvt) {
                // this iteration's direction p = z + beta p, formed on the fly
                // (the x, r update stores it)
                ps[i] = pcg ? pr_fma(beta2, pg[k], make_float2(zg[k], 0.0f)) : pg[k];
                ys[i] = make_float2(0.0f, 0.0f);
            }
        }
    }
    __syncthreads();
    bool ok = true;
    if (kTma) {
        ok = __syncthreads_and(wait_tile(&bar, S, wait_limit)) != 0;   // one decision per block
        if (ok && has_e) {
            H = sh_hi[threadIdx.x];
            L = sh_lo[threadIdx.x];
        }
    }
    float eh = 0.0f, el = 0.0f;   // this thread's share of p.Ap
    if (ok && has_e) {
        float xh[8], xl[8], yh[8], yl[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int lk = loc_of(lw, k);
            const float2 t2 = lk >= 0 ? ps[lk] : make_float2(0.0f, 0.0f);
            xh[k] = t2.x;
            xl[k] = t2.y;
            yh[k] = 0.0f;
            yl[k] = 0.0f;
        }
        if (kTma)
            element_pair(SmemSlots{sh_hi, sh_lo, (int)threadIdx.x}, H, L, xh, xl, yh, yl);
        else
            element_pair(GlobalSlots{ghi, glo, (int)threadIdx.x}, H, L, xh, xl, yh, yl);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float h, l;
            fast_two_sum(yh[k], yl[k], h, l);
            const int lk = loc_of(lw, k);
            if (lk >= 0) {
                const float old = atomicAdd(&ys[lk].x, h);
                float sum, err;
                two_sum(old, h, sum, err);
                atomicAdd(&ys[lk].y, __fadd_rn(err, l));
            }
        }
    }
    __syncthreads();
    if (ok) {
        for (int i = threadIdx.x; i < nvt; i += kBlock) {
            const uint32_t raw = __ldg(&M.tile_verts[v0 + i]);
            const int v = (int)(raw & ~kSharedBit);
            float h, l;
            fast_two_sum(ys[i].x, ys[i].y, h, l);
            // p.Ap summed as p_v times this tile's share of (A p)_v
            pr_dot_acc(eh, el, ps[i], make_float2(h, l));
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
    if (!pcg) return;   // no PCG scalars (single steps, timing runs): no reduction
    float vh[1] = {eh}, vl[1] = {el};
    double tot[1];
    pdl_trigger();   // the successor may launch during the reduction tail
    if (slot_sum_pair<1>(vh, vl, V.partials + w.poff, w.idx, w.count, &S->ticket[0], tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        S->pq = pq;
        if (S->status == CGS_ERR_TIMEOUT) {
            S->done = 1;
        } else if (!(pq > 0.0) || !isfinite(pq)) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        } else {
            S->alpha = S->rho / pq;
            S->alpha2 = split_pair(S->alpha);
        }
    }
}

template <bool kTma>
__global__ void __launch_bounds__(kBlock, kTma ? 3 : 4) apply_pair_tiled_kernel(const DevMesh* __restrict__ meshes,
                                                                                 const Work* __restrict__ work,
                                                                                 Vecs V, int wait_limit) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    apply_pair_tiled_item<kTma>(meshes, w_, V, wait_limit);
}

// q = A p in float-pair arithmetic by rows of the assembled free block
// (sliced ELL, (hi, lo) values): per entry one pair product and one pair
// accumulation, about 27 per row on hexahedral meshes, written once per
// row (no atomics).  p is this iteration's direction, stored by the p update
// that ends the previous iteration.  Inside the PCG also sums p.Ap and
// finalises alpha in the slot's last block; a single step (or a timing run)
// only applies A.
__device__ __forceinline__ void apply_ell_pair_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V) {
    CGS_ITEM_PROLOGUE();
    const bool pcg = S && !V.step;
    const float2* p2 = V.p2 + w.voff;
    float2* q2 = V.q2 + w.voff;
    const int W = M.ell_w;
    float eh = 0.0f, el = 0.0f;   // this thread's share of p.Ap
    for (int64_t i = (int64_t)w.begin + threadIdx.x; i < w.end; i += blockDim.x) {
        const int64_t o0 = (i >> 5) * 32 * (int64_t)W + (i & 31);
        float yh = 0.0f, yl = 0.0f;
#pragma unroll 27
        for (int k = 0; k < W; ++k) {
            const int32_t c = ld_stream_i32(&M.ell_col[o0 + 32 * k]);
            const float2 a = ld_stream_f2(&M.ell_pair[o0 + 32 * k]);
            if (c >= 0) {
                const float2 x = __ldg(&p2[c]);
                float ph, pl;
                pair_mul(a.x, a.y, x.x, x.y, ph, pl);
                pair_acc(yh, yl, ph, pl);
            }
        }
        float h, l;
        fast_two_sum(yh, yl, h, l);
        q2[i] = make_float2(h, l);
        if (pcg) pr_dot_acc(eh, el, __ldg(&p2[i]), make_float2(h, l));
    }
    if (!pcg) return;   // no PCG scalars (single steps, timing runs): no reduction
    float vh[1] = {eh}, vl[1] = {el};
    double tot[1];
    pdl_trigger();   // the successor may launch during the reduction tail
    if (slot_sum_pair<1>(vh, vl, V.partials + w.poff, w.idx, w.count, &S->ticket[0], tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        S->pq = pq;
        if (S->status == CGS_ERR_TIMEOUT) {
            S->done = 1;
        } else if (!(pq > 0.0) || !isfinite(pq)) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        } else {
            S->alpha = S->rho / pq;
            S->alpha2 = split_pair(S->alpha);
        }
    }
}

__global__ void __launch_bounds__(kBlock) apply_ell_pair_kernel(const DevMesh* __restrict__ meshes,
                                                                const Work* __restrict__ work, Vecs V) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    apply_ell_pair_item(meshes, w_, V);
}

// y += alpha A x in float32 (inner apply s -= A l of the hybrid step); the
// same two variants (TMA-staged tile or streamed groups).
template <bool kTma>
__device__ __forceinline__ void apply28f_tiled_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                    const float* __restrict__ xin, float* __restrict__ yout,
                                                    float alpha, int wait_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* xs = reinterpret_cast<float*>(smem);
    float* ys = xs + kTileVerts;
    float4* sh_a = reinterpret_cast<float4*>(ys + kTileVerts);
    __shared__ uint64_t bar;
    CGS_ITEM_PROLOGUE();
    const float* x = xin + w.voff;
    float* y = yout + w.voff;
    const int t = w.begin;
    const float4* ga = reinterpret_cast<const float4*>(M.at_hi) + (size_t)t * kGroups * kTileElems;
    if (kTma && threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, kTileSlotBytes);
        bulk_copy_g2s(sh_a, ga, kTileSlotBytes, &bar);
    }
    const int e0 = __ldg(&M.tile_ptr[t]), net = __ldg(&M.tile_ptr[t + 1]) - e0;
    const int v0 = __ldg(&M.tile_vptr[t]), nvt = __ldg(&M.tile_vptr[t + 1]) - v0;
    const bool has_e = (int)threadIdx.x < net;
    float4 H = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!kTma && has_e) H = ld_stream(ga + threadIdx.x);
    const uint4 lw = has_e ? __ldg(reinterpret_cast<const uint4*>(M.eloc) + e0 + threadIdx.x)
                           : make_uint4(~0u, ~0u, ~0u, ~0u);
    {
        uint32_t raw[kVertsPerThread];
        tile_vertex_ids(M, v0, nvt, raw);
#pragma unroll
        for (int k = 0; k < kVertsPerThread; ++k) {
            const int i = (int)threadIdx.x + k * kBlock;
            if (i < nvt) {
                xs[i] = __ldg(&x[raw[k] & ~kSharedBit]);
                ys[i] = 0.0f;
            }
        }
    }
    __syncthreads();
    if (kTma) {
        if (!__syncthreads_and(wait_tile(&bar, S, wait_limit))) return;   // uniform: the whole block leaves
        if (has_e) H = sh_a[threadIdx.x];
    }
    if (has_e) {
        float xe[8], ye[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int lk = loc_of(lw, k);
            xe[k] = lk >= 0 ? xs[lk] : 0.0f;
            ye[k] = 0.0f;
        }
        if (kTma)
            element_f32(SmemSlots{sh_a, nullptr, (int)threadIdx.x}, H, xe, ye);
        else
            element_f32(GlobalSlots{ga, nullptr, (int)threadIdx.x}, H, xe, ye);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int lk = loc_of(lw, k);
            if (lk >= 0) atomicAdd(&ys[lk], ye[k]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nvt; i += kBlock) {
        const uint32_t raw = __ldg(&M.tile_verts[v0 + i]);
        const int v = (int)(raw & ~kSharedBit);
        if (!(raw & kSharedBit))
            y[v] += alpha * ys[i];
        else
            atomicAdd(&y[v], alpha * ys[i]);
    }
}

template <bool kTma>
__global__ void __launch_bounds__(kBlock, 4) apply28f_tiled_kernel(const DevMesh* __restrict__ meshes,
                                                                               const Work* __restrict__ work, Vecs V,
                                                                               const float* __restrict__ xin,
                                                                               float* __restrict__ yout, float alpha,
                                                                               int wait_limit) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    apply28f_tiled_item<kTma>(meshes, w_, V, xin, yout, alpha, wait_limit);
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
// RAS weights per entry of the warp-kernel index sets
template <typename T>
__device__ __forceinline__ const T* entry_weights(const DevMesh& M);
template <>
__device__ __forceinline__ const double* entry_weights<double>(const DevMesh& M) { return M.went64; }
template <>
__device__ __forceinline__ const float* entry_weights<float>(const DevMesh& M) { return M.went32; }
// the weight of entry k (vertex v) of a subdomain: W_ov(v) (mode 1), the RAS
// entry weight (mode 2) or 1
template <typename T>
__device__ __forceinline__ T out_weight(const T* wov, const T* went, int v, int k) {
    return wov ? __ldg(&wov[v]) : went ? __ldg(&went[k]) : T(1);
}

template <typename T, typename Stor>
__device__ __forceinline__ void local_warp_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                const T* __restrict__ rin, T* __restrict__ outv, int weighted) {
    CGS_ITEM_PROLOGUE();
    const T* r = rin + w.voff;
    T* out = outv + w.voff;
    const Stor* inv = inverse_store<Stor>(M);
    const float* scale = M.inv16_scale;
    const T* wov = weighted == 1 ? overlap_weights<T>(M) : nullptr;
    const T* went = weighted == 2 ? entry_weights<T>(M) : nullptr;
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
            if (h) atomicAdd(&out[v], y * out_weight(wov, went, v, o + lane));
        } else {
            // 33..64 dofs: lane holds rows lane and lane + 32
            const bool h1 = lane + 32 < m;
            const int v0 = __ldg(&M.sub_idx[o + lane]);
            const int v1 = h1 ? __ldg(&M.sub_idx[o + lane + 32]) : 0;
            const T x0 = __ldg(&r[v0]);
            const T x1 = h1 ? __ldg(&r[v1]) : T(0);
            T y0 = stage<T, Stor>(inv, io + lane, sc) * x0;
            T y1 = h1 ? stage<T, Stor>(inv, io + lane + 32, sc) * x1 : T(0);
            // eight diagonals at a time: their (up to) 32 entries per lane are
            // loaded before the shuffles and multiply-adds that use them
            for (int d0 = 1; d0 < nd; d0 += 8) {
                T ep[2][8], em[2][8];
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const int d = d0 + g;
                    const size_t row = io + (size_t)d * m;
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int i = lane + 32 * half;
                        int jm = i - d;
                        if (jm < 0) jm += m;
                        const bool ok = d < nd && i < m;
                        ep[half][g] = ok ? stage<T, Stor>(inv, row + i, sc) : T(0);
                        em[half][g] = (ok && 2 * d != m) ? stage<T, Stor>(inv, row + jm, sc) : T(0);
                    }
                }
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const int d = d0 + g;
                    if (d >= nd) break;
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int i = lane + 32 * half;
                        int jp = i + d;
                        if (jp >= m) jp -= m;
                        int jm = i - d;
                        if (jm < 0) jm += m;
                        const T pa = __shfl_sync(0xffffffffu, x0, jp & 31), pb = __shfl_sync(0xffffffffu, x1, jp & 31);
                        const T ma = __shfl_sync(0xffffffffu, x0, jm & 31), mb = __shfl_sync(0xffffffffu, x1, jm & 31);
                        const T acc = ep[half][g] * (jp < 32 ? pa : pb) + em[half][g] * (jm < 32 ? ma : mb);
                        if (half == 0)
                            y0 += acc;
                        else
                            y1 += acc;
                    }
                }
            }
            atomicAdd(&out[v0], y0 * out_weight(wov, went, v0, o + lane));
            if (h1) atomicAdd(&out[v1], y1 * out_weight(wov, went, v1, o + lane + 32));
        }
    }
}

// ---------------------------------------------------------------------------
// Inexact local solves (Sec. 6): a fixed number of CG steps on A_p y = R_p r
// from y = 0, one warp per subdomain (m_p <= 64; lane i holds entries i and
// i + 32).  A_p is stored by cyclic diagonals like the inverses, so the
// product A_p d uses the same coalesced diagonal reads and shuffles; each
// step adds two warp sums (d.A_p d and the new residual norm).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ const T* local_matrix_store(const DevMesh& M);
template <>
__device__ __forceinline__ const double* local_matrix_store<double>(const DevMesh& M) { return M.ap64; }
template <>
__device__ __forceinline__ const float* local_matrix_store<float>(const DevMesh& M) { return M.ap32; }

// (y0, y1) = A (x0, x1) rows lane and lane + 32 of an m x m symmetric matrix
// in cyclic diagonals at a + io (entry (i, (i+d) mod m) at d m + i)
template <typename T>
__device__ __forceinline__ void cyclic_matvec(const T* __restrict__ a, size_t io, int m, int lane, T x0, T x1,
                                              T& y0, T& y1) {
    const int nd = m / 2 + 1;
    y0 = lane < m ? __ldg(&a[io + lane]) * x0 : T(0);
    y1 = lane + 32 < m ? __ldg(&a[io + lane + 32]) * x1 : T(0);
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
                T acc = __ldg(&a[row + i]) * (jp < 32 ? pa : pb);
                if (2 * d != m) acc = fma(__ldg(&a[row + jm]), jm < 32 ? ma : mb, acc);
                if (half == 0)
                    y0 += acc;
                else
                    y1 += acc;
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void local_cg_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                              const T* __restrict__ rin, T* __restrict__ outv, int weighted) {
    CGS_ITEM_PROLOGUE();
    const T* r = rin + w.voff;
    T* out = outv + w.voff;
    const T* a = local_matrix_store<T>(M);
    const T* wov = weighted == 1 ? overlap_weights<T>(M) : nullptr;
    const T* went = weighted == 2 ? entry_weights<T>(M) : nullptr;
    const int lane = threadIdx.x & 31;
    const int steps = M.cg_steps;
    for (int p = w.begin + (int)(threadIdx.x >> 5); p < w.end; p += kBlock / 32) {
        const int o = __ldg(&M.sub_ptr[p]);
        const int m = __ldg(&M.sub_ptr[p + 1]) - o;
        if (m == 0 || m > 64) continue;
        const size_t io = (size_t)__ldg(&M.inv_ptr[p]);
        const bool h0 = lane < m, h1 = lane + 32 < m;
        const int v0 = h0 ? __ldg(&M.sub_idx[o + lane]) : 0;
        const int v1 = h1 ? __ldg(&M.sub_idx[o + lane + 32]) : 0;
        T res0 = h0 ? __ldg(&r[v0]) : T(0), res1 = h1 ? __ldg(&r[v1]) : T(0);
        T y0 = T(0), y1 = T(0), d0 = res0, d1 = res1;
        T rr = warp_sum_t(fma(res0, res0, res1 * res1));
        for (int it = 0; it < steps; ++it) {
            T q0, q1;
            cyclic_matvec(a, io, m, lane, d0, d1, q0, q1);
            const T dq = warp_sum_t(fma(d0, q0, d1 * q1));
            const T al = dq > T(0) ? rr / dq : T(0);
            y0 = fma(al, d0, y0);
            y1 = fma(al, d1, y1);
            res0 = fma(-al, q0, res0);
            res1 = fma(-al, q1, res1);
            const T rn = warp_sum_t(fma(res0, res0, res1 * res1));
            const T be = rr > T(0) ? rn / rr : T(0);
            d0 = fma(be, d0, res0);
            d1 = fma(be, d1, res1);
            rr = rn;
        }
        if (h0) atomicAdd(&out[v0], y0 * out_weight(wov, went, v0, o + lane));
        if (h1) atomicAdd(&out[v1], y1 * out_weight(wov, went, v1, o + lane + 32));
    }
}

template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_warp_kernel(const DevMesh* __restrict__ meshes,
                                                            const Work* __restrict__ work, Vecs V,
                                                            const T* __restrict__ rin, T* __restrict__ outv,
                                                            int weighted) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    // a mesh set up for inexact local solves runs CG on A_p instead
    if (std::is_same<T, Stor>::value && meshes[w_.mesh].cg_steps > 0)
        local_cg_item<T>(meshes, w_, V, rin, outv, weighted);
    else
        local_warp_item<T, Stor>(meshes, w_, V, rin, outv, weighted);
}

// Subdomains with more than 64 dofs: the whole block on one subdomain, rows
// spread over threads.
template <typename T, typename Stor>
__device__ __forceinline__ void local_block_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                 const T* __restrict__ rin, T* __restrict__ outv, int weighted) {
    CGS_ITEM_PROLOGUE();
    const T* r = rin + w.voff;
    T* out = outv + w.voff;
    const Stor* inv = inverse_store<Stor>(M);
    const T* wov = weighted == 1 ? overlap_weights<T>(M) : nullptr;
    const T* went = weighted == 2 ? entry_weights<T>(M) : nullptr;
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
            atomicAdd(&out[v], y * out_weight(wov, went, v, o + i));
        }
    }
}

template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_block_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const T* __restrict__ rin, T* __restrict__ outv,
                                                             int weighted) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    local_block_item<T, Stor>(meshes, w_, V, rin, outv, weighted);
}

// ---------------------------------------------------------------------------
// Local solves of the mixed forms, one lane per subdomain.  A warp takes a
// pack of 32 subdomains of one size class M (<= 32 dofs, zero-padded): lane
// l keeps its subdomain's x and y (M values each) in registers and walks the
// upper triangle of its inverse, a_ij feeding y_i += a_ij x_j and
// y_j += a_ij x_i.  The entries of the 32 lanes are interleaved in 16-byte
// groups, so each load of the warp reads 512 contiguous bytes; every entry is
// read once, and the warp issues ~M^2/32 + 2M instructions per subdomain
// (the warp-per-subdomain form needs ~20x more).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ld_stream_u4(const uint4* p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ double2 ld_stream_d2(const double2* p) {
    double2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

// entries of one lane, group by group: float (4 per group) or half (8)
struct LaneEntries32 {
    const float4* a;   // pack base, groups [g][32]
    int lane;
    float4 cur;
    __device__ __forceinline__ float get(int e) {
        if ((e & 3) == 0) cur = ld_stream(a + (e >> 2) * 32 + lane);
        return comp(cur, e & 3);
    }
};
struct LaneEntries16 {
    const uint4* a;    // pack base, groups [g][32] of 8 halves
    int lane;
    float scale;
    uint4 cur;
    __device__ __forceinline__ float get(int e) {
        if ((e & 7) == 0) cur = ld_stream_u4(a + (e >> 3) * 32 + lane);
        const uint32_t w = (e & 7) < 2 ? cur.x : (e & 7) < 4 ? cur.y : (e & 7) < 6 ? cur.z : cur.w;
        const __half2 h2 = *reinterpret_cast<const __half2*>(&w);
        return ((e & 1) ? __high2float(h2) : __low2float(h2)) * scale;
    }
};

// entries of one lane in the FP64 form: groups of two doubles
struct LaneEntries64 {
    const double2* a;   // pack base, groups [g][32]
    int lane;
    double2 cur;
    __device__ __forceinline__ double get(int e) {
        if ((e & 1) == 0) cur = ld_stream_d2(a + (e >> 1) * 32 + lane);
        return (e & 1) ? cur.y : cur.x;
    }
};

// wov: W_ov per vertex (hybrid), went: a weight per entry aligned with idx
// (the RAS prolongation), or neither (additive)
template <int Mc, typename T, class Entries>
__device__ __forceinline__ void lane_solve(Entries A, const int32_t* __restrict__ idx, const T* __restrict__ r,
                                           T* __restrict__ out, const T* __restrict__ wov, const T* __restrict__ went,
                                           int lane) {
    T x[Mc], y[Mc];
#pragma unroll
    for (int k = 0; k < Mc; ++k) {
        const int v = __ldg(&idx[k * 32 + lane]);
        x[k] = v >= 0 ? __ldg(&r[v]) : T(0);
        y[k] = T(0);
    }
    int e = 0;
#pragma unroll
    for (int i = 0; i < Mc; ++i) {
#pragma unroll
        for (int j = i; j < Mc; ++j, ++e) {
            const T a = A.get(e);
            if (i == j) {
                y[i] = fma(a, x[i], y[i]);
            } else {
                y[i] = fma(a, x[j], y[i]);
                y[j] = fma(a, x[i], y[j]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < Mc; ++k) {
        const int v = __ldg(&idx[k * 32 + lane]);
        if (v >= 0)
            atomicAdd(&out[v], wov ? y[k] * __ldg(&wov[v]) : went ? y[k] * __ldg(&went[k * 32 + lane]) : y[k]);
    }
}

// the size classes of up to 32 dofs (kBig false) or above (kBig true, the
// mixed forms only: a lane keeps 2 x 64 floats in registers, so these run in
// kernels of their own with one block per SM, leaving the small classes'
// occupancy alone); a class of the other group does nothing
template <bool kBig, typename T, class Entries>
__device__ __forceinline__ void lane_dispatch(int Mc, const Entries& A, const int32_t* idx, const T* r, T* out,
                                              const T* wov, const T* went, int lane) {
    if (!kBig) {
        switch (Mc) {
            case 8: lane_solve<8, T>(A, idx, r, out, wov, went, lane); break;
            case 12: lane_solve<12, T>(A, idx, r, out, wov, went, lane); break;
            case 16: lane_solve<16, T>(A, idx, r, out, wov, went, lane); break;
            case 18: lane_solve<18, T>(A, idx, r, out, wov, went, lane); break;
            case 20: lane_solve<20, T>(A, idx, r, out, wov, went, lane); break;
            case 24: lane_solve<24, T>(A, idx, r, out, wov, went, lane); break;
            case 27: lane_solve<27, T>(A, idx, r, out, wov, went, lane); break;
            case 32: lane_solve<32, T>(A, idx, r, out, wov, went, lane); break;
            default: break;
        }
    } else {
        switch (Mc) {
            case 40: lane_solve<40, T>(A, idx, r, out, wov, went, lane); break;
            case 48: lane_solve<48, T>(A, idx, r, out, wov, went, lane); break;
            case 56: lane_solve<56, T>(A, idx, r, out, wov, went, lane); break;
            case 64: lane_solve<64, T>(A, idx, r, out, wov, went, lane); break;
            default: break;
        }
    }
}

// out += W_ov sum_p R_p^T A_p^{-1} R_p r over the lane packs (float r, out)
// of the small classes, or (kBig) of the classes above 32 dofs.
template <typename Stor, bool kBig = false>
__device__ __forceinline__ void local_lane_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                const float* __restrict__ rin, float* __restrict__ outv, int weighted) {
    CGS_ITEM_PROLOGUE();
    const float* r = rin + w.voff;
    float* out = outv + w.voff;
    const float* wov = weighted == 1 ? M.wov32 : nullptr;
    const int lane = threadIdx.x & 31;
    for (int pk = w.begin + (int)(threadIdx.x >> 5); pk < w.end; pk += kBlock / 32) {
        const int Mc = __ldg(&M.pack_m[pk]);
        const int64_t io = __ldg(&M.pack_idx_off[pk]);
        const int32_t* idx = M.pack_idx + io;
        const float* went = weighted == 2 ? M.pack_went32 + io : nullptr;
        const int64_t ao = __ldg(&M.pack_inv_off[pk]);
        if (std::is_same<Stor, float>::value) {
            LaneEntries32 A{reinterpret_cast<const float4*>(M.pack_inv32 + ao), lane, {}};
            lane_dispatch<kBig>(Mc, A, idx, r, out, wov, went, lane);
        } else {
            LaneEntries16 A{reinterpret_cast<const uint4*>(M.pack_inv16 + ao), lane,
                            __ldg(&M.pack_scale[(size_t)pk * 32 + lane]), {}};
            lane_dispatch<kBig>(Mc, A, idx, r, out, wov, went, lane);
        }
    }
}

template <typename Stor>
__global__ void __launch_bounds__(kBlock, 2) local_lane_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V,
                                                               const float* __restrict__ rin,
                                                               float* __restrict__ outv, int weighted) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    local_lane_item<Stor>(meshes, w_, V, rin, outv, weighted);
}

// the classes above 32 dofs (mixed forms): one block of 8 warps per SM
template <typename Stor>
__global__ void __launch_bounds__(kBlock, 1) local_lane_big_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V,
                                                               const float* __restrict__ rin,
                                                               float* __restrict__ outv, int weighted) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    local_lane_item<Stor, true>(meshes, w_, V, rin, outv, weighted);
}

// The FP64 form's lane packs (meshes with many small subdomains): the same
// one-lane-per-subdomain product in float64.  A lane holds 2 M doubles of x
// and y in registers, so one block per SM (up to 255 registers a thread);
// the kernel is bound by the FP64 FMA rate, M^2 FMAs per subdomain.  (A
// variant with x in shared memory and two blocks per SM spilled and ran
// 16% slower on the cylinder.)
// One block per SM, each pack of 32 subdomains handled by one warp; packs
// are dealt so that block b takes the packs whose virtual index (item x
// chunk + position) is b modulo the grid, its warps in turn: every SM gets
// the same share of the (class-sorted, largest first) packs, to within one,
// instead of the last of several waves of blocks running on part of the GPU.
__global__ void __launch_bounds__(kBlock, 1) local_lane64_kernel(const DevMesh* __restrict__ meshes,
                                                                 const Work* __restrict__ work, int nitems, int chunk,
                                                                 Vecs V, const double* __restrict__ rin,
                                                                 double* __restrict__ outv, int weighted) {
    pdl_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nvirt = (int64_t)nitems * chunk;
    for (int64_t v = blockIdx.x + (int64_t)gridDim.x * warp; v < nvirt; v += (int64_t)gridDim.x * (kBlock / 32)) {
        const Work& w = work[v / chunk];
        const int pk = w.begin + (int)(v % chunk);
        if (pk >= w.end) continue;
        SolveScalars* S = V.S ? V.S + w.slot : nullptr;
        if (is_done(S)) continue;
        const DevMesh& M = meshes[w.mesh];
        const double* r = rin + w.voff;
        double* out = outv + w.voff;
        const double* wov = weighted == 1 ? M.wov64 : nullptr;
        const int Mc = __ldg(&M.pack_m[pk]);
        const int64_t io = __ldg(&M.pack_idx_off[pk]);
        const int32_t* idx = M.pack_idx + io;
        const double* went = weighted == 2 ? M.pack_went64 + io : nullptr;
        const int64_t ao = __ldg(&M.pack_inv_off[pk]);
        LaneEntries64 A{reinterpret_cast<const double2*>(M.pack_inv64 + ao), lane, {}};
        lane_dispatch<false, double>(Mc, A, idx, r, out, wov, went, lane);
    }
}

// ---------------------------------------------------------------------------
// Local solves of small meshes, four lanes per subdomain (row packs): a warp
// takes 8 subdomains of one size class; lane 4 s + g keeps subdomain s's x
// (M values) and forms y_i = sum_j inv(i, j) x_j for its rows i = g, g + 4,
// ... from full stored rows.  Twice the entries of the triangle, a quarter
// of the sequential work per lane: for meshes too small to fill the GPU one
// lane per subdomain.
// ---------------------------------------------------------------------------
template <int Mc, class Entries>
__device__ __forceinline__ void row_solve(Entries A, const int32_t* __restrict__ idx, const float* __restrict__ r,
                                          float* __restrict__ out, const float* __restrict__ wov,
                                          const float* __restrict__ went, int lane) {
    constexpr int R = row_pack_rows(Mc);
    const int g = lane % kRowLanes;
    float x[Mc], y[R];
#pragma unroll
    for (int k = 0; k < Mc; ++k) {
        const int v = __ldg(&idx[k * 32 + lane]);
        x[k] = v >= 0 ? __ldg(&r[v]) : 0.0f;
    }
    int e = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < Mc; ++j, ++e) acc = fmaf(A.get(e), x[j], acc);
        y[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = q * kRowLanes + g;
        if (i >= Mc) continue;
        const int v = __ldg(&idx[i * 32 + lane]);
        if (v >= 0)
            atomicAdd(&out[v], wov ? y[q] * __ldg(&wov[v]) : went ? y[q] * __ldg(&went[i * 32 + lane]) : y[q]);
    }
}

template <bool kBig, class Entries>
__device__ __forceinline__ void row_dispatch(int Mc, const Entries& A, const int32_t* idx, const float* r,
                                             float* out, const float* wov, const float* went, int lane) {
    if (!kBig) {
        switch (Mc) {
            case 8: row_solve<8>(A, idx, r, out, wov, went, lane); break;
            case 12: row_solve<12>(A, idx, r, out, wov, went, lane); break;
            case 16: row_solve<16>(A, idx, r, out, wov, went, lane); break;
            case 18: row_solve<18>(A, idx, r, out, wov, went, lane); break;
            case 20: row_solve<20>(A, idx, r, out, wov, went, lane); break;
            case 24: row_solve<24>(A, idx, r, out, wov, went, lane); break;
            case 27: row_solve<27>(A, idx, r, out, wov, went, lane); break;
            case 32: row_solve<32>(A, idx, r, out, wov, went, lane); break;
            default: break;
        }
    } else {
        switch (Mc) {
            case 40: row_solve<40>(A, idx, r, out, wov, went, lane); break;
            case 48: row_solve<48>(A, idx, r, out, wov, went, lane); break;
            case 56: row_solve<56>(A, idx, r, out, wov, went, lane); break;
            case 64: row_solve<64>(A, idx, r, out, wov, went, lane); break;
            default: break;
        }
    }
}

// out += W_ov sum_p R_p^T A_p^{-1} R_p r over the row packs (float r, out)
// of the small classes, or (kBig) of the classes above 32 dofs.
template <typename Stor, bool kBig = false>
__device__ __forceinline__ void local_rowpack_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                   const float* __restrict__ rin, float* __restrict__ outv,
                                                   int weighted) {
    CGS_ITEM_PROLOGUE();
    const float* r = rin + w.voff;
    float* out = outv + w.voff;
    const float* wov = weighted == 1 ? M.wov32 : nullptr;
    const int lane = threadIdx.x & 31;
    for (int pk = w.begin + (int)(threadIdx.x >> 5); pk < w.end; pk += kBlock / 32) {
        const int Mc = __ldg(&M.rpack_m[pk]);
        const int64_t io = __ldg(&M.rpack_idx_off[pk]);
        const int32_t* idx = M.rpack_idx + io;
        const float* went = weighted == 2 ? M.rpack_went32 + io : nullptr;
        const int64_t ao = __ldg(&M.rpack_inv_off[pk]);
        if (std::is_same<Stor, float>::value) {
            LaneEntries32 A{reinterpret_cast<const float4*>(M.rpack_inv32 + ao), lane, {}};
            row_dispatch<kBig>(Mc, A, idx, r, out, wov, went, lane);
        } else {
            LaneEntries16 A{reinterpret_cast<const uint4*>(M.rpack_inv16 + ao), lane,
                            __ldg(&M.rpack_scale[(size_t)pk * 32 + lane]), {}};
            row_dispatch<kBig>(Mc, A, idx, r, out, wov, went, lane);
        }
    }
}
template <typename Stor>
__global__ void __launch_bounds__(kBlock) local_rowpack_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V,
                                                               const float* __restrict__ rin,
                                                               float* __restrict__ outv, int weighted) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    local_rowpack_item<Stor>(meshes, w_, V, rin, outv, weighted);
}

// the classes above 32 dofs (mixed forms)
template <typename Stor>
__global__ void __launch_bounds__(kBlock, 1) local_rowpack_big_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V,
                                                               const float* __restrict__ rin,
                                                               float* __restrict__ outv, int weighted) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    local_rowpack_item<Stor, true>(meshes, w_, V, rin, outv, weighted);
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

// Box sizes H and 1/H in the kernel's precision (the float copies are
// rounded at setup: no conversion per thread).
template <typename T>
struct BoxGrid;
template <>
struct BoxGrid<double> {
    int bx, by;
    double hx, hy, hz, ihx, ihy, ihz;
    __device__ __forceinline__ explicit BoxGrid(const DevMesh& M)
        : bx(M.b[0]), by(M.b[1]), hx(M.H[0]), hy(M.H[1]), hz(M.H[2]), ihx(M.iH[0]), ihy(M.iH[1]), ihz(M.iH[2]) {}
};
template <>
struct BoxGrid<float> {
    int bx, by;
    float hx, hy, hz, ihx, ihy, ihz;
    __device__ __forceinline__ explicit BoxGrid(const DevMesh& M)
        : bx(M.b[0]), by(M.b[1]), hx(M.Hf[0]), hy(M.Hf[1]), hz(M.Hf[2]), ihx(M.iHf[0]), ihy(M.iHf[1]),
          ihz(M.iHf[2]) {}
};

template <typename T>
__device__ __forceinline__ void corner_weights(T tx, T ty, T tz, T (&w)[8]) {
    const T fx[2] = {T(1) - tx, tx}, fy[2] = {T(1) - ty, ty}, fz[2] = {T(1) - tz, tz};
#pragma unroll
    for (int m = 0; m < 8; ++m) w[m] = fx[m & 1] * fy[(m >> 1) & 1] * fz[(m >> 2) & 1];
}

// A cell-corner total on its way into r_r: a float64 value (FP64 form) or a
// float (mixed forms, whose inputs are float-rounded) that enters r_r as a
// float pair.
struct CellSum64 {
    double v;
    __device__ __forceinline__ double value() const { return v; }
};
struct CellSum32 {
    float h, l;
    __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};
__device__ __forceinline__ CellSum64 one_sum(double v) { return {v}; }
__device__ __forceinline__ CellSum32 one_sum(float v) { return {v, 0.0f}; }

// add a cell total to entry `col` of r_r: float64 atomics, or a float pair
// with the exact rounding error of the high add (two-sum of the returned
// old value) folded into the low word
template <typename C>
__device__ __forceinline__ void pool_add(double* rr, float2*, int col, const C& c, std::false_type) {
    atomicAdd(&rr[col], c.value());
}
__device__ __forceinline__ void pool_add(double*, float2* rr2, int col, const CellSum32& c, std::true_type) {
    float* q = reinterpret_cast<float*>(&rr2[col]);
    const float old = atomicAdd(q, c.h);
    float sum, err;
    two_sum(old, c.h, sum, err);
    atomicAdd(q + 1, __fadd_rn(err, c.l));
}

// trilinear weights of the 8 corners of the cell with packed coordinates pc
// (ci | cj << 10 | ck << 20) at point (x, y, z); returns the cell id
template <typename T>
__device__ __forceinline__ int cell_weights(const BoxGrid<T>& g, int pc, T x, T y, T z, T (&wt)[8]) {
    const int ci = pc & 1023, cj = (pc >> 10) & 1023, ck = pc >> 20;
    corner_weights<T>((x - ci * g.hx) * g.ihx, (y - cj * g.hy) * g.ihy, (z - ck * g.hz) * g.ihz, wt);
    return ci + g.bx * (cj + g.by * ck);
}
__device__ __forceinline__ const double* box_w(const DevMesh& M, double) { return M.vb_w64; }
__device__ __forceinline__ const float* box_w(const DevMesh& M, float) { return M.vb_w32; }

// r_r += J^T W s over the cell-sorted box-list entries: each warp takes a
// range of one cell's entries (v, weight) (<= kBoxRange, a work item holds 8
// ranges), forms w_m(x_v) * weight * s_v for the cell's 8 corners, sums them
// over the warp (reduce-scatter) and adds each corner's total to r_r once.
// kPairOut: r_r is a float pair per entry (compensated float atomics);
// otherwise float64.
__device__ __forceinline__ const double* rent_w(const DevMesh& M, double) { return M.re_w64; }
__device__ __forceinline__ const float* rent_w(const DevMesh& M, float) { return M.re_w32; }

// Reduce-scatter of 8 values over a warp: lane 4m ends with the warp's total
// of value m (lanes exchange halves of their values, then sum over bits 1, 0).
template <typename T>
__device__ __forceinline__ T warp_scatter8(const T (&a)[8], int lane) {
    T v4[4], v2[2];
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        v4[k] = (b4 ? a[k + 4] : a[k]) + __shfl_xor_sync(0xffffffffu, b4 ? a[k] : a[k + 4], 16);
#pragma unroll
    for (int k = 0; k < 2; ++k)
        v2[k] = (b3 ? v4[k + 2] : v4[k]) + __shfl_xor_sync(0xffffffffu, b3 ? v4[k] : v4[k + 2], 8);
    T v1 = (b2 ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? v2[0] : v2[1], 4);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 2);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
    return v1;
}

template <typename T, typename Tin, bool kPairOut>
__device__ __forceinline__ void restrict_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                              const Tin* __restrict__ sin, void* __restrict__ rrv) {
    CGS_ITEM_PROLOGUE();
    const int r = w.begin + (int)(threadIdx.x >> 5);
    if (r >= w.end) return;
    const Tin* s = sin + w.voff;
    const BoxGrid<T> g(M);
    const auto vx = vertex_data(M, T(0));
    const T* rw = rent_w(M, T(0));
    const int lane = threadIdx.x & 31;
    const int2 rg = __ldg(&M.re_rng[r]);
    const int pc = __ldg(&M.re_cell[rg.x]);   // one cell per range
    T acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = T(0);
    for (int i0 = rg.x + lane; i0 < rg.y; i0 += 128) {
        // four entries per lane and round, their loads first
        int v[4];
        T f[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + 32 * k;
            v[k] = i < rg.y ? __ldg(&M.re_vert[i]) : -1;
            f[k] = i < rg.y ? __ldg(&rw[i]) : T(0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (v[k] < 0) continue;
            T x, y, z, ic;
            vx.load(v[k], x, y, z, ic);
            T wt[8];
            cell_weights(g, pc, x, y, z, wt);
            const T fv = f[k] * (T)__ldg(&s[v[k]]);
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] += wt[m] * fv;
        }
    }
    const T tot = warp_scatter8(acc, lane);
    if ((lane & 3) == 0) {
        const int c = (pc & 1023) + g.bx * (((pc >> 10) & 1023) + g.by * (pc >> 20));
        const int col = __ldg(&M.cell_cols[(size_t)c * 8 + (lane >> 2)]);
        if (col >= 0)
            pool_add(static_cast<double*>(rrv) + w.roff, static_cast<float2*>(rrv) + w.roff, col, one_sum(tot),
                     std::integral_constant<bool, kPairOut>());
    }
}

template <typename T, typename Tin, bool kPairOut>
__global__ void __launch_bounds__(kBlock) restrict_kernel(const DevMesh* __restrict__ meshes,
                                                          const Work* __restrict__ work, Vecs V,
                                                          const Tin* __restrict__ sin, void* __restrict__ rrv) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    restrict_item<T, Tin, kPairOut>(meshes, w_, V, sin, rrv);
}

// Restriction of the hybrid step without the residual update (Eq. (5)):
// r_r = J~^T (r - A l) = J~^T r - (A J~)^T l, A symmetric, over explicit
// entries (v, J~_vc, (A J~)_vc) sorted by reduced column c.  One warp per
// range of one column (<= kHybRange entries): each lane takes every 32nd
// entry, four at a time with the loads first, the warp sums, and lane 0 adds
// the total to r_r[c] once.  This replaces the inner operator apply s -= A l
// (one pass over the element matrices) and the restriction of s.
// T = double: float64 entries, r_r float64; T = float (mixed forms): float
// entries and inputs, r_r a float pair (compensated atomic).
__device__ __forceinline__ double2 hr_entry(const DevMesh& M, int i, double) { return __ldg(&M.hr_jg64[i]); }
__device__ __forceinline__ float2 hr_entry(const DevMesh& M, int i, float) { return __ldg(&M.hr_jg32[i]); }

template <typename T>
__device__ __forceinline__ void restrict_hyb_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                  const T* __restrict__ rin, const T* __restrict__ lin,
                                                  void* __restrict__ rrv) {
    CGS_ITEM_PROLOGUE();
    const int q = w.begin + (int)(threadIdx.x >> 5);
    if (q >= w.end) return;   // whole warps leave
    const T* r = rin + w.voff;
    const T* l = lin + w.voff;
    const int lane = threadIdx.x & 31;
    const int4 rg = __ldg(&M.hr_rng[q]);
    using JG = decltype(hr_entry(M, 0, T(0)));
    // software pipeline over rounds of four entries per lane: the entry
    // loads of round k + 1 are issued before the gathers of round k are
    // used, so the two dependent round trips of consecutive rounds overlap
    int v[4];
    JG jg[4];
    auto load_round = [&](int i0, int (&vv)[4], JG (&jj)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + 32 * k;
            vv[k] = i < rg.y ? __ldg(&M.hr_vert[i]) : -1;
            if (i < rg.y) jj[k] = hr_entry(M, i, T(0));
        }
    };
    load_round(rg.x + lane, v, jg);
    T acc = T(0);
    for (int i0 = rg.x + lane; i0 < rg.y; i0 += 128) {
        T rv[4], lv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            rv[k] = v[k] >= 0 ? __ldg(&r[v[k]]) : T(0);
            lv[k] = v[k] >= 0 ? __ldg(&l[v[k]]) : T(0);
        }
        JG cur[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cur[k] = jg[k];
        const bool live[4] = {v[0] >= 0, v[1] >= 0, v[2] >= 0, v[3] >= 0};
        load_round(i0 + 128, v, jg);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!live[k]) continue;
            acc = fma(cur[k].x, rv[k], acc);
            acc = fma(-cur[k].y, lv[k], acc);
        }
    }
    acc = warp_sum_t(acc);
    if (lane == 0)
        pool_add(static_cast<double*>(rrv) + w.roff, static_cast<float2*>(rrv) + w.roff, rg.z, one_sum(acc),
                 std::integral_constant<bool, std::is_same<T, float>::value>());
}

template <typename T>
__global__ void __launch_bounds__(kBlock) restrict_hyb_kernel(const DevMesh* __restrict__ meshes,
                                                              const Work* __restrict__ work, Vecs V,
                                                              const T* __restrict__ rin, const T* __restrict__ lin,
                                                              void* __restrict__ rrv) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    restrict_hyb_item<T>(meshes, w_, V, rin, lin, rrv);
}

// z += J~ u_r by the explicit float64 rows of J~ (FP64 form): one thread per
// row, rows ordered by length (so a warp's rows have the same length) and
// padded to multiples of four entries, read as 16-byte groups; u_r gathered
// from L2.  kDots also forms the PCG dots z.r, z.q and beta (as interp_add).
template <int kDots>
__device__ __forceinline__ void interp_rows_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                 const double* __restrict__ urv, double* __restrict__ zv) {
    CGS_ITEM_PROLOGUE();
    const double* __restrict__ ur = urv + w.roff;
    double* __restrict__ z = zv + w.voff;
    const double* __restrict__ r64 = V.r + w.voff;
    const double* __restrict__ q64 = V.q + w.voff;
    const int4* __restrict__ col4 = reinterpret_cast<const int4*>(M.jt_col);
    const double2* __restrict__ val2 = reinterpret_cast<const double2*>(M.jt_val);
    double zr = 0.0, zq = 0.0;
    for (int i0 = w.begin + (int)threadIdx.x; i0 < w.end; i0 += 2 * (int)blockDim.x) {
        int v[2], g0[2], g1[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = i0 + k * (int)blockDim.x;
            v[k] = -1;
            g0[k] = g1[k] = 0;
            if (i < w.end) {
                v[k] = __ldg(&M.jt_vert[i]);
                g0[k] = __ldg(&M.jt_ptr[i]) >> 2;
                g1[k] = __ldg(&M.jt_ptr[i + 1]) >> 2;
            }
        }
        double zo[2], rd[2], qd[2], val[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const bool ok = v[k] >= 0;
            zo[k] = ok ? z[v[k]] : 0.0;
            rd[k] = (kDots && ok) ? r64[v[k]] : 0.0;
            qd[k] = (kDots && ok) ? q64[v[k]] : 0.0;
            val[k] = 0.0;
        }
        // both rows advance together, one group of four entries each per step
        const int n = max(g1[0] - g0[0], g1[1] - g0[1]);
        for (int t = 0; t < n; ++t) {
            int4 c[2];
            double2 a[2], b[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const bool ok = g0[k] + t < g1[k];
                c[k] = ok ? __ldg(&col4[g0[k] + t]) : make_int4(0, 0, 0, 0);
                a[k] = ok ? __ldg(&val2[2 * (g0[k] + t)]) : make_double2(0.0, 0.0);
                b[k] = ok ? __ldg(&val2[2 * (g0[k] + t) + 1]) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                val[k] = fma(a[k].x, __ldg(&ur[c[k].x]), val[k]);
                val[k] = fma(a[k].y, __ldg(&ur[c[k].y]), val[k]);
                val[k] = fma(b[k].x, __ldg(&ur[c[k].z]), val[k]);
                val[k] = fma(b[k].y, __ldg(&ur[c[k].w]), val[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (v[k] < 0) continue;
            const double zi = zo[k] + val[k];
            z[v[k]] = zi;
            if (kDots) {
                zr = fma(zi, rd[k], zr);
                zq = fma(zi, qd[k], zq);
            }
        }
    }
    if (kDots == 0 || !S) return;
    double val2s[2] = {zr, zq}, tot[2];
    pdl_trigger();   // the successor may launch during the reduction tail
    if (slot_sum<2>(val2s, V.partials + w.poff, w.idx, w.count, &S->ticket[3], tot) && threadIdx.x == 0) {
        S->zr = tot[0];
        S->zq = tot[1];
        const double beta = -S->alpha * tot[1] / S->rho;
        S->beta = beta;
        S->beta2 = split_pair(beta);
        S->rho = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0]) || !isfinite(beta)) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        }
    }
}

template <int kDots>
__global__ void __launch_bounds__(kBlock) interp_rows_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const double* __restrict__ urv,
                                                             double* __restrict__ zv, int nslots,
                                                             cudaGraphConditionalHandle cond, int set_cond) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    if (set_cond && blockIdx.x == 0) loop_condition(V.S, nslots, cond);
    interp_rows_item<kDots>(meshes, w_, V, urv, zv);
}

// z += W Q^T J_L u_r over the cell-sorted box-list entries (the transpose of
// the restriction, the same (vertex, cell, weight) entries): each warp takes
// a range of one cell's entries, holds the cell's 8 values of u_r in
// registers and adds weight * sum_m w_m(x_v) u_r[m] to z_v by an atomic add
// (a vertex in several cells receives one add per cell, in any order).
template <typename T, typename Tu>
__device__ __forceinline__ void interp_cell_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                 const Tu* __restrict__ urv, T* __restrict__ zv) {
    CGS_ITEM_PROLOGUE();
    const int r = w.begin + (int)(threadIdx.x >> 5);
    if (r >= w.end) return;   // whole warps leave
    const Tu* ur = urv + w.roff;
    T* z = zv + w.voff;
    const BoxGrid<T> g(M);
    const auto vx = vertex_data(M, T(0));
    const T* rw = rent_w(M, T(0));
    const int lane = threadIdx.x & 31;
    const int2 rg = __ldg(&M.re_rng[r]);
    const int pc = __ldg(&M.re_cell[rg.x]);   // one cell per range
    const int c = (pc & 1023) + g.bx * (((pc >> 10) & 1023) + g.by * (pc >> 20));
    // corner m's value (0 for an inactive corner), loaded by lane m
    T um = T(0);
    if (lane < 8) {
        const int col = __ldg(&M.cell_cols[(size_t)c * 8 + lane]);
        um = col >= 0 ? (T)__ldg(&ur[col]) : T(0);
    }
    T u[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) u[m] = __shfl_sync(0xffffffffu, um, m);
    for (int i0 = rg.x + lane; i0 < rg.y; i0 += 128) {
        // four entries per lane and round, their loads first
        int v[4];
        T f[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + 32 * k;
            v[k] = i < rg.y ? __ldg(&M.re_vert[i]) : -1;
            f[k] = i < rg.y ? __ldg(&rw[i]) : T(0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (v[k] < 0) continue;
            T x, y, zz, ic;
            vx.load(v[k], x, y, zz, ic);
            T wt[8];
            cell_weights(g, pc, x, y, zz, wt);
            T sum = T(0);
#pragma unroll
            for (int m = 0; m < 8; ++m) sum += wt[m] * u[m];
            atomicAdd(&z[v[k]], f[k] * sum);
        }
    }
}

template <typename T, typename Tu>
__global__ void __launch_bounds__(kBlock) interp_cell_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const Tu* __restrict__ urv, T* __restrict__ zv) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    interp_cell_item<T, Tu>(meshes, w_, V, urv, zv);
}

// z += W Q^T J_L u_r by vertex: z_v += sum_c weight_c sum_m w_m^c(x_v) u_r[m]
// (each box-list vertex once: plain read-modify-write).  kDots fuses the
// PCG dots that follow the preconditioner, z.r and z.q (Dirichlet and
// element-free vertices have z = 0): 1 = float64 vectors, 2 = float-pair r
// and q; the slot's last block forms beta = -alpha (z.q) / rho, rho = z.r.
template <typename T, typename Tu, int kDots>
__device__ __forceinline__ void interp_add_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                const Tu* __restrict__ urv, T* __restrict__ zv) {
    CGS_ITEM_PROLOGUE();
    const Tu* ur = urv + w.roff;
    T* z = zv + w.voff;
    double zr = 0.0, zq = 0.0;
    float rh = 0.0f, rl = 0.0f, qh = 0.0f, ql = 0.0f;
    const BoxGrid<T> g(M);
    const auto vx = vertex_data(M, T(0));
    const T* bw = box_w(M, T(0));
    const float2* __restrict__ r2 = reinterpret_cast<const float2*>(V.r) + w.voff;
    float2* __restrict__ q2 = V.q2 + w.voff;
    const double* __restrict__ r64 = V.r + w.voff;
    const double* __restrict__ q64 = V.q + w.voff;
    // four vertices per thread and round: the list heads and every vertex
    // operand are loaded first, the four sums formed next and all stores
    // issued last, so that no store sits between a round's loads
    for (int64_t i0 = (int64_t)w.begin + threadIdx.x; i0 < w.end; i0 += 4 * (int64_t)blockDim.x) {
        int v[4], e0[4], e1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            v[k] = -1;
            e0[k] = e1[k] = 0;
            if (i < w.end) {
                v[k] = __ldg(&M.vb_vert[i]);
                e0[k] = __ldg(&M.vb_ptr[i]);
                e1[k] = __ldg(&M.vb_ptr[i + 1]);
            }
        }
        T zo[4];
        float2 rk[4], qk[4];
        double rd[4], qd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = v[k] >= 0;
            zo[k] = ok ? z[v[k]] : T(0);
            if (kDots == 2) {
                rk[k] = ok ? r2[v[k]] : make_float2(0.0f, 0.0f);
                qk[k] = ok ? q2[v[k]] : make_float2(0.0f, 0.0f);
            } else if (kDots == 1) {
                rd[k] = ok ? r64[v[k]] : 0.0;
                qd[k] = ok ? q64[v[k]] : 0.0;
            }
        }
        T val[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            val[k] = T(0);
            if (v[k] < 0 || M.nr <= 0) continue;
            T x, y, zz, ic;
            vx.load(v[k], x, y, zz, ic);
            for (int e = e0[k]; e < e1[k]; ++e) {
                T wt[8];
                const int c = cell_weights(g, __ldg(&M.vb_cell[e]), x, y, zz, wt);
                // the cell's 8 active columns in two 16-byte loads
                const int4 ca = __ldg(reinterpret_cast<const int4*>(M.cell_cols) + 2 * (size_t)c);
                const int4 cb = __ldg(reinterpret_cast<const int4*>(M.cell_cols) + 2 * (size_t)c + 1);
                const int col[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
                T sum = T(0);
#pragma unroll
                for (int m = 0; m < 8; ++m) sum += wt[m] * (col[m] >= 0 ? (T)__ldg(&ur[col[m]]) : T(0));
                val[k] += __ldg(&bw[e]) * sum;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (v[k] < 0) continue;
            const T zi = zo[k] + val[k];
            z[v[k]] = zi;
            if (kDots == 1) {
                zr = fma((double)zi, rd[k], zr);
                zq = fma((double)zi, qd[k], zq);
            } else if (kDots == 2) {
                const float2 z2 = make_float2((float)zi, 0.0f);
                pr_dot_acc(rh, rl, z2, rk[k]);
                pr_dot_acc(qh, ql, z2, qk[k]);
                q2[v[k]] = zero_after(qk[k]);   // q = 0 for the next product
            }
        }
    }
    if (kDots == 0 || !S) return;
    double tot[2];
    bool last;
    if (kDots == 2) {
        float vh[2] = {rh, qh}, vl[2] = {rl, ql};
        pdl_trigger();   // the successor may launch during the reduction tail
        last = slot_sum_pair<2>(vh, vl, V.partials + w.poff, w.idx, w.count, &S->ticket[3], tot);
    } else {
        double val2[2] = {zr, zq};
        pdl_trigger();   // the successor may launch during the reduction tail
        last = slot_sum<2>(val2, V.partials + w.poff, w.idx, w.count, &S->ticket[3], tot);
    }
    if (last && threadIdx.x == 0) {
        S->zr = tot[0];
        S->zq = tot[1];
        const double beta = -S->alpha * tot[1] / S->rho;
        S->beta = beta;
        S->beta2 = split_pair(beta);
        S->rho = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0]) || !isfinite(beta)) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        }
    }
}

// three blocks per SM for the float forms, two for float64 (no spills)
template <typename T, typename Tu, int kDots>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 3 : 2) interp_add_kernel(const DevMesh* __restrict__ meshes,
                                                            const Work* __restrict__ work, Vecs V,
                                                            const Tu* __restrict__ urv, T* __restrict__ zv,
                                                            int nslots, cudaGraphConditionalHandle cond,
                                                            int set_cond) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    if (set_cond && blockIdx.x == 0) loop_condition(V.S, nslots, cond);
    interp_add_item<T, Tu, kDots>(meshes, w_, V, urv, zv);
}

// Additive form, mixed precision: the local solves and the restriction
// r_r = J^T W s read the same s and are independent, so one launch does both
// (the restriction fused with the local solve): blocks [0, nl) take
// local-solve items (lane or row packs), the others restriction ranges.
template <typename Stor>
__global__ void __launch_bounds__(kBlock, 2) local_restrict_kernel(const DevMesh* __restrict__ meshes,
                                                                   const Work* __restrict__ wl, unsigned int nl,
                                                                   int row_packs, const Work* __restrict__ wr,
                                                                   Vecs V, const float* __restrict__ s,
                                                                   float* __restrict__ z, void* __restrict__ rr) {
    const bool local = blockIdx.x < nl;
    const Work w_ = local ? wl[blockIdx.x] : wr[blockIdx.x - nl];
    pdl_wait();
    if (!local)
        restrict_item<float, float, true>(meshes, w_, V, s, rr);
    else if (row_packs)
        local_rowpack_item<Stor>(meshes, w_, V, s, z, 0);
    else
        local_lane_item<Stor>(meshes, w_, V, s, z, 0);
}

// sum over entries [e, e1) of val[e] * x[idx[e]] by one warp: each lane
// takes every 32nd entry, eight at a time with all index loads issued first,
// then the values and the gathers (two dependent round trips per eight).
// Float pairs: error-free products, pair accumulation, pair warp sum.
__device__ __forceinline__ void gather_dot_pair(const float2* __restrict__ val, const uint16_t* __restrict__ idx,
                                                const float2* __restrict__ x, int e, int e1, int lane, float& h,
                                                float& l) {
    h = 0.0f;
    l = 0.0f;
    for (int e0 = e + lane; e0 < e1; e0 += 256) {
        int j[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) j[k] = e0 + 32 * k < e1 ? (int)__ldg(&idx[e0 + 32 * k]) : -1;
        float2 a[8], b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a[k] = j[k] >= 0 ? __ldg(&val[e0 + 32 * k]) : make_float2(0.0f, 0.0f);
            b[k] = j[k] >= 0 ? __ldg(&x[j[k]]) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float ph, pl;
            pair_mul(a[k].x, a[k].y, b[k].x, b[k].y, ph, pl);
            pair_acc(h, l, ph, pl);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        pair_acc(h, l, oh, ol);
    }
}
__device__ __forceinline__ double gather_dot64(const double* __restrict__ val, const uint16_t* __restrict__ idx,
                                               const double* __restrict__ x, int e, int e1, int lane) {
    double s = 0.0;
    for (int e0 = e + lane; e0 < e1; e0 += 256) {
        int j[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) j[k] = e0 + 32 * k < e1 ? (int)__ldg(&idx[e0 + 32 * k]) : -1;
        double a[8], b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a[k] = j[k] >= 0 ? __ldg(&val[e0 + 32 * k]) : 0.0;
            b[k] = j[k] >= 0 ? __ldg(&x[j[k]]) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s = fma(a[k], b[k], s);
    }
    return warp_sum(s);
}

// u_r = A_r^{-1} r_r: one warp per row of the full symmetric inverse; also a
// float copy of u_r for the float interpolation (no conversions per element).
__device__ __forceinline__ void coarse_gemv_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                 const double* __restrict__ rrv, double* __restrict__ urv,
                                                 float* __restrict__ ur32v) {
    CGS_ITEM_PROLOGUE();
    const int64_t nr = M.nr;
    const double* rr = rrv + w.roff;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)w.begin + (threadIdx.x >> 5);
    if (i >= w.end) return;
    if (M.xxt) {   // second XX^T pass: u_i = sum_k X_ik t_k
        const double s = gather_dot64(static_cast<const double*>(M.xr_val), M.xr_idx, V.rt + w.roff,
                                      __ldg(&M.xr_ptr[i]), __ldg(&M.xr_ptr[i + 1]), lane);
        if (lane == 0) {
            urv[w.roff + i] = s;
            if (ur32v) ur32v[w.roff + i] = (float)s;
        }
        return;
    }
    const double* row = M.ar_inv + (size_t)i * nr;
    double s = 0.0;
    for (int64_t j = lane; j < nr; j += 32) s = fma(__ldg(&row[j]), __ldg(&rr[j]), s);
    s = warp_sum(s);
    if (lane == 0) {
        urv[w.roff + i] = s;
        if (ur32v) ur32v[w.roff + i] = (float)s;
    }
}
__global__ void __launch_bounds__(kBlock) coarse_gemv_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const double* __restrict__ rrv,
                                                             double* __restrict__ urv, float* __restrict__ ur32v) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    coarse_gemv_item(meshes, w_, V, rrv, urv, ur32v);
}

// u_r = A_r^{-1} r_r in float-pair arithmetic (mixed forms): the inverse and
// r_r are hi/lo float pairs, every lane keeps a pair accumulator, the warp
// sums pairs by shuffles.  Same ~48-bit accuracy as the float64 product on
// the FP32 pipes, so the product runs at the bandwidth of the 8-byte entries.
// Writes u_r as float64 (ur, optional) and rounded to float (ur32, optional).
__device__ __forceinline__ void coarse_pair_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                 const float2* __restrict__ rr2v, double* __restrict__ urv,
                                                 float* __restrict__ ur32v) {
    CGS_ITEM_PROLOGUE();
    const int64_t nr = M.nr;
    const float2* rr = rr2v + w.roff;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)w.begin + (threadIdx.x >> 5);
    if (i >= w.end) return;
    if (M.xxt) {   // second XX^T pass: u_i = sum_k X_ik t_k, in float pairs
        float h, l;
        gather_dot_pair(static_cast<const float2*>(M.xr_val), M.xr_idx, reinterpret_cast<const float2*>(V.rt) + w.roff,
                        __ldg(&M.xr_ptr[i]), __ldg(&M.xr_ptr[i + 1]), lane, h, l);
        if (lane == 0) {
            if (urv) urv[w.roff + i] = (double)h + (double)l;
            if (ur32v) ur32v[w.roff + i] = __fadd_rn(h, l);
        }
        return;
    }
    // the row as 16-byte groups of two entries; four groups per lane in flight
    const float4* row = reinterpret_cast<const float4*>(M.ar_inv2 + (size_t)i * M.nr2);
    const int64_t ng = M.nr2 / 2;
    float h = 0.0f, l = 0.0f, h2 = 0.0f, l2 = 0.0f;
    for (int64_t g0 = lane; g0 < ng; g0 += 128) {
        float4 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t g = g0 + 32 * k;
            a[k] = g < ng ? ld_stream(row + g) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t j = 2 * (g0 + 32 * k);
            if (j >= nr) continue;
            const float2 r0 = __ldg(&rr[j]);
            const float2 r1 = j + 1 < nr ? __ldg(&rr[j + 1]) : make_float2(0.0f, 0.0f);
            float ph, pl;
            pair_mul(a[k].x, a[k].y, r0.x, r0.y, ph, pl);
            pair_acc(h, l, ph, pl);
            pair_mul(a[k].z, a[k].w, r1.x, r1.y, ph, pl);
            pair_acc(h2, l2, ph, pl);
        }
    }
    pair_acc(h, l, h2, l2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        pair_acc(h, l, oh, ol);
    }
    if (lane == 0) {
        if (urv) urv[w.roff + i] = (double)h + (double)l;
        if (ur32v) ur32v[w.roff + i] = __fadd_rn(h, l);
    }
}
__global__ void __launch_bounds__(kBlock) coarse_pair_kernel(const DevMesh* __restrict__ meshes,
                                                             const Work* __restrict__ work, Vecs V,
                                                             const float2* __restrict__ rr2v,
                                                             double* __restrict__ urv, float* __restrict__ ur32v) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    coarse_pair_item(meshes, w_, V, rr2v, urv, ur32v);
}

// First XX^T pass (Sec. 2): t = X^T r_r.  One warp per segment of at most
// kXxtSeg entries of one column x_k of X (long columns are split); the
// segment's partial dot product x_k . r_r is added to t_k, which is zero on
// entry: a float64 atomic (FP64 form), or, in the mixed forms, float pairs
// whose high add's exact rounding error goes into the low word.
template <bool kPair>
__device__ __forceinline__ void xxt_seg_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                             const double* __restrict__ rrv) {
    CGS_ITEM_PROLOGUE();
    const int64_t sidx = (int64_t)w.begin + (threadIdx.x >> 5);
    if (sidx >= w.end) return;   // whole warps leave
    const int lane = threadIdx.x & 31;
    const int4 sg = __ldg(&M.xs_seg[sidx]);   // column, begin, end
    if (kPair) {
        float h, l;
        gather_dot_pair(static_cast<const float2*>(M.xc_val), M.xc_idx,
                        reinterpret_cast<const float2*>(rrv) + w.roff, sg.y, sg.z, lane, h, l);
        if (lane == 0) {
            float* t = reinterpret_cast<float*>(reinterpret_cast<float2*>(V.rt) + w.roff + sg.x);
            const float old = atomicAdd(t, h);
            float sum, err;
            two_sum(old, h, sum, err);
            atomicAdd(t + 1, __fadd_rn(err, l));
        }
    } else {
        const double acc = gather_dot64(static_cast<const double*>(M.xc_val), M.xc_idx, rrv + w.roff, sg.y, sg.z, lane);
        if (lane == 0) atomicAdd(&V.rt[w.roff + sg.x], acc);
    }
}
template <bool kPair>
__global__ void __launch_bounds__(32 * kRowChunk) xxt_seg_kernel(const DevMesh* __restrict__ meshes,
                                                                 const Work* __restrict__ work, Vecs V,
                                                                 const double* __restrict__ rrv) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    xxt_seg_item<kPair>(meshes, w_, V, rrv);
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

#define CGS_VERT_LOOP(i) for (int64_t i = (int64_t)w.begin + threadIdx.x; i < w.end; i += blockDim.x)
// four vertices per thread and round: i0, i0 + blockDim, ... (loads first)
#define CGS_VERT_LOOP4(i0) \
    for (int64_t i0 = (int64_t)w.begin + threadIdx.x; i0 < w.end; i0 += 4 * (int64_t)blockDim.x)

// r = b with Dirichlet entries zeroed, x = 0, q = 0; ||b||^2 -> bnorm2, tol2.
template <typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_init_kernel(const DevMesh* __restrict__ meshes,
                                                          const Work* __restrict__ work, Vecs V, Tq* qv,
                                                          double rtol, int maxit) {
    const Work w = work[blockIdx.x];
    pdl_wait();
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
    pdl_trigger();   // the successor may launch during the reduction tail
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
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        V.rr[w.roff + i] = 0.0;
        if (M.xxt) V.rt[w.roff + i] = 0.0;   // t = X^T r_r accumulates by segments
    }
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
    pdl_trigger();   // the successor may launch during the reduction tail
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
__device__ __forceinline__ void pcg_update_xr_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                   const Tq* __restrict__ qv) {
    CGS_ITEM_PROLOGUE();
    double* x = V.x + w.voff;
    double* r = V.r + w.voff;
    const double* p = V.p + w.voff;
    const Tq* q = qv + w.voff;
    Tz* z = static_cast<Tz*>(V.z) + w.voff;
    Tz* s = static_cast<Tz*>(V.s) + w.voff;
    const double alpha = S->alpha;
    // s is r itself when the preconditioner only reads its input
    const bool copy_s = (const void*)s != (const void*)r;
    double acc = 0.0;
    // four vertices per thread and round, every load issued before the stores
    CGS_VERT_LOOP4(i0) {
        double xi[4], pi[4], ri[4], qi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) {
                xi[k] = x[i];
                pi[k] = p[i];
                ri[k] = r[i];
                qi[k] = qval(q, i);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) {
                x[i] = fma(alpha, pi[k], xi[k]);
                const double rn = fma(-alpha, qi[k], ri[k]);
                r[i] = rn;
                acc = fma(rn, rn, acc);
                z[i] = Tz(0);
                if (copy_s) s[i] = (Tz)rn;
            }
        }
    }
    const int64_t chunk = (M.nr + w.count - 1) / w.count;
    const int64_t r0 = (int64_t)w.idx * chunk, r1 = min((int64_t)M.nr, r0 + chunk);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        V.rr[w.roff + i] = 0.0;
        if (M.xxt) V.rt[w.roff + i] = 0.0;   // t = X^T r_r accumulates by segments
    }
    double val[1] = {acc}, tot[1];
    pdl_trigger();   // the successor may launch during the reduction tail
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

template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock, 3) pcg_update_xr_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V,
                                                               const Tq* __restrict__ qv) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    pcg_update_xr_item<Tz, Tq>(meshes, w_, V, qv);
}

// z.r and z.q; beta = -alpha (z.q) / rho (Polak-Ribiere, since
// r_new - r_old = -alpha q), rho = z.r.
template <typename Tz, typename Tq>
__device__ __forceinline__ void pcg_dots_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                              const Tq* __restrict__ qv) {
    CGS_ITEM_PROLOGUE();
    const Tz* z = static_cast<const Tz*>(V.z) + w.voff;
    const double* r = V.r + w.voff;
    const Tq* q = qv + w.voff;
    double zr = 0.0, zq = 0.0;
    CGS_VERT_LOOP(i) {
        const double zi = (double)z[i];
        zr = fma(zi, r[i], zr);
        zq = fma(zi, qval(q, i), zq);
    }
    if (!S) return;   // no slot scalars (timing runs): no reduction
    double val[2] = {zr, zq}, tot[2];
    pdl_trigger();   // the successor may launch during the reduction tail
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

template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock) pcg_dots_kernel(const DevMesh* __restrict__ meshes,
                                                          const Work* __restrict__ work, Vecs V,
                                                          const Tq* __restrict__ qv) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    pcg_dots_item<Tz, Tq>(meshes, w_, V, qv);
}

// p = z + beta p (and p2), q = 0 for the next product.
template <typename Tz, typename Tq>
__device__ __forceinline__ void pcg_update_p_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V, Tq* qv) {
    CGS_ITEM_PROLOGUE();
    const Tz* z = static_cast<const Tz*>(V.z) + w.voff;
    double* p = V.p + w.voff;
    float2* p2 = V.p2 ? V.p2 + w.voff : nullptr;
    Tq* q = qv + w.voff;
    const double beta = S->beta;
    CGS_VERT_LOOP4(i0) {
        double pk[4], zk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) {
                pk[k] = p[i];
                zk[k] = (double)z[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) {
                const double pi = fma(beta, pk[k], zk[k]);
                p[i] = pi;
                if (p2) p2[i] = split_pair(pi);
                qzero(q, i);
            }
        }
    }
}


template <typename Tz, typename Tq>
__global__ void __launch_bounds__(kBlock, 4) pcg_update_p_kernel(const DevMesh* __restrict__ meshes,
                                                              const Work* __restrict__ work, Vecs V, Tq* qv,
                                                              int nslots, cudaGraphConditionalHandle cond,
                                                              int set_cond) {
    if (set_cond && blockIdx.x == 0) loop_condition(V.S, nslots, cond);
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    pcg_update_p_item<Tz, Tq>(meshes, w_, V, qv);
}

// ---------------------------------------------------------------------------
// Outer iteration of the mixed forms in float-pair arithmetic.  x, r, p and
// q = A p are hi/lo float pairs (~48 significant bits); the products and sums
// run on the FP32 pipes, each thread keeps pair accumulators for its dot
// products and converts them to float64 once, and the per-slot reduction of
// those partials is float64.  B300 issues FP64 (and float<->double
// conversions) at 1/60 of its FP32 rate, which made the float64 form of these
// kernels FP64-bound at a fraction of the memory bandwidth.
// ---------------------------------------------------------------------------

// r = b with Dirichlet entries zeroed, x = 0, q = 0; ||b||^2 -> bnorm2, tol2.
__global__ void __launch_bounds__(kBlock) pcg_init_pair_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V, double rtol,
                                                               int maxit) {
    const Work w = work[blockIdx.x];
    pdl_wait();
    SolveScalars* S = V.S + w.slot;
    const DevMesh& M = meshes[w.mesh];
    const double* b = V.bptr ? V.bptr[w.slot] : V.b + w.voff;
    float2* x = as_pair(V.x) + w.voff;
    float2* r = as_pair(V.r) + w.voff;
    float2* q = V.q2 + w.voff;
    double acc = 0.0;
    CGS_VERT_LOOP(i) {
        const double bi = M.dir[i] ? 0.0 : b[i];
        r[i] = split_pair(bi);
        x[i] = make_float2(0.0f, 0.0f);
        q[i] = make_float2(0.0f, 0.0f);
        acc = fma(bi, bi, acc);
    }
    double val[1] = {acc}, tot[1];
    pdl_trigger();   // the successor may launch during the reduction tail
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

// z = 0, s = hi(r) (the float rounding of r), r_r = 0.
__global__ void __launch_bounds__(kBlock) precond_prep_pair_kernel(const DevMesh* __restrict__ meshes,
                                                                   const Work* __restrict__ work, Vecs V) {
    CGS_WORK_PROLOGUE();
    const float2* r = as_pair(V.r) + w.voff;
    float* z = static_cast<float*>(V.z) + w.voff;
    float* s = static_cast<float*>(V.s) + w.voff;
    CGS_VERT_LOOP(i) {
        z[i] = 0.0f;
        s[i] = r[i].x;
    }
    const int64_t chunk = (M.nr + w.count - 1) / w.count;
    const int64_t r0 = (int64_t)w.idx * chunk, r1 = min((int64_t)M.nr, r0 + chunk);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        V.rr[w.roff + i] = 0.0;
        if (M.xxt) V.rt[w.roff + i] = 0.0;   // t = X^T r_r accumulates by segments
    }
}

// p = z, rho = r.z.
__global__ void __launch_bounds__(kBlock) pcg_first_dir_pair_kernel(const DevMesh* __restrict__ meshes,
                                                                    const Work* __restrict__ work, Vecs V) {
    CGS_WORK_PROLOGUE();
    const float* z = static_cast<const float*>(V.z) + w.voff;
    const float2* r = as_pair(V.r) + w.voff;
    float2* p = V.p2 + w.voff;
    float h = 0.0f, l = 0.0f;
    CGS_VERT_LOOP(i) {
        const float2 zi = make_float2(z[i], 0.0f);
        p[i] = zi;
        pr_dot_acc(h, l, zi, r[i]);
    }
    float vh[1] = {h}, vl[1] = {l};
    double tot[1];
    pdl_trigger();   // the successor may launch during the reduction tail
    if (slot_sum_pair<1>(vh, vl, V.partials + w.poff, w.idx, w.count, &S->ticket[1], tot) && threadIdx.x == 0) {
        S->rho = tot[0];
        S->beta = 0.0;   // the first iteration's direction z + beta p is z
        S->beta2 = make_float2(0.0f, 0.0f);
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        }
    }
}

// x += alpha p, r -= alpha q, ||r||^2; z = 0, s = hi(r), r_r = 0.  The
// slot's last block counts the iteration and applies the stopping test.
// form_p: p = z + beta p is formed here and stored (the tiled apply formed
// it on the fly); otherwise p is current already (the row apply needs it
// stored before the apply, so the p update ends the previous iteration).
__device__ __forceinline__ void pcg_update_xr_pair_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V,
                                                        bool form_p = true) {
    CGS_ITEM_PROLOGUE();
    float2* __restrict__ x = as_pair(V.x) + w.voff;
    float2* __restrict__ r = as_pair(V.r) + w.voff;
    float2* __restrict__ p = V.p2 + w.voff;
    const float2* __restrict__ q = V.q2 + w.voff;
    float* __restrict__ z = static_cast<float*>(V.z) + w.voff;
    float* __restrict__ s = static_cast<float*>(V.s) + w.voff;
    const float2 a = S->alpha2, na = make_float2(-a.x, -a.y), beta = S->beta2;
    float h = 0.0f, l = 0.0f;
    for (int64_t i0 = (int64_t)w.begin + threadIdx.x; i0 < w.end; i0 += 2 * (int64_t)blockDim.x) {
        // the loads of two vertices are issued before their arithmetic
        float2 pi[2], qi[2], xi[2], ri[2];
        float zi[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) {
                pi[k] = p[i];
                zi[k] = z[i];
                qi[k] = q[i];
                xi[k] = x[i];
                ri[k] = r[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) {
                // p = z + beta p: the same arithmetic as the operator apply's
                const float2 pn = form_p ? pr_fma(beta, pi[k], make_float2(zi[k], 0.0f)) : pi[k];
                if (form_p) p[i] = pn;
                x[i] = pr_fma(a, pn, xi[k]);
                const float2 rn = pr_fma(na, qi[k], ri[k]);
                r[i] = rn;
                pr_dot_acc(h, l, rn, rn);
                z[i] = zero_after(zi[k]);
                s[i] = rn.x;
            }
        }
    }
    const int64_t chunk = (M.nr + w.count - 1) / w.count;
    const int64_t r0 = (int64_t)w.idx * chunk, r1 = min((int64_t)M.nr, r0 + chunk);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        V.rr[w.roff + i] = 0.0;
        if (M.xxt) V.rt[w.roff + i] = 0.0;   // t = X^T r_r accumulates by segments
    }
    float vh[1] = {h}, vl[1] = {l};
    double tot[1];
    pdl_trigger();   // the successor may launch during the reduction tail
    if (slot_sum_pair<1>(vh, vl, V.partials + w.poff, w.idx, w.count, &S->ticket[2], tot) && threadIdx.x == 0) {
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
__global__ void __launch_bounds__(kBlock, 4) pcg_update_xr_pair_kernel(const DevMesh* __restrict__ meshes,
                                                                    const Work* __restrict__ work, Vecs V,
                                                                    int form_p) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    pcg_update_xr_pair_item(meshes, w_, V, form_p != 0);
}

// p = z + beta p in float pairs (the row apply's direction), ending the
// iteration: block 0 also sets the loop condition.
__device__ __forceinline__ void pcg_update_p_pair_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V) {
    CGS_ITEM_PROLOGUE();
    float2* __restrict__ p = V.p2 + w.voff;
    const float* __restrict__ z = static_cast<const float*>(V.z) + w.voff;
    const float2 beta = S->beta2;
    CGS_VERT_LOOP4(i0) {
        float2 pk[4];
        float zk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) {
                pk[k] = p[i];
                zk[k] = z[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) p[i] = pr_fma(beta, pk[k], make_float2(zk[k], 0.0f));
        }
    }
}
__global__ void __launch_bounds__(kBlock, 4) pcg_update_p_pair_kernel(const DevMesh* __restrict__ meshes,
                                                                   const Work* __restrict__ work, Vecs V, int nslots,
                                                                   cudaGraphConditionalHandle cond, int set_cond) {
    if (set_cond && blockIdx.x == 0) loop_condition(V.S, nslots, cond);
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    pcg_update_p_pair_item(meshes, w_, V);
}

// z.r and z.q; beta = -alpha (z.q) / rho, rho = z.r.
__device__ __forceinline__ void pcg_dots_pair_item(const DevMesh* __restrict__ meshes, const Work& w, Vecs V) {
    CGS_ITEM_PROLOGUE();
    const float* __restrict__ z = static_cast<const float*>(V.z) + w.voff;
    const float2* __restrict__ r = as_pair(V.r) + w.voff;
    float2* __restrict__ q = V.q2 + w.voff;
    float rh = 0.0f, rl = 0.0f, qh = 0.0f, ql = 0.0f;
    CGS_VERT_LOOP4(i0) {
        // a round's loads, then its arithmetic, then its stores
        float zi[4];
        float2 ri[4], qi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            zi[k] = 0.0f;
            ri[k] = qi[k] = make_float2(0.0f, 0.0f);
            if (i < w.end) {
                zi[k] = z[i];
                ri[k] = r[i];
                qi[k] = q[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 z2 = make_float2(zi[k], 0.0f);
            pr_dot_acc(rh, rl, z2, ri[k]);
            pr_dot_acc(qh, ql, z2, qi[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * (int64_t)blockDim.x;
            if (i < w.end) q[i] = zero_after(qi[k]);   // q = 0 for the next product
        }
    }
    if (!S) return;   // no slot scalars (timing runs): no reduction
    float vh[2] = {rh, qh}, vl[2] = {rl, ql};
    double tot[2];
    pdl_trigger();   // the successor may launch during the reduction tail
    if (slot_sum_pair<2>(vh, vl, V.partials + w.poff, w.idx, w.count, &S->ticket[3], tot) && threadIdx.x == 0) {
        S->zr = tot[0];
        S->zq = tot[1];
        const double beta = -S->alpha * tot[1] / S->rho;
        S->beta = beta;
        S->beta2 = split_pair(beta);
        S->rho = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0]) || !isfinite(beta)) {
            S->status = CGS_ERR_BREAKDOWN;
            S->done = 1;
        }
    }
}
__global__ void __launch_bounds__(kBlock) pcg_dots_pair_kernel(const DevMesh* __restrict__ meshes,
                                                               const Work* __restrict__ work, Vecs V, int nslots,
                                                               cudaGraphConditionalHandle cond, int set_cond) {
    const Work w_ = work[blockIdx.x];
    pdl_wait();
    if (set_cond && blockIdx.x == 0) loop_condition(V.S, nslots, cond);
    pcg_dots_pair_item(meshes, w_, V);
}


// x (float pair) -> float64 in place, before the final residual.
__global__ void __launch_bounds__(kBlock) finalize_x_pair_kernel(const DevMesh* __restrict__ meshes,
                                                                 const Work* __restrict__ work, Vecs V) {
    const Work w = work[blockIdx.x];
    pdl_wait();
    double* x = V.x + w.voff;
    CGS_VERT_LOOP(i) {
        const float2 t = as_pair(x)[i];
        x[i] = (double)t.x + (double)t.y;
    }
}


// ---------------------------------------------------------------------------
// Persistent PCG loop of the mixed forms: one cooperative launch runs whole
// iterations, every block walking each phase's work items (the same
// per-item functions as the one-kernel-per-phase path) with a grid barrier
// between phases.  For problems too small to fill the GPU per kernel, this
// trades ~8 kernel launches and their ramp-up and drain per iteration for 8
// barriers.  The barrier waits are bounded: a block that gives up records
// the failure and every block leaves at its next barrier.
// ---------------------------------------------------------------------------
__device__ bool grid_sync(GridBar* b, int limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int g = *(volatile unsigned int*)&b->gen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
            b->count = 0u;
            __threadfence();
            atomicAdd(&b->gen, 1u);
            ok = 1;
        } else {
            int i = 0;
            while (*(volatile unsigned int*)&b->gen == g && i < limit) {
                __nanosleep(64);
                ++i;
            }
            ok = i < limit;
            if (!ok) atomicExch(&b->error, 1);
        }
        __threadfence();
        if (*(volatile int*)&b->error) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// Work tables of the persistent loop, by value.
struct LoopTables {
    const Work* w[kWorkKinds];
    unsigned int n[kWorkKinds];
};
#define CGS_FOR_ITEMS(kind, k) for (unsigned int k = blockIdx.x; k < T.n[kind]; k += gridDim.x)

// A barrier wait gave up: stop every slot with CGS_ERR_TIMEOUT (idempotent,
// any block may do it) and leave.
__device__ void abort_slots(SolveScalars* S, int nslots) {
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        S[i].status = CGS_ERR_TIMEOUT;
        S[i].done = 1;
    }
}
#define CGS_SYNC_OR_LEAVE()                \
    if (!grid_sync(bar, bar_limit)) {      \
        abort_slots(V.S, nslots);          \
        return;                            \
    }

// kBig: some mesh has packs above 32 dofs, run here too (a lane then holds
// up to 2 x 64 floats, so one block per SM)
template <typename Stor, bool kBig>
__global__ void __launch_bounds__(kBlock, kBig ? 1 : 2) pcg_persistent_kernel(const DevMesh* __restrict__ meshes, LoopTables T,
                                                                   Vecs V, GridBar* bar, int nslots, int hybrid,
                                                                   int any_nr, int big_subs, int max_iters,
                                                                   int wait_limit, int bar_limit) {
    float* s = static_cast<float*>(V.s);
    float* z = static_cast<float*>(V.z);
    for (int it = 0; it < max_iters; ++it) {
        // q = A p, p.q and alpha
        CGS_FOR_ITEMS(kWorkTile, k) apply_pair_tiled_item<false>(meshes, T.w[kWorkTile][k], V, wait_limit);
        CGS_SYNC_OR_LEAVE();
        // x, r, ||r||, stopping test; z = 0, s = hi(r), r_r = 0
        CGS_FOR_ITEMS(kWorkVert, k) pcg_update_xr_pair_item(meshes, T.w[kWorkVert][k], V, true);
        CGS_SYNC_OR_LEAVE();
        int running = 0;
        for (int i = threadIdx.x; i < nslots; i += blockDim.x) running |= !*(volatile const int*)&V.S[i].done;
        if (!__syncthreads_or(running)) return;
        // z = M r
        CGS_FOR_ITEMS(kWorkPack, k) local_lane_item<Stor>(meshes, T.w[kWorkPack][k], V, s, z, hybrid);
        CGS_FOR_ITEMS(kWorkRowPack, k) local_rowpack_item<Stor>(meshes, T.w[kWorkRowPack][k], V, s, z, hybrid);
        if (kBig) {
            CGS_FOR_ITEMS(kWorkPack, k) local_lane_item<Stor, true>(meshes, T.w[kWorkPack][k], V, s, z, hybrid);
            CGS_FOR_ITEMS(kWorkRowPack, k)
                local_rowpack_item<Stor, true>(meshes, T.w[kWorkRowPack][k], V, s, z, hybrid);
        }
        CGS_FOR_ITEMS(kWorkSub, k) local_warp_item<float, Stor>(meshes, T.w[kWorkSub][k], V, s, z, hybrid);
        if (big_subs)
            CGS_FOR_ITEMS(kWorkSub, k) local_block_item<float, Stor>(meshes, T.w[kWorkSub][k], V, s, z, hybrid);
        CGS_SYNC_OR_LEAVE();
        if (hybrid) {
            CGS_FOR_ITEMS(kWorkTile, k)
                apply28f_tiled_item<false>(meshes, T.w[kWorkTile][k], V, z, s, -1.0f, wait_limit);
            CGS_SYNC_OR_LEAVE();
        }
        if (any_nr) {
            CGS_FOR_ITEMS(kWorkBoxEnt, k) restrict_item<float, float, true>(meshes, T.w[kWorkBoxEnt][k], V, s, V.rr);
            CGS_SYNC_OR_LEAVE();
            CGS_FOR_ITEMS(kWorkRow, k)
                coarse_pair_item(meshes, T.w[kWorkRow][k], V, reinterpret_cast<const float2*>(V.rr), nullptr, V.ur32);
            CGS_SYNC_OR_LEAVE();
            // z += J u_r with the dots z.r, z.q and beta
            CGS_FOR_ITEMS(kWorkBox, k) interp_add_item<float, float, 2>(meshes, T.w[kWorkBox][k], V, V.ur32, z);
        } else {
            CGS_FOR_ITEMS(kWorkVert, k) pcg_dots_pair_item(meshes, T.w[kWorkVert][k], V);
        }
        CGS_SYNC_OR_LEAVE();
        // (p = z + beta p is formed by the next operator apply and stored by
        // the next x, r update)
    }
}
#undef CGS_FOR_ITEMS
#undef CGS_SYNC_OR_LEAVE

// x_out = x (copy-out), then ||b - y||^2 and ||b||^2 over free entries.
__global__ void __launch_bounds__(kBlock) resid_norm_kernel(const DevMesh* __restrict__ meshes,
                                                            const Work* __restrict__ work, Vecs V) {
    const Work w = work[blockIdx.x];
    pdl_wait();
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
    pdl_trigger();   // the successor may launch during the reduction tail
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
    pdl_wait();
    const DevMesh& M = meshes[w.mesh];
    CGS_VERT_LOOP(i) b[w.voff + i] = (mask_dirichlet && M.dir[i]) ? Tb(0) : (Tb)a[w.voff + i];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) fill_kernel(int64_t n, T* __restrict__ a, T v) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

}  // namespace

// Launch `kern` with programmatic stream serialization when `pdl` is set
// (the kernel may start while its predecessor in the stream runs; it waits in
// pdl_wait before reading upstream data).  Empty grids launch nothing.
template <typename... KArgs, typename... Args>
void launch_pdl(bool pdl, void (*kern)(KArgs...), unsigned int grid, unsigned int block, size_t smem,
                cudaStream_t st, Args... args) {
    if (grid == 0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Launchers.  A Plan names the mesh descriptors and the work tables of one
// set of slots (one mesh with one right-hand side, or a batch).
// ---------------------------------------------------------------------------

void launch_apply64(const Plan& P, const Vecs& V, const double* x, double* y, double alpha, bool dot,
                    cudaStream_t st) {
    if (P.ell) {   // the assembled rows
        if (!P.nwork[kWorkEll]) return;
        if (dot)
            launch_pdl(P.pdl, apply_ell64_kernel<true>, P.nwork[kWorkEll], kBlock, 0, st, P.meshes, P.work[kWorkEll],
                       V, x, y, alpha);
        else
            launch_pdl(P.pdl, apply_ell64_kernel<false>, P.nwork[kWorkEll], kBlock, 0, st, P.meshes, P.work[kWorkEll],
                       V, x, y, alpha);
        return;
    }
    if (!P.nwork[kWorkElem]) return;
    if (dot)
        launch_pdl(P.pdl, apply64_kernel<true>, P.nwork[kWorkElem], kBlock, 0, st, P.meshes, P.work[kWorkElem], V, x, y,
                   alpha);
    else
        launch_pdl(P.pdl, apply64_kernel<false>, P.nwork[kWorkElem], kBlock, 0, st, P.meshes, P.work[kWorkElem], V, x,
                   y, alpha);
}

template <bool kTma>
void set_smem_attr(const void* fn, int bytes, bool& done) {
    if (!done) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        done = true;
    }
}

bool rows_outer(const Plan& P) { return P.ell_pair && !P.tile_tma && P.nwork[kWorkEll] > 0; }

void launch_apply_outer(const Plan& P, const Vecs& V, cudaStream_t st) {
    if (rows_outer(P))
        launch_pdl(P.pdl, apply_ell_pair_kernel, P.nwork[kWorkEll], kBlock, 0, st, P.meshes, P.work[kWorkEll], V);
    else
        launch_apply_pair_tiled(P, V, st);
}

void launch_apply_pair_tiled(const Plan& P, const Vecs& V, cudaStream_t st) {
    if (!P.nwork[kWorkTile]) return;
    const int verts = (int)(2 * kTileVerts * sizeof(float2));
    if (P.tile_tma) {
        static bool attr = false;
        const int smem = verts + (int)(2 * kTileSlotBytes);
        set_smem_attr<true>((const void*)apply_pair_tiled_kernel<true>, smem, attr);
        launch_pdl(P.pdl, apply_pair_tiled_kernel<true>, P.nwork[kWorkTile], kBlock, smem, st, P.meshes,
                   P.work[kWorkTile], V, P.wait_limit);
    } else {
        launch_pdl(P.pdl, apply_pair_tiled_kernel<false>, P.nwork[kWorkTile], kBlock, verts, st, P.meshes,
                   P.work[kWorkTile], V, P.wait_limit);
    }
}

void launch_apply28f_tiled(const Plan& P, const Vecs& V, const float* x, float* y, float alpha, cudaStream_t st) {
    if (!P.nwork[kWorkTile]) return;
    const int verts = (int)(2 * kTileVerts * sizeof(float));
    if (P.tile_tma) {
        static bool attr = false;
        const int smem = verts + (int)kTileSlotBytes;
        set_smem_attr<true>((const void*)apply28f_tiled_kernel<true>, smem, attr);
        launch_pdl(P.pdl, apply28f_tiled_kernel<true>, P.nwork[kWorkTile], kBlock, smem, st, P.meshes,
                   P.work[kWorkTile], V, x, y, alpha, P.wait_limit);
    } else {
        launch_pdl(P.pdl, apply28f_tiled_kernel<false>, P.nwork[kWorkTile], kBlock, verts, st, P.meshes,
                   P.work[kWorkTile], V, x, y, alpha, P.wait_limit);
    }
}

void launch_local(const Plan& P, const Vecs& V, cgs_precision prec, const void* r, void* out, int weighted,
                  cudaStream_t st) {
    const int wt = weighted;
    // mixed forms: subdomains of at most kLaneMaxMixed dofs in lane packs, or
    // in row packs (small meshes); the classes above 32 dofs in kernels of
    // their own
    if (prec != CGS_FP64 && P.nwork[kWorkRowPack]) {
        const float* rf = static_cast<const float*>(r);
        float* of = static_cast<float*>(out);
        if (prec == CGS_FP32_BULK)
            launch_pdl(P.pdl, local_rowpack_kernel<float>, P.nwork[kWorkRowPack], kBlock, 0, st, P.meshes,
                       P.work[kWorkRowPack], V, rf, of, wt);
        else
            launch_pdl(P.pdl, local_rowpack_kernel<__half>, P.nwork[kWorkRowPack], kBlock, 0, st, P.meshes,
                       P.work[kWorkRowPack], V, rf, of, wt);
        if (P.lane_big) {
            if (prec == CGS_FP32_BULK)
                launch_pdl(P.pdl, local_rowpack_big_kernel<float>, P.nwork[kWorkRowPack], kBlock, 0, st, P.meshes,
                           P.work[kWorkRowPack], V, rf, of, wt);
            else
                launch_pdl(P.pdl, local_rowpack_big_kernel<__half>, P.nwork[kWorkRowPack], kBlock, 0, st, P.meshes,
                           P.work[kWorkRowPack], V, rf, of, wt);
        }
    }
    if (prec != CGS_FP64 && P.nwork[kWorkPack]) {
        const float* rf = static_cast<const float*>(r);
        float* of = static_cast<float*>(out);
        if (prec == CGS_FP32_BULK)
            launch_pdl(P.pdl, local_lane_kernel<float>, P.nwork[kWorkPack], kBlock, 0, st, P.meshes, P.work[kWorkPack],
                       V, rf, of, wt);
        else
            launch_pdl(P.pdl, local_lane_kernel<__half>, P.nwork[kWorkPack], kBlock, 0, st, P.meshes, P.work[kWorkPack],
                       V, rf, of, wt);
        if (P.lane_big) {
            if (prec == CGS_FP32_BULK)
                launch_pdl(P.pdl, local_lane_big_kernel<float>, P.nwork[kWorkPack], kBlock, 0, st, P.meshes,
                           P.work[kWorkPack], V, rf, of, wt);
            else
                launch_pdl(P.pdl, local_lane_big_kernel<__half>, P.nwork[kWorkPack], kBlock, 0, st, P.meshes,
                           P.work[kWorkPack], V, rf, of, wt);
        }
    }
    if (prec == CGS_FP64 && P.nwork[kWorkPack]) {
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            sms = std::max(sms, 1);
        }
        const int64_t warps = (int64_t)P.nwork[kWorkPack] * P.pack_chunk;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (warps + kBlock / 32 - 1) / (kBlock / 32)));
        launch_pdl(P.pdl, local_lane64_kernel, grid, kBlock, 0, st, P.meshes, P.work[kWorkPack],
                   (int)P.nwork[kWorkPack], P.pack_chunk, V, static_cast<const double*>(r), static_cast<double*>(out),
                   wt);
    }
    // the rest (in the FP64 form every subdomain outside lane packs): a warp
    // per subdomain of up to 64 dofs, a block per larger one
    if (!P.nwork[kWorkSub]) return;
    const unsigned int n = P.nwork[kWorkSub];
    const Work* W = P.work[kWorkSub];
    // r is float64 in the FP64 form and the float copy of the residual otherwise
    if (prec == CGS_FP64) {
        launch_pdl(P.pdl, local_warp_kernel<double, double>, n, kBlock, 0, st, P.meshes, W, V,
                   static_cast<const double*>(r), static_cast<double*>(out), wt);
        if (P.max_m > 64)
            launch_pdl(P.pdl, local_block_kernel<double, double>, n, kBlock, 0, st, P.meshes, W, V,
                       static_cast<const double*>(r), static_cast<double*>(out), wt);
    } else if (prec == CGS_FP32_BULK) {
        launch_pdl(P.pdl, local_warp_kernel<float, float>, n, kBlock, 0, st, P.meshes, W, V,
                   static_cast<const float*>(r), static_cast<float*>(out), wt);
        if (P.max_m > 64)
            launch_pdl(P.pdl, local_block_kernel<float, float>, n, kBlock, 0, st, P.meshes, W, V,
                       static_cast<const float*>(r), static_cast<float*>(out), wt);
    } else {
        launch_pdl(P.pdl, local_warp_kernel<float, __half>, n, kBlock, 0, st, P.meshes, W, V,
                   static_cast<const float*>(r), static_cast<float*>(out), wt);
        if (P.max_m > 64)
            launch_pdl(P.pdl, local_block_kernel<float, __half>, n, kBlock, 0, st, P.meshes, W, V,
                       static_cast<const float*>(r), static_cast<float*>(out), wt);
    }
}

bool launch_local_restrict(const Plan& P, const Vecs& V, cgs_precision prec, const float* s, float* z, void* rr,
                           cudaStream_t st) {
    // only when every subdomain is in packs of at most 32 dofs (no warp-list
    // or large-class launch needed)
    if (prec == CGS_FP64 || P.nwork[kWorkSub] || P.lane_big || !P.any_nr || !P.nwork[kWorkBoxEnt]) return false;
    const bool rowp = P.nwork[kWorkRowPack] > 0;
    const unsigned int nl = rowp ? P.nwork[kWorkRowPack] : P.nwork[kWorkPack];
    const Work* wl = rowp ? P.work[kWorkRowPack] : P.work[kWorkPack];
    const unsigned int grid = nl + P.nwork[kWorkBoxEnt];
    if (prec == CGS_FP32_BULK)
        launch_pdl(P.pdl, local_restrict_kernel<float>, grid, kBlock, 0, st, P.meshes, wl, nl, rowp ? 1 : 0,
                   P.work[kWorkBoxEnt], V, s, z, rr);
    else
        launch_pdl(P.pdl, local_restrict_kernel<__half>, grid, kBlock, 0, st, P.meshes, wl, nl, rowp ? 1 : 0,
                   P.work[kWorkBoxEnt], V, s, z, rr);
    return true;
}

void launch_restrict_hybrid(const Plan& P, const Vecs& V, bool fp64, const void* r, const void* l, void* rr,
                            cudaStream_t st) {
    if (!P.nwork[kWorkHybR] || !P.any_nr) return;
    const unsigned int n = P.nwork[kWorkHybR];
    if (fp64)
        launch_pdl(P.pdl, restrict_hyb_kernel<double>, n, kBlock, 0, st, P.meshes, P.work[kWorkHybR], V,
                   static_cast<const double*>(r), static_cast<const double*>(l), rr);
    else
        launch_pdl(P.pdl, restrict_hyb_kernel<float>, n, kBlock, 0, st, P.meshes, P.work[kWorkHybR], V,
                   static_cast<const float*>(r), static_cast<const float*>(l), rr);
}

void launch_restrict(const Plan& P, const Vecs& V, bool fp64, const void* s, bool s_is_double, void* rr,
                     bool pair_out, cudaStream_t st) {
    if (!P.nwork[kWorkBoxEnt] || !P.any_nr) return;
    const unsigned int n = P.nwork[kWorkBoxEnt];
    const Work* W = P.work[kWorkBoxEnt];
    if (fp64)
        launch_pdl(P.pdl, restrict_kernel<double, double, false>, n, kBlock, 0, st, P.meshes, W, V,
                   static_cast<const double*>(s), rr);
    else if (s_is_double)
        launch_pdl(P.pdl, restrict_kernel<float, double, false>, n, kBlock, 0, st, P.meshes, W, V,
                   static_cast<const double*>(s), rr);
    else if (pair_out)
        launch_pdl(P.pdl, restrict_kernel<float, float, true>, n, kBlock, 0, st, P.meshes, W, V,
                   static_cast<const float*>(s), rr);
    else
        launch_pdl(P.pdl, restrict_kernel<float, float, false>, n, kBlock, 0, st, P.meshes, W, V,
                   static_cast<const float*>(s), rr);
}

bool launch_interp_add(const Plan& P, const Vecs& V, bool fp64, const double* ur, const float* ur32, void* z,
                       bool dots, const cudaGraphConditionalHandle* cond, cudaStream_t st) {
    if (fp64) {   // by the explicit float64 rows of J~, the dots fused
        if (!P.nwork[kWorkBox] || !P.any_nr) return false;
        const cudaGraphConditionalHandle h = cond ? *cond : 0;
        if (dots)
            launch_pdl(P.pdl, interp_rows_kernel<1>, P.nwork[kWorkBox], kBlock, 0, st, P.meshes, P.work[kWorkBox], V,
                       ur, static_cast<double*>(z), P.nslots, h, cond ? 1 : 0);
        else
            launch_pdl(P.pdl, interp_rows_kernel<0>, P.nwork[kWorkBox], kBlock, 0, st, P.meshes, P.work[kWorkBox], V,
                       ur, static_cast<double*>(z), P.nslots, h, cond ? 1 : 0);
        return dots;
    }
    if (P.interp_cells) {   // by cell-sorted entries; the dots are left to the caller
        if (!P.nwork[kWorkBoxEnt] || !P.any_nr) return false;
        const unsigned int n = P.nwork[kWorkBoxEnt];
        const Work* W = P.work[kWorkBoxEnt];
        if (fp64)
            launch_pdl(P.pdl, interp_cell_kernel<double, double>, n, kBlock, 0, st, P.meshes, W, V, ur,
                       static_cast<double*>(z));
        else if (ur32)
            launch_pdl(P.pdl, interp_cell_kernel<float, float>, n, kBlock, 0, st, P.meshes, W, V, ur32,
                       static_cast<float*>(z));
        else
            launch_pdl(P.pdl, interp_cell_kernel<float, double>, n, kBlock, 0, st, P.meshes, W, V, ur,
                       static_cast<float*>(z));
        return false;
    }
    if (!P.nwork[kWorkBox] || !P.any_nr) return false;
    const unsigned int n = P.nwork[kWorkBox];
    const Work* W = P.work[kWorkBox];
    const cudaGraphConditionalHandle h = cond ? *cond : 0;
    const int sc = cond ? 1 : 0;
    if (fp64) {
        if (dots)
            launch_pdl(P.pdl, interp_add_kernel<double, double, 1>, n, kBlock, 0, st, P.meshes, W, V, ur,
                       static_cast<double*>(z), P.nslots, h, sc);
        else
            launch_pdl(P.pdl, interp_add_kernel<double, double, 0>, n, kBlock, 0, st, P.meshes, W, V, ur,
                       static_cast<double*>(z), P.nslots, h, sc);
    } else if (ur32) {   // float copy of u_r written by the reduced solve: no conversions per vertex
        if (dots)
            launch_pdl(P.pdl, interp_add_kernel<float, float, 2>, n, kBlock, 0, st, P.meshes, W, V, ur32,
                       static_cast<float*>(z), P.nslots, h, sc);
        else
            launch_pdl(P.pdl, interp_add_kernel<float, float, 0>, n, kBlock, 0, st, P.meshes, W, V, ur32,
                       static_cast<float*>(z), P.nslots, h, sc);
    } else {
        launch_pdl(P.pdl, interp_add_kernel<float, double, 0>, n, kBlock, 0, st, P.meshes, W, V, ur,
                   static_cast<float*>(z), P.nslots, h, sc);
        return false;
    }
    return dots;
}

void launch_coarse(const Plan& P, const Vecs& V, const double* rr, double* ur, float* ur32, cudaStream_t st) {
    if (!P.nwork[kWorkRow]) return;
    launch_pdl(P.pdl, coarse_gemv_kernel, P.nwork[kWorkRow], 32 * kRowChunk, 0, st, P.meshes, P.work[kWorkRow], V, rr,
               ur, ur32);
}

bool launch_xxt_pass1(const Plan& P, const Vecs& V, bool pair, const double* rr, cudaStream_t st) {
    if (!P.nwork[kWorkXSeg]) return false;
    if (pair)
        launch_pdl(P.pdl, xxt_seg_kernel<true>, P.nwork[kWorkXSeg], 32 * kRowChunk, 0, st, P.meshes,
                   P.work[kWorkXSeg], V, rr);
    else
        launch_pdl(P.pdl, xxt_seg_kernel<false>, P.nwork[kWorkXSeg], 32 * kRowChunk, 0, st, P.meshes,
                   P.work[kWorkXSeg], V, rr);
    return true;
}

void launch_coarse_pair(const Plan& P, const Vecs& V, const float2* rr2, double* ur, float* ur32, cudaStream_t st) {
    if (!P.nwork[kWorkRow]) return;
    launch_pdl(P.pdl, coarse_pair_kernel, P.nwork[kWorkRow], 32 * kRowChunk, 0, st, P.meshes, P.work[kWorkRow], V, rr2,
               ur, ur32);
}

#define CGS_VLAUNCH(kernel, ...) \
    launch_pdl(P.pdl, kernel, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V, ##__VA_ARGS__)
void launch_pcg_init_pair(const Plan& P, const Vecs& V, double rtol, int maxit, cudaStream_t st) {
    CGS_VLAUNCH(pcg_init_pair_kernel, rtol, maxit);
}

void launch_precond_prep_pair(const Plan& P, const Vecs& V, cudaStream_t st) {
    CGS_VLAUNCH(precond_prep_pair_kernel);
}

void launch_pcg_first_dir_pair(const Plan& P, const Vecs& V, cudaStream_t st) {
    CGS_VLAUNCH(pcg_first_dir_pair_kernel);
}

void launch_pcg_update_xr_pair(const Plan& P, const Vecs& V, cudaStream_t st, bool form_p) {
    CGS_VLAUNCH(pcg_update_xr_pair_kernel, form_p ? 1 : 0);
}

void launch_pcg_update_p_pair(const Plan& P, const Vecs& V, const cudaGraphConditionalHandle* cond,
                              cudaStream_t st) {
    CGS_VLAUNCH(pcg_update_p_pair_kernel, P.nslots, cond ? *cond : 0, cond ? 1 : 0);
}

void launch_pcg_dots_pair(const Plan& P, const Vecs& V, const cudaGraphConditionalHandle* cond, cudaStream_t st) {
    CGS_VLAUNCH(pcg_dots_pair_kernel, P.nslots, cond ? *cond : 0, cond ? 1 : 0);
}

void launch_finalize_x_pair(const Plan& P, const Vecs& V, cudaStream_t st) { CGS_VLAUNCH(finalize_x_pair_kernel); }
#undef CGS_VLAUNCH

// float64 -> float pair over n entries (r_r of the single-step reduced solve)
__global__ void split_pair_kernel(int64_t n, const double* __restrict__ a, float2* __restrict__ b) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = split_pair(a[i]);
}

void launch_split_pair(int64_t n, const double* a, float2* b, cudaStream_t st) {
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 1024);
    launch_pdl(true, split_pair_kernel, blocks, kBlock, 0, st, n, a, b);
}

// float pair -> float64 (hi + lo) over n entries (single-step outer operator)
__global__ void pair_to_double_kernel(int64_t n, const float2* __restrict__ a, double* __restrict__ b) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 t = a[i];
        b[i] = (double)t.x + (double)t.y;
    }
}

void launch_pair_to_double(int64_t n, const float2* a, double* b, cudaStream_t st) {
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 1024);
    launch_pdl(true, pair_to_double_kernel, blocks, kBlock, 0, st, n, a, b);
}

template <typename Tq>
void launch_pcg_init(const Plan& P, const Vecs& V, Tq* q, double rtol, int maxit, cudaStream_t st) {
    launch_pdl(P.pdl, pcg_init_kernel<Tq>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V, q, rtol,
               maxit);
}

template <typename Tz>
void launch_precond_prep(const Plan& P, const Vecs& V, const double* r, cudaStream_t st) {
    launch_pdl(P.pdl, precond_prep_kernel<Tz>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V, r);
}

template <typename Tz>
void launch_pcg_first_dir(const Plan& P, const Vecs& V, cudaStream_t st) {
    launch_pdl(P.pdl, pcg_first_dir_kernel<Tz>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V);
}

template <typename Tz, typename Tq>
void launch_pcg_update_xr(const Plan& P, const Vecs& V, const Tq* q, cudaStream_t st) {
    launch_pdl(P.pdl, pcg_update_xr_kernel<Tz, Tq>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V,
               q);
}

template <typename Tz, typename Tq>
void launch_pcg_dots(const Plan& P, const Vecs& V, const Tq* q, cudaStream_t st) {
    launch_pdl(P.pdl, pcg_dots_kernel<Tz, Tq>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V, q);
}

template <typename Tz, typename Tq>
void launch_pcg_update_p(const Plan& P, const Vecs& V, Tq* q, const cudaGraphConditionalHandle* cond,
                         cudaStream_t st) {
    launch_pdl(P.pdl, pcg_update_p_kernel<Tz, Tq>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V, q,
               P.nslots, cond ? *cond : 0, cond ? 1 : 0);
}

// Blocks of the persistent loop that fit on the device at once (the
// cooperative launch requires all of them resident).
static const void* persistent_fn(cgs_precision prec, bool big) {
    if (prec == CGS_FP16_LOCAL)
        return big ? (const void*)pcg_persistent_kernel<__half, true> : (const void*)pcg_persistent_kernel<__half, false>;
    return big ? (const void*)pcg_persistent_kernel<float, true> : (const void*)pcg_persistent_kernel<float, false>;
}

int persistent_blocks(cgs_precision prec, bool big) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem = (int)(2 * kTileVerts * sizeof(float2));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_fn(prec, big), kBlock, smem);
    return per_sm * sms;
}

cudaError_t launch_pcg_persistent(const Plan& P, const Vecs& V, cgs_precision prec, bool hybrid, GridBar* bar,
                                  int max_iters, int blocks, cudaStream_t st) {
    LoopTables T;
    for (int k = 0; k < kWorkKinds; ++k) {
        T.w[k] = P.work[k];
        T.n[k] = P.nwork[k];
    }
    int nslots = P.nslots, hyb = hybrid ? 1 : 0, any_nr = P.any_nr ? 1 : 0, big = P.max_m > 64 ? 1 : 0;
    int wait_limit = P.wait_limit, bar_limit = P.bar_limit;
    Vecs Vv = V;
    const DevMesh* meshes = P.meshes;
    void* args[] = {(void*)&meshes, &T, &Vv, &bar, &nslots, &hyb, &any_nr, &big, &max_iters, &wait_limit, &bar_limit};
    const int smem = (int)(2 * kTileVerts * sizeof(float2));
    return cudaLaunchCooperativeKernel(persistent_fn(prec, P.lane_big), dim3(blocks), dim3(kBlock), args, smem, st);
}

void launch_resid_norm(const Plan& P, const Vecs& V, cudaStream_t st) {
    launch_pdl(P.pdl, resid_norm_kernel, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], V);
}

constexpr int64_t kInterpCellsMinVerts = 65536;
Schedule default_schedule(int64_t total_nv, int64_t total_sub, int64_t total_pack, int64_t total_lane_subs) {
    const int64_t target = 4 * 148;
    Schedule s;
    int64_t v = (total_nv + target - 1) / target;
    s.vert_chunk = (int)std::min<int64_t>(2048, std::max<int64_t>(256, (v + 255) / 256 * 256));
    int64_t c = (total_sub + target - 1) / target;
    s.sub_chunk = (int)std::min<int64_t>(64, std::max<int64_t>(8, (c + 7) / 8 * 8));
    int64_t k = (total_pack + target - 1) / target;
    s.pack_chunk = (int)std::min<int64_t>(32, std::max<int64_t>(8, (k + 7) / 8 * 8));
    s.box_chunk = (int)std::min<int64_t>(1024, std::max<int64_t>(256, (v + 255) / 256 * 256));
    // four lanes per small subdomain only while one lane each leaves the GPU idle
    s.row_packs = total_lane_subs < kRowPackMaxSubs ? 1 : 0;
    // the interpolation by cells (and a separate dots kernel) once the vertex
    // count fills the GPU; below that, one launch fewer per iteration counts more
    s.interp_cells = total_nv >= kInterpCellsMinVerts ? 1 : 0;
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
    if (sch.row_packs && z.n_rpack > 0)
        add(kWorkRowPack, z.n_rpack, sch.pack_chunk);
    else
        add(kWorkPack, z.n_pack, sch.pack_chunk);
    add(kWorkBox, z.nvb, sch.box_chunk);
    if (z.nr > 0) add(kWorkBoxEnt, z.nrng, kBlock / 32);
    if (z.nxseg > 0) add(kWorkXSeg, z.nxseg, kRowChunk);
    if (z.nr > 0 && z.nhr > 0) add(kWorkHybR, z.nhr, kBlock / 32);
    add(kWorkEll, z.nv, kEllChunk);
}

int64_t mesh_partial_slots(const MeshSizes& z, const Schedule& sch) {
    int64_t c = (z.ne + kElemChunk - 1) / kElemChunk;
    c = std::max(c, z.ntiles);
    c = std::max(c, (z.nv + sch.vert_chunk - 1) / sch.vert_chunk);
    c = std::max(c, (z.nvb + sch.box_chunk - 1) / sch.box_chunk);
    c = std::max(c, (z.nv + kEllChunk - 1) / kEllChunk);
    return 2 * std::max<int64_t>(c, 1);
}

template void launch_pcg_update_xr<double, double>(const Plan&, const Vecs&, const double*, cudaStream_t);
template void launch_pcg_dots<double, double>(const Plan&, const Vecs&, const double*, cudaStream_t);
template void launch_pcg_update_p<double, double>(const Plan&, const Vecs&, double*,
                                                  const cudaGraphConditionalHandle*, cudaStream_t);
template void launch_pcg_init<double>(const Plan&, const Vecs&, double*, double, int, cudaStream_t);
template void launch_precond_prep<double>(const Plan&, const Vecs&, const double*, cudaStream_t);
template void launch_precond_prep<float>(const Plan&, const Vecs&, const double*, cudaStream_t);
template void launch_pcg_first_dir<double>(const Plan&, const Vecs&, cudaStream_t);

void launch_convert_f2d(const Plan& P, const float* a, double* b, bool mask, cudaStream_t st) {
    launch_pdl(P.pdl, convert_kernel<float, double>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], a,
               b, mask);
}

void launch_convert_d2f(const Plan& P, const double* a, float* b, bool mask, cudaStream_t st) {
    launch_pdl(P.pdl, convert_kernel<double, float>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], a,
               b, mask);
}

void launch_copy_d(const Plan& P, const double* a, double* b, bool mask, cudaStream_t st) {
    launch_pdl(P.pdl, convert_kernel<double, double>, P.nwork[kWorkVert], kBlock, 0, st, P.meshes, P.work[kWorkVert], a,
               b, mask);
}

void launch_fill_d(int64_t n, double* a, double v, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t b = std::min<int64_t>((n + kBlock - 1) / kBlock, 148 * 8);
    launch_pdl(true, fill_kernel<double>, (unsigned int)b, kBlock, 0, st, n, a, v);
}

void launch_fill_f(int64_t n, float* a, float v, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t b = std::min<int64_t>((n + kBlock - 1) / kBlock, 148 * 8);
    launch_pdl(true, fill_kernel<float>, (unsigned int)b, kBlock, 0, st, n, a, v);
}

}  // namespace cgs
