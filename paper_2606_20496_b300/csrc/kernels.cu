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

// Operator apply, float32, 28 off-diagonals: y_i += alpha * sum_j a_ij (x_j - x_i)
// (zero row sums of A^e give the diagonal).
__global__ void __launch_bounds__(kBlock) apply28f_kernel(int64_t ne, const int32_t* __restrict__ conn,
                                                          const float* __restrict__ a28,
                                                          const float* __restrict__ x, float* __restrict__ y,
                                                          float alpha, const SolveScalars* S) {
    if (is_done(S)) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    int v[8];
    load_conn(conn, e, v);
    float xe[8], ye[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        xe[k] = v[k] >= 0 ? __ldg(&x[v[k]]) : 0.0f;
        ye[k] = 0.0f;
    }
    int s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = i + 1; j < 8; ++j, ++s) {
            const float d = __ldg(&a28[(size_t)s * ne + e]) * (xe[j] - xe[i]);
            ye[i] += d;
            ye[j] -= d;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (v[k] >= 0) atomicAdd(&y[v[k]], alpha * ye[k]);
}

// ---------------------------------------------------------------------------
// Local solves, one warp per subdomain with m_p <= 64 dofs (lanes hold dofs
// lane and lane+32).  The packed lower-triangular inverse is staged in the
// warp's slice of shared memory by coalesced loads, then lane i forms
// y_i = sum_j inv(i,j) x_j with x_j broadcast by shuffles.
// ---------------------------------------------------------------------------
template <typename Stor>
__device__ __forceinline__ float load_entry(const Stor* p, size_t i, float scale);
template <>
__device__ __forceinline__ float load_entry<float>(const float* p, size_t i, float) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float load_entry<__half>(const __half* p, size_t i, float scale) {
    return __half2float(p[i]) * scale;
}

template <typename T, typename Stor>
__device__ __forceinline__ T stage(const Stor* p, size_t i, float scale) {
    return (T)load_entry<Stor>(p, i, scale);
}
template <>
__device__ __forceinline__ double stage<double, double>(const double* p, size_t i, float) { return __ldg(p + i); }

__device__ __forceinline__ int pk(int i, int j) { return i >= j ? (i * (i + 1) >> 1) + j : (j * (j + 1) >> 1) + i; }

template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_warp_kernel(int64_t n_sub, const int32_t* __restrict__ sub_ptr,
                                                            const int32_t* __restrict__ sub_idx,
                                                            const int64_t* __restrict__ inv_ptr,
                                                            const Stor* __restrict__ inv,
                                                            const float* __restrict__ scale,
                                                            const double* __restrict__ r,
                                                            const T* __restrict__ wov, T* __restrict__ out,
                                                            int cap, const SolveScalars* S) {
    if (is_done(S)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sh = reinterpret_cast<T*>(smem_raw) + (size_t)(threadIdx.x >> 5) * cap;
    const int lane = threadIdx.x & 31;
    const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_sub; p += nwt) {
        const int o = __ldg(&sub_ptr[p]);
        const int m = __ldg(&sub_ptr[p + 1]) - o;
        if (m == 0 || m > 64) continue;
        const bool h0 = lane < m, h1 = lane + 32 < m;
        const int v0 = h0 ? __ldg(&sub_idx[o + lane]) : 0;
        const int v1 = h1 ? __ldg(&sub_idx[o + lane + 32]) : 0;
        const T x0 = h0 ? (T)__ldg(&r[v0]) : T(0);
        const T x1 = h1 ? (T)__ldg(&r[v1]) : T(0);
        const size_t io = (size_t)__ldg(&inv_ptr[p]);
        const int np = m * (m + 1) / 2;
        const float sc = scale ? __ldg(&scale[p]) : 1.0f;
        for (int t = lane; t < np; t += 32) sh[t] = stage<T, Stor>(inv, io + t, sc);
        __syncwarp();
        T y0 = 0, y1 = 0;
        for (int j = 0; j < m; ++j) {
            const T xj = j < 32 ? __shfl_sync(0xffffffffu, x0, j) : __shfl_sync(0xffffffffu, x1, j - 32);
            if (h0) y0 += sh[pk(lane, j)] * xj;
            if (h1) y1 += sh[pk(lane + 32, j)] * xj;
        }
        __syncwarp();
        if (h0) atomicAdd(&out[v0], wov ? y0 * __ldg(&wov[v0]) : y0);
        if (h1) atomicAdd(&out[v1], wov ? y1 * __ldg(&wov[v1]) : y1);
    }
}

// Subdomains with more than 64 dofs: one block each, rows spread over threads.
template <typename T, typename Stor>
__global__ void __launch_bounds__(kBlock) local_block_kernel(int64_t n_sub, const int32_t* __restrict__ sub_ptr,
                                                             const int32_t* __restrict__ sub_idx,
                                                             const int64_t* __restrict__ inv_ptr,
                                                             const Stor* __restrict__ inv,
                                                             const float* __restrict__ scale,
                                                             const double* __restrict__ r,
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
            for (int j = 0; j < m; ++j)
                y += stage<T, Stor>(inv, io + pk(i, j), sc) * (T)__ldg(&r[sub_idx[o + j]]);
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
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const double sum = warp_sum(mine ? (double)acc[m] : 0.0);
            if (lane == leader) {
                const int col = __ldg(&cell_cols[(size_t)cc * 8 + m]);
                if (col >= 0) atomicAdd(&rr[col], sum);
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) interp_add_kernel(int64_t ne, const int32_t* __restrict__ conn,
                                                            const int32_t* __restrict__ cell,
                                                            const int32_t* __restrict__ cell_cols,
                                                            VertexXYZW<T> vx, BoxGrid<T> g,
                                                            const double* __restrict__ ur, T* __restrict__ z,
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
                                                             double* __restrict__ ur, const SolveScalars* S) {
    if (is_done(S)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nr; i += nwt) {
        const double* row = Ainv + (size_t)i * nr;
        double s = 0.0;
        for (int64_t j = lane; j < nr; j += 32) s = fma(__ldg(&row[j]), __ldg(&rr[j]), s);
        s = warp_sum(s);
        if (lane == 0) ur[i] = s;
    }
}

// ---------------------------------------------------------------------------
// PCG vector kernels (float64 outer iteration)
// ---------------------------------------------------------------------------

// r = b with Dirichlet entries zeroed, x = 0, q = 0; ||b||^2 -> bnorm2, tol2.
__global__ void __launch_bounds__(kBlock) pcg_init_kernel(int64_t nv, const double* __restrict__ b,
                                                          const uint8_t* __restrict__ dir, double* __restrict__ x,
                                                          double* __restrict__ r, double* __restrict__ q,
                                                          double rtol, int maxit, double* partials,
                                                          SolveScalars* S) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = dir[i] ? 0.0 : b[i];
        r[i] = bi;
        x[i] = 0.0;
        q[i] = 0.0;
        acc = fma(bi, bi, acc);
    }
    double val[1] = {acc}, tot[1];
    if (grid_sum<1>(val, partials, &S->ticket[1], tot) && threadIdx.x == 0) {
        S->bnorm2 = tot[0];
        S->tol2 = rtol * rtol * tot[0];
        S->iters = 0;
        S->maxit = maxit;
        S->status = CGS_OK;
        S->done = (tot[0] == 0.0 || maxit <= 0) ? 1 : 0;
        if (maxit <= 0 && tot[0] != 0.0) S->status = CGS_ERR_NO_CONVERGENCE;
        S->rho = 0.0;
    }
}

// p = z, rho = r.z (start of the iteration).
template <typename Tz>
__global__ void __launch_bounds__(kBlock) pcg_first_dir_kernel(int64_t nv, const Tz* __restrict__ z,
                                                               const double* __restrict__ r, double* __restrict__ p,
                                                               double* partials, SolveScalars* S) {
    if (is_done(S)) return;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = (double)z[i];
        p[i] = zi;
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
template <typename Tz>
__global__ void __launch_bounds__(kBlock) pcg_update_xr_kernel(int64_t nv, double* __restrict__ x,
                                                               double* __restrict__ r, const double* __restrict__ p,
                                                               const double* __restrict__ q, Tz* __restrict__ z,
                                                               Tz* __restrict__ s, double* __restrict__ rr_vec,
                                                               int64_t nr, double* partials, SolveScalars* S) {
    if (is_done(S)) return;
    const double alpha = S->alpha;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
        z[i] = Tz(0);
        if (s) s[i] = (Tz)ri;
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
template <typename Tz>
__global__ void __launch_bounds__(kBlock) pcg_dots_kernel(int64_t nv, const Tz* __restrict__ z,
                                                          const double* __restrict__ r, const double* __restrict__ q,
                                                          double* partials, SolveScalars* S) {
    if (is_done(S)) return;
    double zr = 0.0, zq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = (double)z[i];
        zr = fma(zi, r[i], zr);
        zq = fma(zi, q[i], zq);
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

// p = z + beta p; q = 0 for the next product.
template <typename Tz>
__global__ void __launch_bounds__(kBlock) pcg_update_p_kernel(int64_t nv, const Tz* __restrict__ z,
                                                              double* __restrict__ p, double* __restrict__ q,
                                                              const SolveScalars* S) {
    if (is_done(S)) return;
    const double beta = S->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        p[i] = fma(beta, p[i], (double)z[i]);
        q[i] = 0.0;
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
    return std::max(grid_exact(m.ne), grid_for(m.nv));
}

void launch_apply64(const DevMesh& m, const double* x, double* y, double alpha, double* partials,
                    SolveScalars* S, bool dot, cudaStream_t st) {
    if (dot)
        apply64_kernel<true><<<grid_exact(m.ne), kBlock, 0, st>>>(m.ne, m.conn, m.a36, x, y, alpha, partials, S);
    else
        apply64_kernel<false><<<grid_exact(m.ne), kBlock, 0, st>>>(m.ne, m.conn, m.a36, x, y, alpha, partials, S);
}

void launch_apply28f(const DevMesh& m, const float* x, float* y, float alpha, const SolveScalars* S,
                     cudaStream_t st) {
    apply28f_kernel<<<grid_exact(m.ne), kBlock, 0, st>>>(m.ne, m.conn, m.a28, x, y, alpha, S);
}

template <typename T, typename Stor>
static void local_launch(const DevMesh& m, const Stor* inv, const float* scale, const double* r, const T* wov, T* out,
                         const SolveScalars* S, cudaStream_t st) {
    if (m.n_sub == 0) return;
    // each warp stages one packed inverse of at most min(max_m, 64) dofs
    const int mm = std::min(m.max_m, 64);
    const int cap = (mm * (mm + 1) / 2 + 3) / 4 * 4;
    const size_t smem = (size_t)(kBlock / 32) * cap * sizeof(T);
    static bool attr_set = false;
    if (!attr_set) {
        const int most = (int)((size_t)(kBlock / 32) * (64 * 65 / 2) * sizeof(T));
        cudaFuncSetAttribute(local_warp_kernel<T, Stor>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        attr_set = true;
    }
    const int64_t warps_needed = m.n_sub;
    const unsigned int blocks =
        (unsigned int)std::max<int64_t>(1, std::min<int64_t>((warps_needed + 7) / 8, 148 * 16));
    local_warp_kernel<T, Stor><<<blocks, kBlock, smem, st>>>(m.n_sub, m.sub_ptr, m.sub_idx, m.inv_ptr, inv, scale, r,
                                                             wov, out, cap, S);
    if (m.max_m > 64)
        local_block_kernel<T, Stor><<<(unsigned int)std::min<int64_t>(m.n_sub, 148 * 8), kBlock, 0, st>>>(
            m.n_sub, m.sub_ptr, m.sub_idx, m.inv_ptr, inv, scale, r, wov, out, S);
}

void launch_local(const DevMesh& m, cgs_precision prec, const double* r, void* out, bool weighted,
                  const SolveScalars* S, cudaStream_t st) {
    if (prec == CGS_FP64)
        local_launch<double, double>(m, m.inv64, nullptr, r, weighted ? m.wov64 : nullptr,
                                     static_cast<double*>(out), S, st);
    else if (prec == CGS_FP32_BULK)
        local_launch<float, float>(m, m.inv32, nullptr, r, weighted ? m.wov32 : nullptr, static_cast<float*>(out), S,
                                   st);
    else
        local_launch<float, __half>(m, m.inv16, m.inv16_scale, r, weighted ? m.wov32 : nullptr,
                                    static_cast<float*>(out), S, st);
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

void launch_interp_add(const DevMesh& m, bool fp64, const double* ur, void* z, const SolveScalars* S,
                       cudaStream_t st) {
    if (fp64) {
        VertexXYZW<double> vx{m.xyzw};
        interp_add_kernel<double><<<grid_exact(m.ne), kBlock, 0, st>>>(m.ne, m.conn, m.cell, m.cell_cols, vx,
                                                                       box_grid<double>(m), ur,
                                                                       static_cast<double*>(z), S);
    } else {
        VertexXYZW<float> vx{m.xyzwf};
        interp_add_kernel<float><<<grid_exact(m.ne), kBlock, 0, st>>>(m.ne, m.conn, m.cell, m.cell_cols, vx,
                                                                      box_grid<float>(m), ur, static_cast<float*>(z),
                                                                      S);
    }
}

void launch_coarse(const DevMesh& m, const double* rr, double* ur, const SolveScalars* S, cudaStream_t st) {
    if (m.nr == 0) return;
    const unsigned int blocks = (unsigned int)std::min<int64_t>((m.nr + 7) / 8, 148 * 16);
    coarse_gemv_kernel<<<blocks, kBlock, 0, st>>>(m.nr, m.ar_inv, rr, ur, S);
}

void launch_pcg_init(const DevMesh& m, const double* b, const uint8_t* dir, double* x, double* r, double* q,
                     double rtol, int maxit, double* partials, SolveScalars* S, cudaStream_t st) {
    pcg_init_kernel<<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, b, dir, x, r, q, rtol, maxit, partials, S);
}

template <typename Tz>
void launch_pcg_first_dir(const DevMesh& m, const Tz* z, const double* r, double* p, double* partials,
                          SolveScalars* S, cudaStream_t st) {
    pcg_first_dir_kernel<Tz><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, z, r, p, partials, S);
}
template <typename Tz>
void launch_pcg_update_xr(const DevMesh& m, double* x, double* r, const double* p, const double* q, Tz* z, Tz* s,
                          double* rr_vec, double* partials, SolveScalars* S, cudaStream_t st) {
    pcg_update_xr_kernel<Tz><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, x, r, p, q, z, s, rr_vec, m.nr, partials, S);
}
template <typename Tz>
void launch_pcg_dots(const DevMesh& m, const Tz* z, const double* r, const double* q, double* partials,
                     SolveScalars* S, cudaStream_t st) {
    pcg_dots_kernel<Tz><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, z, r, q, partials, S);
}
template <typename Tz>
void launch_pcg_update_p(const DevMesh& m, const Tz* z, double* p, double* q, const SolveScalars* S,
                         cudaStream_t st) {
    pcg_update_p_kernel<Tz><<<grid_for(m.nv), kBlock, 0, st>>>(m.nv, z, p, q, S);
}
template void launch_pcg_first_dir<double>(const DevMesh&, const double*, const double*, double*, double*,
                                           SolveScalars*, cudaStream_t);
template void launch_pcg_first_dir<float>(const DevMesh&, const float*, const double*, double*, double*,
                                          SolveScalars*, cudaStream_t);
template void launch_pcg_update_xr<double>(const DevMesh&, double*, double*, const double*, const double*, double*,
                                           double*, double*, double*, SolveScalars*, cudaStream_t);
template void launch_pcg_update_xr<float>(const DevMesh&, double*, double*, const double*, const double*, float*,
                                          float*, double*, double*, SolveScalars*, cudaStream_t);
template void launch_pcg_dots<double>(const DevMesh&, const double*, const double*, const double*, double*,
                                      SolveScalars*, cudaStream_t);
template void launch_pcg_dots<float>(const DevMesh&, const float*, const double*, const double*, double*,
                                     SolveScalars*, cudaStream_t);
template void launch_pcg_update_p<double>(const DevMesh&, const double*, double*, double*, const SolveScalars*,
                                          cudaStream_t);
template void launch_pcg_update_p<float>(const DevMesh&, const float*, double*, double*, const SolveScalars*,
                                         cudaStream_t);

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
