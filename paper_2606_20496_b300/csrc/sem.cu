// Kernels of the p-multigrid wrap's spectral-element levels (Sec. 1, Sec. 5,
// Eqs. (13) and (14)), one block of p x p threads per element:
// thread (i, j) holds the column k = 0..p-1 of its element in registers and
// exchanges layers through shared memory for the contractions along i and j.
//
//   sem_ax        y += A_n x, A^e = Dhat^T G^e Dhat (GLL quadrature)
//   sem_fdm       z += W sum_e R_e^T A~_e^-1 R_e r by fast diagonalisation
//   sem_restrict  r_c += J^T r_f = Q_c^T I^T Q_f W_f r_f
//   sem_prolong   z_f += J u_c = W_f Q_f^T I Q_c u_c
//
// Element-local to global maps store a Dirichlet node g as -(g + 1): gathers
// read zero there and scatters skip it, so Dirichlet entries are ignored on
// input and never written.  Scatters are atomic adds (the order of the
// additions, and so the last bits, varies from run to run).
//
// Precision follows the coarse mesh.  Under an FP64 mesh everything is
// float64.  Under the mixed forms' meshes the operator runs in float-pair
// arithmetic (about 48 bits: GMRES's residual, like the coarse solver's
// outer operator), and the smoother and the transfers in float (the
// multilevel preconditioner needs no more: the outer GMRES is flexible),
// with level vectors in float below the finest level; the finest level's
// vectors, and the order-1 vectors handed to the coarse preconditioner, stay
// float64.
#include <cuda_runtime.h>

#include "sem.h"

namespace cgs {

namespace {

__device__ __forceinline__ double gather(const double* __restrict__ v, int32_t g) { return g >= 0 ? __ldg(&v[g]) : 0.0; }

template <int P>
__global__ void __launch_bounds__(P * P) sem_ax_kernel(const int32_t* __restrict__ l2g, const double* __restrict__ G,
                                                      const double* __restrict__ Dg, const double* __restrict__ x,
                                                      double* __restrict__ y) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ double sD[P][P];        // sD[a][b] = D[a][b] = l_b'(x_a)
    __shared__ double su[P][P][P];     // u[k][j][i]
    __shared__ double sr[P][P][P];     // G-weighted r-gradient
    __shared__ double ss[P][P][P];     // G-weighted s-gradient
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    sD[j][i] = Dg[j * P + i];
    const int32_t* L = l2g + (size_t)e * P3;
    int32_t gk[P];
    double uk[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        gk[k] = __ldg(&L[k * P2 + j * P + i]);
        uk[k] = gather(x, gk[k]);
        su[k][j][i] = uk[k];
    }
    __syncthreads();
    const double* Ge = G + (size_t)e * 6 * P3;
    double wt[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) {
            ur = fma(sD[i][m], su[k][j][m], ur);
            us = fma(sD[j][m], su[k][m][i], us);
            ut = fma(sD[k][m], uk[m], ut);
        }
        const int node = k * P2 + j * P + i;
        const double g00 = __ldg(&Ge[node]), g01 = __ldg(&Ge[P3 + node]), g02 = __ldg(&Ge[2 * P3 + node]);
        const double g11 = __ldg(&Ge[3 * P3 + node]), g12 = __ldg(&Ge[4 * P3 + node]), g22 = __ldg(&Ge[5 * P3 + node]);
        sr[k][j][i] = g00 * ur + g01 * us + g02 * ut;
        ss[k][j][i] = g01 * ur + g11 * us + g12 * ut;
        wt[k] = g02 * ur + g12 * us + g22 * ut;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double v = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) {
            v = fma(sD[m][i], sr[k][j][m], v);
            v = fma(sD[m][j], ss[k][m][i], v);
            v = fma(sD[m][k], wt[m], v);
        }
        if (gk[k] >= 0) atomicAdd(&y[gk[k]], v);
    }
}

// Float-pair ("double-float") arithmetic of the mixed forms' operator: a
// value is hi + lo (about 48 bits); products by the FMA-based two-product,
// sums by Knuth's two-sum (published error-free transformations).
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (a.x + a.y)(b.x + b.y) ~= ph + pl (the lo * lo term dropped)
__device__ __forceinline__ void pmul(float2 a, float2 b, float& ph, float& pl) {
    ph = __fmul_rn(a.x, b.x);
    pl = __fmaf_rn(a.x, b.x, -ph);
    pl = __fmaf_rn(a.x, b.y, pl);
    pl = __fmaf_rn(a.y, b.x, pl);
}
// (yh, yl) += a b, the low word left unnormalised
__device__ __forceinline__ void pmad(float2 a, float2 b, float& yh, float& yl) {
    float ph, pl, s, e;
    pmul(a, b, ph, pl);
    two_sum_f(yh, ph, s, e);
    yh = s;
    yl = __fadd_rn(yl, __fadd_rn(e, pl));
}
__device__ __forceinline__ float2 pnorm(float h, float l) {
    const float s = __fadd_rn(h, l);
    return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}
__device__ __forceinline__ float2 psplit(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// y += A_n x with the metric and D as float pairs and every product and sum
// in pair arithmetic on the FP32 pipes (about 2^-44 of the sum of the
// terms' magnitudes), x read and y accumulated in float64: the operator of
// the mixed forms, where float64 arithmetic (two FMAs per clock per SM on
// B300) would bound the whole solve.
template <int P>
__global__ void __launch_bounds__(P * P) sem_ax_pair_kernel(const int32_t* __restrict__ l2g,
                                                           const float2* __restrict__ G,
                                                           const float2* __restrict__ Dg,
                                                           const double* __restrict__ x, double* __restrict__ y) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ float2 sD[P][P];
    __shared__ float2 su[P][P][P];
    __shared__ float2 sr[P][P][P];
    __shared__ float2 ss[P][P][P];
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    sD[j][i] = Dg[j * P + i];
    const int32_t* L = l2g + (size_t)e * P3;
    int32_t gk[P];
    float2 uk[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        gk[k] = __ldg(&L[k * P2 + j * P + i]);
        uk[k] = gk[k] >= 0 ? psplit(__ldg(&x[gk[k]])) : make_float2(0.0f, 0.0f);
        su[k][j][i] = uk[k];
    }
    __syncthreads();
    const float2* Ge = G + (size_t)e * 6 * P3;
    float2 wt[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        float rh = 0.f, rl = 0.f, sh = 0.f, sl = 0.f, th = 0.f, tl = 0.f;
#pragma unroll
        for (int m = 0; m < P; ++m) {
            pmad(sD[i][m], su[k][j][m], rh, rl);
            pmad(sD[j][m], su[k][m][i], sh, sl);
            pmad(sD[k][m], uk[m], th, tl);
        }
        const float2 ur = pnorm(rh, rl), us = pnorm(sh, sl), ut = pnorm(th, tl);
        const int node = k * P2 + j * P + i;
        const float2 g00 = __ldg(&Ge[node]), g01 = __ldg(&Ge[P3 + node]), g02 = __ldg(&Ge[2 * P3 + node]);
        const float2 g11 = __ldg(&Ge[3 * P3 + node]), g12 = __ldg(&Ge[4 * P3 + node]), g22 = __ldg(&Ge[5 * P3 + node]);
        float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f, ch = 0.f, cl = 0.f;
        pmad(g00, ur, ah, al);
        pmad(g01, us, ah, al);
        pmad(g02, ut, ah, al);
        pmad(g01, ur, bh, bl);
        pmad(g11, us, bh, bl);
        pmad(g12, ut, bh, bl);
        pmad(g02, ur, ch, cl);
        pmad(g12, us, ch, cl);
        pmad(g22, ut, ch, cl);
        sr[k][j][i] = pnorm(ah, al);
        ss[k][j][i] = pnorm(bh, bl);
        wt[k] = pnorm(ch, cl);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        float vh = 0.f, vl = 0.f;
#pragma unroll
        for (int m = 0; m < P; ++m) {
            pmad(sD[m][i], sr[k][j][m], vh, vl);
            pmad(sD[m][j], ss[k][m][i], vh, vl);
            pmad(sD[m][k], wt[m], vh, vl);
        }
        if (gk[k] >= 0) atomicAdd(&y[gk[k]], (double)vh + (double)vl);
    }
}

__device__ __forceinline__ double mad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <class T, class V>
__device__ __forceinline__ T load_as(const V* __restrict__ v, int32_t g) {
    return g >= 0 ? (T)__ldg(&v[g]) : T(0);
}

// z += W sum_e R_e^T S_e (lam_x + lam_y + lam_z)^-1 S_e^T R_e r, arithmetic in
// T (float64, or float for the mixed forms' preconditioner), vectors in V
template <int P, class T, class V>
__global__ void __launch_bounds__(P * P) sem_fdm_kernel(const int32_t* __restrict__ l2g, const T* __restrict__ S,
                                                       const T* __restrict__ lam, const T* __restrict__ inv_mult,
                                                       const V* __restrict__ r, V* __restrict__ z) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ T sS[3][P][P];     // S_d[node][mode]
    __shared__ T sl[3][P];
    __shared__ T sx[P][P][P];
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    const T* Se = S + (size_t)e * 3 * P2;
#pragma unroll
    for (int d = 0; d < 3; ++d) sS[d][j][i] = __ldg(&Se[d * P2 + j * P + i]);
    if (threadIdx.x < 3 * P) sl[threadIdx.x / P][threadIdx.x % P] = __ldg(&lam[(size_t)e * 3 * P + threadIdx.x]);
    const int32_t* L = l2g + (size_t)e * P3;
    int32_t gk[P];
    T a[P], b[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        gk[k] = __ldg(&L[k * P2 + j * P + i]);
        a[k] = load_as<T>(r, gk[k]);
    }
    __syncthreads();
    // S_z^T along k (registers)
#pragma unroll
    for (int k = 0; k < P; ++k) {
        T t = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = mad(sS[2][m][k], a[m], t);
        b[k] = t;
    }
    // S_y^T along j
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = b[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        T t = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = mad(sS[1][m][j], sx[k][m][i], t);
        a[k] = t;
    }
    __syncthreads();
    // S_x^T along i, then the diagonal
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = a[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        T t = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = mad(sS[0][m][i], sx[k][j][m], t);
        b[k] = t / (sl[0][i] + sl[1][j] + sl[2][k]);
    }
    __syncthreads();
    // back: S_x along i
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = b[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        T t = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = mad(sS[0][i][m], sx[k][j][m], t);
        a[k] = t;
    }
    __syncthreads();
    // S_y along j
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = a[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        T t = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = mad(sS[1][j][m], sx[k][m][i], t);
        b[k] = t;
    }
    // S_z along k, then W and the scatter
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (gk[k] < 0) continue;
        T t = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = mad(sS[2][k][m], b[m], t);
        atomicAdd(&z[gk[k]], (V)(__ldg(&inv_mult[gk[k]]) * t));
    }
}

// r_c += Q_c^T I^T Q_f W_f r_f over one element: the fine block is p x p
// threads, the coarse element has pc <= P nodes per direction
template <int P, class T, class VF, class VC>
__global__ void __launch_bounds__(P * P) sem_restrict_kernel(const int32_t* __restrict__ l2g_f,
                                                            const T* __restrict__ inv_mult_f,
                                                            const T* __restrict__ Ig, int pc,
                                                            const int32_t* __restrict__ l2g_c,
                                                            const VF* __restrict__ rf, VC* __restrict__ rc) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ T sI[P][P];        // sI[fine][coarse]
    __shared__ T s1[P][P][P];     // [kc][j][i]
    __shared__ T s2[P][P][P];     // [kc][jc][i]
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    if (i < pc) sI[j][i] = __ldg(&Ig[j * pc + i]);
    const int32_t* L = l2g_f + (size_t)e * P3;
    T a[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int32_t g = __ldg(&L[k * P2 + j * P + i]);
        a[k] = g >= 0 ? (T)__ldg(&rf[g]) * __ldg(&inv_mult_f[g]) : T(0);
    }
    __syncthreads();
    // I^T along k
#pragma unroll
    for (int kc = 0; kc < P; ++kc) {
        if (kc >= pc) break;
        T t = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) t = mad(sI[k][kc], a[k], t);
        s1[kc][j][i] = t;
    }
    __syncthreads();
    // I^T along j: thread (i, jc) for jc < pc
    if (j < pc) {
        for (int kc = 0; kc < pc; ++kc) {
            T t = 0;
#pragma unroll
            for (int m = 0; m < P; ++m) t = mad(sI[m][j], s1[kc][m][i], t);
            s2[kc][j][i] = t;
        }
    }
    __syncthreads();
    // I^T along i: thread (ic, jc)
    if (i < pc && j < pc) {
        const int pc2 = pc * pc;
        const int32_t* Lc = l2g_c + (size_t)e * pc2 * pc;
        for (int kc = 0; kc < pc; ++kc) {
            T t = 0;
#pragma unroll
            for (int m = 0; m < P; ++m) t = mad(sI[m][i], s2[kc][j][m], t);
            const int32_t g = __ldg(&Lc[kc * pc2 + j * pc + i]);
            if (g >= 0) atomicAdd(&rc[g], (VC)t);
        }
    }
}

// z_f += W_f Q_f^T I Q_c u_c over one element
template <int P, class T, class VC, class VF>
__global__ void __launch_bounds__(P * P) sem_prolong_kernel(const int32_t* __restrict__ l2g_f,
                                                           const T* __restrict__ inv_mult_f,
                                                           const T* __restrict__ Ig, int pc,
                                                           const int32_t* __restrict__ l2g_c,
                                                           const VC* __restrict__ uc, VF* __restrict__ zf) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ T sI[P][P];        // sI[fine][coarse]
    __shared__ T sc[P][P][P];     // coarse values [kc][jc][ic]
    __shared__ T s1[P][P][P];     // [kc][jc][i]
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    if (i < pc) sI[j][i] = __ldg(&Ig[j * pc + i]);
    const int pc2 = pc * pc;
    const int32_t* Lc = l2g_c + (size_t)e * pc2 * pc;
    for (int q = threadIdx.x; q < pc2 * pc; q += P2) {
        const int kc = q / pc2, jc = (q / pc) % pc, ic = q % pc;
        sc[kc][jc][ic] = load_as<T>(uc, __ldg(&Lc[q]));
    }
    __syncthreads();
    // I along i: thread (i, jc)
    if (j < pc) {
        for (int kc = 0; kc < pc; ++kc) {
            T t = 0;
            for (int m = 0; m < pc; ++m) t = mad(sI[i][m], sc[kc][j][m], t);
            s1[kc][j][i] = t;
        }
    }
    __syncthreads();
    // I along j (registers over kc), then along k
    T b[P];
#pragma unroll
    for (int kc = 0; kc < P; ++kc) {
        T t = 0;
        if (kc < pc)
            for (int m = 0; m < pc; ++m) t = mad(sI[j][m], s1[kc][m][i], t);
        b[kc] = t;
    }
    const int32_t* L = l2g_f + (size_t)e * P3;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int32_t g = __ldg(&L[k * P2 + j * P + i]);
        if (g < 0) continue;
        T t = 0;
#pragma unroll
        for (int m = 0; m < P; ++m)
            if (m < pc) t = mad(sI[k][m], b[m], t);
        atomicAdd(&zf[g], (VF)(__ldg(&inv_mult_f[g]) * t));
    }
}

#define SEM_DISPATCH(p, KERNEL, ...)                                                   \
    switch (p) {                                                                       \
        case 3: KERNEL<3><<<grid, 9, 0, st>>>(__VA_ARGS__); break;                      \
        case 4: KERNEL<4><<<grid, 16, 0, st>>>(__VA_ARGS__); break;                     \
        case 5: KERNEL<5><<<grid, 25, 0, st>>>(__VA_ARGS__); break;                     \
        case 6: KERNEL<6><<<grid, 36, 0, st>>>(__VA_ARGS__); break;                     \
        case 7: KERNEL<7><<<grid, 49, 0, st>>>(__VA_ARGS__); break;                     \
        case 8: KERNEL<8><<<grid, 64, 0, st>>>(__VA_ARGS__); break;                     \
        case 9: KERNEL<9><<<grid, 81, 0, st>>>(__VA_ARGS__); break;                     \
        default: break;                                                                \
    }
// one launch per supported p (orders 2..8)
#define SEM_CASES(p, LAUNCH)                                                           \
    switch (p) {                                                                       \
        case 3: LAUNCH(3); break;                                                      \
        case 4: LAUNCH(4); break;                                                      \
        case 5: LAUNCH(5); break;                                                      \
        case 6: LAUNCH(6); break;                                                      \
        case 7: LAUNCH(7); break;                                                      \
        case 8: LAUNCH(8); break;                                                      \
        case 9: LAUNCH(9); break;                                                      \
        default: break;                                                                \
    }

}  // namespace

void launch_sem_ax(const SemDevLevel& L, int64_t ne, const double* x, double* y, cudaStream_t st) {
    if (ne == 0) return;
    const dim3 grid((unsigned)ne);
    if (L.Gp) {
        SEM_DISPATCH(L.p, sem_ax_pair_kernel, L.l2g, L.Gp, L.Dp, x, y);
    } else {
        SEM_DISPATCH(L.p, sem_ax_kernel, L.l2g, L.G, L.D, x, y);
    }
}

namespace {

template <class T, class V>
void fdm_typed(const SemDevLevel& L, int64_t ne, const T* S, const T* lam, const T* w, const void* r, void* z,
               cudaStream_t st) {
    const dim3 grid((unsigned)ne);
    const V* rv = static_cast<const V*>(r);
    V* zv = static_cast<V*>(z);
#define SEM_FDM(p) sem_fdm_kernel<p, T, V><<<grid, p * p, 0, st>>>(L.l2g, S, lam, w, rv, zv)
    SEM_CASES(L.p, SEM_FDM)
#undef SEM_FDM
}

}  // namespace

void launch_sem_fdm(const SemDevLevel& L, int64_t ne, const void* r, void* z, bool vec_f32, cudaStream_t st) {
    if (ne == 0) return;
    if (!L.f32)
        fdm_typed<double, double>(L, ne, L.S, L.lam, L.inv_mult, r, z, st);
    else if (vec_f32)
        fdm_typed<float, float>(L, ne, L.S32, L.lam32, L.inv_mult32, r, z, st);
    else
        fdm_typed<float, double>(L, ne, L.S32, L.lam32, L.inv_mult32, r, z, st);
}

namespace {

template <class T, class VF, class VC>
void transfer_typed(bool restrict_, const SemDevLevel& F, const T* w, const T* I, int pc, const int32_t* l2g_c,
                    int64_t ne, const void* in, void* out, cudaStream_t st) {
    const dim3 grid((unsigned)ne);
    if (restrict_) {
        const VF* a = static_cast<const VF*>(in);
        VC* b = static_cast<VC*>(out);
#define SEM_R(p) sem_restrict_kernel<p, T, VF, VC><<<grid, p * p, 0, st>>>(F.l2g, w, I, pc, l2g_c, a, b)
        SEM_CASES(F.p, SEM_R)
#undef SEM_R
    } else {
        const VC* a = static_cast<const VC*>(in);
        VF* b = static_cast<VF*>(out);
#define SEM_P(p) sem_prolong_kernel<p, T, VC, VF><<<grid, p * p, 0, st>>>(F.l2g, w, I, pc, l2g_c, a, b)
        SEM_CASES(F.p, SEM_P)
#undef SEM_P
    }
}

void transfer(bool restrict_, const SemDevLevel& F, int pc, const int32_t* l2g_c, int64_t ne, const void* in,
              void* out, bool f_f32, bool c_f32, cudaStream_t st) {
    if (ne == 0) return;
    if (!F.f32) {
        transfer_typed<double, double, double>(restrict_, F, F.inv_mult, F.I_next, pc, l2g_c, ne, in, out, st);
        return;
    }
    const float* w = F.inv_mult32;
    const float* I = F.I_next32;
    if (!f_f32 && !c_f32)
        transfer_typed<float, double, double>(restrict_, F, w, I, pc, l2g_c, ne, in, out, st);
    else if (!f_f32 && c_f32)
        transfer_typed<float, double, float>(restrict_, F, w, I, pc, l2g_c, ne, in, out, st);
    else if (f_f32 && c_f32)
        transfer_typed<float, float, float>(restrict_, F, w, I, pc, l2g_c, ne, in, out, st);
    else
        transfer_typed<float, float, double>(restrict_, F, w, I, pc, l2g_c, ne, in, out, st);
}

}  // namespace

void launch_sem_restrict(const SemDevLevel& F, int pc, const int32_t* l2g_c, int64_t ne, const void* rf, void* rc,
                         bool f_f32, bool c_f32, cudaStream_t st) {
    transfer(true, F, pc, l2g_c, ne, rf, rc, f_f32, c_f32, st);
}

void launch_sem_prolong(const SemDevLevel& F, int pc, const int32_t* l2g_c, int64_t ne, const void* uc, void* zf,
                        bool c_f32, bool f_f32, cudaStream_t st) {
    transfer(false, F, pc, l2g_c, ne, uc, zf, f_f32, c_f32, st);
}

}  // namespace cgs
