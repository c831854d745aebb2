// Kernels of the p-multigrid wrap's spectral-element levels (Sec. 1, Sec. 5,
// Eqs. (13) and (14)), float64, one block of p x p threads per element:
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
// input and never written.  Scatters are float64 atomic adds (the order of
// the additions, and so the last bits, varies from run to run).
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

// z += W sum_e R_e^T S_e (lam_x + lam_y + lam_z)^-1 S_e^T R_e r
template <int P>
__global__ void __launch_bounds__(P * P) sem_fdm_kernel(const int32_t* __restrict__ l2g, const double* __restrict__ S,
                                                       const double* __restrict__ lam,
                                                       const double* __restrict__ inv_mult,
                                                       const double* __restrict__ r, double* __restrict__ z) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ double sS[3][P][P];     // S_d[node][mode]
    __shared__ double sl[3][P];
    __shared__ double sx[P][P][P];
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    const double* Se = S + (size_t)e * 3 * P2;
#pragma unroll
    for (int d = 0; d < 3; ++d) sS[d][j][i] = __ldg(&Se[d * P2 + j * P + i]);
    if (threadIdx.x < 3 * P) sl[threadIdx.x / P][threadIdx.x % P] = __ldg(&lam[(size_t)e * 3 * P + threadIdx.x]);
    const int32_t* L = l2g + (size_t)e * P3;
    int32_t gk[P];
    double a[P], b[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        gk[k] = __ldg(&L[k * P2 + j * P + i]);
        a[k] = gather(r, gk[k]);
    }
    __syncthreads();
    // S_z^T along k (registers)
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = fma(sS[2][m][k], a[m], t);
        b[k] = t;
    }
    // S_y^T along j
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = b[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = fma(sS[1][m][j], sx[k][m][i], t);
        a[k] = t;
    }
    __syncthreads();
    // S_x^T along i, then the diagonal
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = a[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = fma(sS[0][m][i], sx[k][j][m], t);
        b[k] = t / (sl[0][i] + sl[1][j] + sl[2][k]);
    }
    __syncthreads();
    // back: S_x along i
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = b[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = fma(sS[0][i][m], sx[k][j][m], t);
        a[k] = t;
    }
    __syncthreads();
    // S_y along j
#pragma unroll
    for (int k = 0; k < P; ++k) sx[k][j][i] = a[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = fma(sS[1][j][m], sx[k][m][i], t);
        b[k] = t;
    }
    // S_z along k, then W and the scatter
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (gk[k] < 0) continue;
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m) t = fma(sS[2][k][m], b[m], t);
        atomicAdd(&z[gk[k]], __ldg(&inv_mult[gk[k]]) * t);
    }
}

// r_c += Q_c^T I^T Q_f W_f r_f over one element: the fine block is p x p
// threads, the coarse element has pc <= P nodes per direction
template <int P>
__global__ void __launch_bounds__(P * P) sem_restrict_kernel(const int32_t* __restrict__ l2g_f,
                                                            const double* __restrict__ inv_mult_f,
                                                            const double* __restrict__ Ig, int pc,
                                                            const int32_t* __restrict__ l2g_c,
                                                            const double* __restrict__ rf, double* __restrict__ rc) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ double sI[P][P];        // sI[fine][coarse]
    __shared__ double s1[P][P][P];     // [kc][j][i]
    __shared__ double s2[P][P][P];     // [kc][jc][i]
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    if (i < pc) sI[j][i] = __ldg(&Ig[j * pc + i]);
    const int32_t* L = l2g_f + (size_t)e * P3;
    double a[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int32_t g = __ldg(&L[k * P2 + j * P + i]);
        a[k] = g >= 0 ? __ldg(&rf[g]) * __ldg(&inv_mult_f[g]) : 0.0;
    }
    __syncthreads();
    // I^T along k
#pragma unroll
    for (int kc = 0; kc < P; ++kc) {
        if (kc >= pc) break;
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < P; ++k) t = fma(sI[k][kc], a[k], t);
        s1[kc][j][i] = t;
    }
    __syncthreads();
    // I^T along j: thread (i, jc) for jc < pc
    if (j < pc) {
        for (int kc = 0; kc < pc; ++kc) {
            double t = 0.0;
#pragma unroll
            for (int m = 0; m < P; ++m) t = fma(sI[m][j], s1[kc][m][i], t);
            s2[kc][j][i] = t;
        }
    }
    __syncthreads();
    // I^T along i: thread (ic, jc)
    if (i < pc && j < pc) {
        const int pc2 = pc * pc;
        const int32_t* Lc = l2g_c + (size_t)e * pc2 * pc;
        for (int kc = 0; kc < pc; ++kc) {
            double t = 0.0;
#pragma unroll
            for (int m = 0; m < P; ++m) t = fma(sI[m][i], s2[kc][j][m], t);
            const int32_t g = __ldg(&Lc[kc * pc2 + j * pc + i]);
            if (g >= 0) atomicAdd(&rc[g], t);
        }
    }
}

// z_f += W_f Q_f^T I Q_c u_c over one element
template <int P>
__global__ void __launch_bounds__(P * P) sem_prolong_kernel(const int32_t* __restrict__ l2g_f,
                                                           const double* __restrict__ inv_mult_f,
                                                           const double* __restrict__ Ig, int pc,
                                                           const int32_t* __restrict__ l2g_c,
                                                           const double* __restrict__ uc, double* __restrict__ zf) {
    constexpr int P2 = P * P, P3 = P * P * P;
    __shared__ double sI[P][P];        // sI[fine][coarse]
    __shared__ double sc[P][P][P];     // coarse values [kc][jc][ic]
    __shared__ double s1[P][P][P];     // [kc][jc][i]
    const int e = blockIdx.x;
    const int i = threadIdx.x % P, j = threadIdx.x / P;
    if (i < pc) sI[j][i] = __ldg(&Ig[j * pc + i]);
    const int pc2 = pc * pc;
    const int32_t* Lc = l2g_c + (size_t)e * pc2 * pc;
    for (int q = threadIdx.x; q < pc2 * pc; q += P2) {
        const int kc = q / pc2, jc = (q / pc) % pc, ic = q % pc;
        sc[kc][jc][ic] = gather(uc, __ldg(&Lc[q]));
    }
    __syncthreads();
    // I along i: thread (i, jc)
    if (j < pc) {
        for (int kc = 0; kc < pc; ++kc) {
            double t = 0.0;
            for (int m = 0; m < pc; ++m) t = fma(sI[i][m], sc[kc][j][m], t);
            s1[kc][j][i] = t;
        }
    }
    __syncthreads();
    // I along j (registers over kc), then along k
    double b[P];
#pragma unroll
    for (int kc = 0; kc < P; ++kc) {
        double t = 0.0;
        if (kc < pc)
            for (int m = 0; m < pc; ++m) t = fma(sI[j][m], s1[kc][m][i], t);
        b[kc] = t;
    }
    const int32_t* L = l2g_f + (size_t)e * P3;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int32_t g = __ldg(&L[k * P2 + j * P + i]);
        if (g < 0) continue;
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < P; ++m)
            if (m < pc) t = fma(sI[k][m], b[m], t);
        atomicAdd(&zf[g], __ldg(&inv_mult_f[g]) * t);
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

}  // namespace

void launch_sem_ax(const SemDevLevel& L, int64_t ne, const double* x, double* y, cudaStream_t st) {
    if (ne == 0) return;
    const dim3 grid((unsigned)ne);
    SEM_DISPATCH(L.p, sem_ax_kernel, L.l2g, L.G, L.D, x, y);
}

void launch_sem_fdm(const SemDevLevel& L, int64_t ne, const double* r, double* z, cudaStream_t st) {
    if (ne == 0) return;
    const dim3 grid((unsigned)ne);
    SEM_DISPATCH(L.p, sem_fdm_kernel, L.l2g, L.S, L.lam, L.inv_mult, r, z);
}

void launch_sem_restrict(const SemDevLevel& F, int pc, const int32_t* l2g_c, int64_t ne, const double* rf,
                         double* rc, cudaStream_t st) {
    if (ne == 0) return;
    const dim3 grid((unsigned)ne);
    SEM_DISPATCH(F.p, sem_restrict_kernel, F.l2g, F.inv_mult, F.I_next, pc, l2g_c, rf, rc);
}

void launch_sem_prolong(const SemDevLevel& F, int pc, const int32_t* l2g_c, int64_t ne, const double* uc,
                        double* zf, cudaStream_t st) {
    if (ne == 0) return;
    const dim3 grid((unsigned)ne);
    SEM_DISPATCH(F.p, sem_prolong_kernel, F.l2g, F.inv_mult, F.I_next, pc, l2g_c, uc, zf);
}

}  // namespace cgs
