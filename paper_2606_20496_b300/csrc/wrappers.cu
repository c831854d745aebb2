// Outer iterations other than the flexible PCG, around the same two-level
// Schwarz preconditioner: Schwarz-Richardson, x += M (b - A x), and flexible
// GMRES(restart), right-preconditioned with the preconditioned directions
// kept (so M may vary between steps, as the inexact local solves of Sec. 6
// make it).  The paper solves the coarse problem inside GMRES-wrapped pMG and
// names Schwarz-Richardson as the alternative wrapper (Sec. 3).
//
// Everything runs on the device in float64 through the library's own
// kernels: the operator (cgs_apply_A), the preconditioner in the mesh's form
// and precision (cgs_apply_preconditioner), and the dot-product and
// combination kernels of the projection (deterministic block sums).  The
// host keeps the (restart + 1) x restart Hessenberg matrix, its Givens
// rotations and the least-squares solve, and reads a few scalars per step.
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"
#include "krylov.h"

using namespace cgs;

namespace {

// Device buffers of one wrapped solve, freed together.
struct Buffers {
    std::vector<void*> ptrs;
    cudaError_t alloc(double** p, size_t n) {
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(double));
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = static_cast<double*>(q);
        }
        return e;
    }
    ~Buffers() {
        for (void* q : ptrs) cudaFree(q);
    }
};

cgs_status cuda_status(cudaError_t e, const char* where) {
    set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CGS_ERR_OOM : CGS_ERR_CUDA;
}

#define WRAP_CUDA(call)                                         \
    do {                                                        \
        const cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_status(e_, #call);   \
    } while (0)
#define WRAP_OK(call)                                           \
    do {                                                        \
        const cgs_status s_ = (call);                           \
        if (s_ != CGS_OK) return s_;                            \
    } while (0)

// Scalars the host needs: out[0..k] of a dot-product launch.
struct Dots {
    double* partial = nullptr;   // proj_partial_entries(kmax) doubles
    double* out = nullptr;       // kmax + 2 doubles (device): the dots, then one more slot
    std::vector<double> host;
};

// host copy of X_j . v (j < k) and v . v, Dirichlet entries of v as zero
cgs_status dots(Dots& D, const double* X, int k, int64_t n, const double* v, const uint8_t* dir, cudaStream_t st) {
    launch_proj_dots(X, k, n, v, dir, D.partial, D.out, st);
    D.host.resize(k + 1);
    WRAP_CUDA(cudaMemcpyAsync(D.host.data(), D.out, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
    WRAP_CUDA(cudaStreamSynchronize(st));
    return CGS_OK;
}

}  // namespace

namespace cgs {

size_t fgmres_work_doubles(int64_t n, int restart) {
    const size_t kmax = (size_t)restart + 1;
    // every piece rounded up to 32 doubles (256-byte alignment)
    auto r32 = [](size_t x) { return (x + 31) / 32 * 32; };
    return r32(proj_partial_entries((int)kmax)) + r32(kmax + 2) + 3 * r32((size_t)n) + r32(1) + r32(kmax) +
           r32((size_t)(restart + 1) * n) + r32((size_t)restart * n);
}

cgs_status fgmres_device(const KrylovOps& ops, const double* b, double* x, double rtol, int maxit, int restart,
                         int* iters, double* relres, cudaStream_t st) {
    *iters = 0;
    *relres = 0.0;
    const int64_t n = ops.n;
    const uint8_t* dir = ops.dir;
    const int kmax = restart + 1;
    Buffers buf;
    Dots D;
    double *bm, *r, *one, *coef, *V, *Z, *w;
    if (ops.work && ops.work_doubles >= fgmres_work_doubles(n, restart)) {
        auto r32 = [](size_t v) { return (v + 31) / 32 * 32; };
        double* p = ops.work;
        auto take = [&](double** q, size_t cnt) {
            *q = p;
            p += r32(cnt);
        };
        take(&D.partial, proj_partial_entries(kmax));
        take(&D.out, kmax + 2);
        take(&bm, n);
        take(&r, n);
        take(&w, n);
        take(&one, 1);
        take(&coef, kmax);
        take(&V, (size_t)(restart + 1) * n);
        take(&Z, (size_t)restart * n);
    } else {
        WRAP_CUDA(buf.alloc(&D.partial, proj_partial_entries(kmax)));
        WRAP_CUDA(buf.alloc(&D.out, kmax + 2));
        WRAP_CUDA(buf.alloc(&bm, n));
        WRAP_CUDA(buf.alloc(&r, n));
        WRAP_CUDA(buf.alloc(&one, 1));
        WRAP_CUDA(buf.alloc(&coef, kmax));
        WRAP_CUDA(buf.alloc(&V, (size_t)(restart + 1) * n));
        WRAP_CUDA(buf.alloc(&Z, (size_t)restart * n));
        WRAP_CUDA(buf.alloc(&w, n));
    }
    const double h_one = 1.0;
    WRAP_CUDA(cudaMemcpyAsync(one, &h_one, sizeof(double), cudaMemcpyHostToDevice, st));
    // b with its Dirichlet entries zeroed, x = 0
    launch_proj_combine(n, b, dir, 0.0, one, 0, nullptr, bm, st);
    WRAP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    WRAP_OK(dots(D, nullptr, 0, n, bm, dir, st));
    const double nb = std::sqrt(D.host[0]);
    if (nb == 0.0) return CGS_OK;
    const int m = restart;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), yv(m);
    auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    int its = 0;
    cgs_status result = CGS_ERR_NO_CONVERGENCE;
    for (;;) {
        // r = bm - A x
        WRAP_OK(ops.apply_A(x, w));
        launch_proj_combine(n, bm, dir, -1.0, one, 1, w, r, st);
        WRAP_OK(dots(D, nullptr, 0, n, r, dir, st));
        const double beta = std::sqrt(D.host[0]);
        *relres = beta / nb;
        *iters = its;
        if (!std::isfinite(beta)) {
            result = CGS_ERR_BREAKDOWN;
            break;
        }
        if (beta <= rtol * nb) {
            result = CGS_OK;
            break;
        }
        if (its >= maxit) break;
        launch_proj_combine(n, nullptr, dir, 1.0 / beta, one, 1, r, V, st);
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int used = 0;
        bool breakdown = false;
        for (int j = 0; j < m; ++j) {
            double* Vj = V + (size_t)j * n;
            double* Zj = Z + (size_t)j * n;
            WRAP_OK(ops.apply_M(Vj, Zj));
            WRAP_OK(ops.apply_A(Zj, w));
            ++its;
            // classical Gram-Schmidt against V_0..V_j, repeated once when the
            // first pass cancels more than half of w's norm (the
            // Daniel-Gragg-Kaufman-Stewart test, eta = 1/sqrt(2)); each pass is
            // the dots (with ||w||^2 before) and the correction (with ||w||^2
            // after)
            // (the dots stay on the device as the correction's coefficients;
            // they and ||w||^2 after come back in one copy, one wait per pass)
            double hn = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                launch_proj_dots(V, j + 1, n, w, dir, D.partial, D.out, st);
                launch_gs_update(V, j + 1, n, D.out, dir, w, D.partial, D.out + (j + 2), false, st);
                D.host.resize(j + 3);
                WRAP_CUDA(cudaMemcpyAsync(D.host.data(), D.out, sizeof(double) * (j + 3), cudaMemcpyDeviceToHost,
                                          st));
                WRAP_CUDA(cudaStreamSynchronize(st));
                for (int i = 0; i <= j; ++i) Hij(i, j) += D.host[i];
                const double before = D.host[j + 1], after = D.host[j + 2];
                hn = std::sqrt(after);
                if (!(after < 0.5 * before)) break;
            }
            Hij(j + 1, j) = hn;
            if (!std::isfinite(hn)) {
                breakdown = true;
                break;
            }
            // previous rotations on column j, then the new one
            for (int i = 0; i < j; ++i) {
                const double a = Hij(i, j), c = Hij(i + 1, j);
                Hij(i, j) = cs[i] * a + sn[i] * c;
                Hij(i + 1, j) = -sn[i] * a + cs[i] * c;
            }
            const double a = Hij(j, j), c = Hij(j + 1, j), rho = std::hypot(a, c);
            cs[j] = rho > 0.0 ? a / rho : 1.0;
            sn[j] = rho > 0.0 ? c / rho : 0.0;
            Hij(j, j) = rho;
            Hij(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            used = j + 1;
            if (std::fabs(g[j + 1]) <= rtol * nb || its >= maxit || hn == 0.0) break;
            launch_proj_combine(n, nullptr, dir, 1.0 / hn, one, 1, w, V + (size_t)(j + 1) * n, st);
        }
        if (breakdown) {
            result = CGS_ERR_BREAKDOWN;
            break;
        }
        // y = R^{-1} g by back substitution, x += Z y
        for (int i = used - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < used; ++k) s -= Hij(i, k) * yv[k];
            yv[i] = Hij(i, i) != 0.0 ? s / Hij(i, i) : 0.0;
        }
        WRAP_CUDA(cudaMemcpyAsync(coef, yv.data(), sizeof(double) * used, cudaMemcpyHostToDevice, st));
        launch_proj_combine(n, x, dir, 1.0, coef, used, Z, x, st);
    }
    WRAP_CUDA(cudaStreamSynchronize(st));
    WRAP_CUDA(cudaGetLastError());
    if (result == CGS_ERR_NO_CONVERGENCE) set_last_error("maxit reached before the tolerance");
    if (result == CGS_ERR_BREAKDOWN) set_last_error("non-finite value in the wrapped iteration");
    return result;
}

}  // namespace cgs

extern "C" cgs_status cgs_solve_wrapped(cgs_mesh* mesh, const double* b, double* x, cgs_method method, double rtol,
                                        int maxit, int restart, int* iters, double* relres, void* stream) {
    if (!mesh || !b || !x || !iters || !relres || maxit < 0 || !(rtol > 0.0)) {
        set_last_error("null argument, negative maxit or non-positive rtol");
        return CGS_ERR_INVALID_ARG;
    }
    if (method == CGS_METHOD_PCG) return cgs_solve(mesh, b, x, 1, rtol, maxit, iters, relres, stream);
    if (method != CGS_METHOD_RICHARDSON && method != CGS_METHOD_FGMRES) {
        set_last_error("unknown method");
        return CGS_ERR_INVALID_ARG;
    }
    if (method == CGS_METHOD_FGMRES && (restart < 1 || restart > 1024)) {
        set_last_error("restart must be in [1, 1024]");
        return CGS_ERR_INVALID_ARG;
    }
    *iters = 0;
    *relres = 0.0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WRAP_CUDA(cudaSetDevice(mesh_device(mesh)));
    const int64_t n = mesh_dev(mesh).nv;
    const uint8_t* dir = mesh_dir(mesh);
    cgs_status result = CGS_ERR_NO_CONVERGENCE;
    if (method == CGS_METHOD_FGMRES) {
        KrylovOps ops;
        ops.n = n;
        ops.dir = dir;
        ops.apply_A = [&](const double* u, double* y) { return cgs_apply_A(mesh, u, y, stream); };
        ops.apply_M = [&](const double* r, double* z) { return cgs_apply_preconditioner(mesh, r, z, stream); };
        result = fgmres_device(ops, b, x, rtol, maxit, restart, iters, relres, st);
        if (result != CGS_OK && result != CGS_ERR_NO_CONVERGENCE && result != CGS_ERR_BREAKDOWN) return result;
    } else {
        Buffers buf;
        Dots D;
        double *bm, *r, *y, *one;
        WRAP_CUDA(buf.alloc(&D.partial, proj_partial_entries(1)));
        WRAP_CUDA(buf.alloc(&D.out, 2));
        WRAP_CUDA(buf.alloc(&bm, n));
        WRAP_CUDA(buf.alloc(&r, n));
        WRAP_CUDA(buf.alloc(&y, n));
        WRAP_CUDA(buf.alloc(&one, 1));
        const double h_one = 1.0;
        WRAP_CUDA(cudaMemcpyAsync(one, &h_one, sizeof(double), cudaMemcpyHostToDevice, st));
        launch_proj_combine(n, b, dir, 0.0, one, 0, nullptr, bm, st);
        WRAP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
        WRAP_OK(dots(D, nullptr, 0, n, bm, dir, st));
        const double nb = std::sqrt(D.host[0]);
        if (nb == 0.0) return CGS_OK;
        // Schwarz-Richardson, undamped: x += M (b - A x) until the true
        // residual meets the tolerance; iters = updates of x
        WRAP_CUDA(cudaMemcpyAsync(r, bm, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        for (int k = 0;; ++k) {
            WRAP_OK(dots(D, nullptr, 0, n, r, dir, st));
            const double rel = std::sqrt(D.host[0]) / nb;
            *iters = k;
            *relres = rel;
            if (!std::isfinite(rel)) {
                result = CGS_ERR_BREAKDOWN;
                break;
            }
            if (rel <= rtol) {
                result = CGS_OK;
                break;
            }
            if (k == maxit) break;
            WRAP_OK(cgs_apply_preconditioner(mesh, r, y, st));
            launch_vec_add(n, x, y, x, st);
            WRAP_OK(cgs_apply_A(mesh, x, y, st));
            launch_proj_combine(n, bm, dir, -1.0, one, 1, y, r, st);
        }
        WRAP_CUDA(cudaStreamSynchronize(st));
        WRAP_CUDA(cudaGetLastError());
        if (result == CGS_ERR_NO_CONVERGENCE) set_last_error("maxit reached before the tolerance");
        if (result == CGS_ERR_BREAKDOWN) set_last_error("non-finite value in the wrapped iteration");
    }
    // a bounded device wait that expired inside the single steps
    const cgs_status ws = cgs_mesh_step_status(mesh, stream);
    if (ws != CGS_OK) return ws;
    if (result == CGS_ERR_NO_CONVERGENCE) set_last_error("maxit reached before the tolerance");
    if (result == CGS_ERR_BREAKDOWN) set_last_error("non-finite value in the wrapped iteration");
    return result;
}
