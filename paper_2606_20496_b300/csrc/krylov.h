// Flexible GMRES on the device around any operator and preconditioner given
// as callbacks (wrappers.cu): used by cgs_solve_wrapped on a coarse mesh and
// by cgs_pmg_solve on the finest spectral-element level.
#pragma once

#include <cstdint>
#include <functional>

#include <cuda_runtime.h>

#include "../../include/cgs.h"

namespace cgs {

struct KrylovOps {
    int64_t n = 0;                      // vector length
    const uint8_t* dir = nullptr;       // device, n: Dirichlet entries (taken as zero in every dot)
    std::function<cgs_status(const double* x, double* y)> apply_A;
    std::function<cgs_status(const double* r, double* z)> apply_M;
    // optional device workspace of fgmres_work_doubles(n, restart) doubles,
    // kept by the caller across solves; without it the call allocates its own
    double* work = nullptr;
    size_t work_doubles = 0;
};

size_t fgmres_work_doubles(int64_t n, int restart);

// Right-preconditioned flexible GMRES(restart) from x = 0 on device vectors:
// the Arnoldi basis V of the preconditioned directions Z = M V (classical
// Gram-Schmidt applied twice), Givens rotations on the host, x += Z y at each
// restart.  iters = products A z; relres = ||b - A x|| / ||b|| of the last
// restart's residual.  Uses ops.work when it is large enough, else
// allocates its (2 restart + 3) n doubles (and a few more) for the call.
cgs_status fgmres_device(const KrylovOps& ops, const double* b, double* x, double rtol, int maxit, int restart,
                         int* iters, double* relres, cudaStream_t st);

}  // namespace cgs
