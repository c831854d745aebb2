// C ABI of the p-multigrid wrap (Sec. 1, Sec. 5, Eqs. (13) and (14)): set-up
// of the spectral-element levels on the device, the single steps, the
// additive multilevel preconditioner and flexible GMRES on the finest level.
#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"
#include "krylov.h"
#include "sem.h"

using namespace cgs;

struct cgs_pmg {
    cgs_mesh* mesh = nullptr;
    int device = 0;
    int64_t nv = 0, ne = 0;
    int64_t nfree1 = 0;                            // free mesh vertices
    std::vector<int> orders;                       // the SEM levels' orders
    std::vector<SemDevLevel> lev;
    std::vector<std::vector<int32_t>> host_l2g;    // plain numbering, for the queries
    std::vector<double> xyz;
    std::vector<int32_t> conn;
    int32_t* l2g1 = nullptr;                       // order 1: conn, Dirichlet vertices encoded
    double* r1 = nullptr;
    double* z1 = nullptr;
    bool f32 = false;                              // float smoothers and transfers
    double* gmres_work = nullptr;                  // GMRES workspace, kept across solves
    size_t gmres_doubles = 0;
    std::vector<void*> allocs;
    ~cgs_pmg() {
        for (void* p : allocs) cudaFree(p);
        if (gmres_work) cudaFree(gmres_work);
    }
};

namespace {

cgs_status pmg_fail(cgs_status s, const std::string& msg) {
    set_last_error(msg);
    return s;
}

cgs_status pmg_cuda(cudaError_t e, const char* what) {
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CGS_ERR_OOM : CGS_ERR_CUDA;
}

#define PMG_CUDA(call)                                          \
    do {                                                        \
        const cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return pmg_cuda(e_, #call);      \
    } while (0)
#define PMG_OK(call)                                            \
    do {                                                        \
        const cgs_status s_ = (call);                           \
        if (s_ != CGS_OK) return s_;                            \
    } while (0)

template <class T>
cudaError_t upload(cgs_pmg* P, T** dst, const T* src, size_t n) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    P->allocs.push_back(p);
    *dst = static_cast<T*>(p);
    if (src && n) e = cudaMemcpy(p, src, n * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

int n_levels(const cgs_pmg* P) { return (int)P->orders.size(); }

// The next-coarser level of level l: nodes per direction, map, size, work
// vectors and whether they are float (order 1: the mesh's float64 vectors).
struct Next {
    int pc;
    const int32_t* l2g;
    int64_t ng;
    void* r;
    void* z;
    bool f32;
    bool sem;    // a spectral-element level (else order 1)
};
Next next_level(const cgs_pmg* P, int l) {
    if (l + 1 < n_levels(P)) {
        const SemDevLevel& C = P->lev[l + 1];
        return {C.p, C.l2g, C.ng, C.r, C.z, C.f32, true};
    }
    return {2, P->l2g1, P->nv, P->r1, P->z1, false, false};
}

size_t vec_bytes(int64_t n, bool f32) { return (size_t)n * (f32 ? sizeof(float) : sizeof(double)); }

// z = M r on level l and below (Eq. (13)), z overwritten; the vectors of
// level l are float when l > 0 and the level is f32
cgs_status pmg_level(cgs_pmg* P, int l, const void* r, void* z, cudaStream_t st) {
    const SemDevLevel& L = P->lev[l];
    const bool vf = l > 0 && L.f32;
    PMG_CUDA(cudaMemsetAsync(z, 0, vec_bytes(L.ng, vf), st));
    launch_sem_fdm(L, P->ne, r, z, vf, st);
    const Next c = next_level(P, l);
    PMG_CUDA(cudaMemsetAsync(c.r, 0, vec_bytes(c.ng, c.f32), st));
    launch_sem_restrict(L, c.pc, c.l2g, P->ne, r, c.r, vf, c.f32, st);
    if (c.sem)
        PMG_OK(pmg_level(P, l + 1, c.r, c.z, st));
    else
        PMG_OK(cgs_apply_preconditioner(P->mesh, static_cast<const double*>(c.r), static_cast<double*>(c.z), st));
    launch_sem_prolong(L, c.pc, c.l2g, P->ne, c.z, z, c.f32, vf, st);
    PMG_CUDA(cudaGetLastError());
    return CGS_OK;
}

}  // namespace

extern "C" {

cgs_status cgs_pmg_setup(cgs_mesh* mesh, const double* xyz, int64_t nv, const int32_t* conn, int64_t ne,
                         const int32_t* orders, int n_orders, cgs_pmg** out) {
    if (!mesh || !xyz || !conn || !orders || !out) return pmg_fail(CGS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_orders < 1 || n_orders > 4) return pmg_fail(CGS_ERR_INVALID_ARG, "n_orders must be in [1, 4]");
    for (int i = 0; i < n_orders; ++i) {
        if (orders[i] < kSemMinOrder || orders[i] > kSemMaxOrder)
            return pmg_fail(CGS_ERR_INVALID_ARG, "orders must be in [2, 8]");
        if (i && orders[i] >= orders[i - 1]) return pmg_fail(CGS_ERR_INVALID_ARG, "orders must decrease");
    }
    const DevMesh& M = mesh_dev(mesh);
    if (nv != M.nv || ne != M.ne) return pmg_fail(CGS_ERR_INVALID_ARG, "xyz/conn sizes differ from the mesh's");
    if (ne == 0) return pmg_fail(CGS_ERR_INVALID_ARG, "empty mesh");
    for (int64_t q = 0; q < ne * 8; ++q)
        if (conn[q] < 0 || conn[q] >= nv) return pmg_fail(CGS_ERR_INVALID_MESH, "vertex index out of range");
    PMG_CUDA(cudaSetDevice(mesh_device(mesh)));
    // the mesh must carry the default Dirichlet set
    std::vector<uint8_t> mdir((size_t)nv);
    PMG_CUDA(cudaMemcpy(mdir.data(), mesh_dir(mesh), (size_t)nv, cudaMemcpyDeviceToHost));
    const std::vector<uint8_t> bdir = sem_boundary_vertices(conn, ne, nv);
    for (int64_t v = 0; v < nv; ++v)
        if ((mdir[v] != 0) != (bdir[v] != 0))
            return pmg_fail(CGS_ERR_INVALID_ARG, "the mesh's Dirichlet set is not the boundary-face vertices");
    auto P = std::make_unique<cgs_pmg>();
    P->mesh = mesh;
    P->device = mesh_device(mesh);
    P->nv = nv;
    P->ne = ne;
    P->orders.assign(orders, orders + n_orders);
    P->xyz.assign(xyz, xyz + nv * 3);
    P->conn.assign(conn, conn + ne * 8);
    // the smoothers and transfers follow the coarse mesh's precision: float64
    // under the FP64 form, float under the mixed forms
    const bool f32 = mesh_prec(mesh) != CGS_FP64;
    P->f32 = f32;
    std::vector<SemHostLevel> H(n_orders);
    for (int l = 0; l < n_orders; ++l) {
        const std::string err = sem_build_level(orders[l], xyz, nv, conn, ne, H[l]);
        if (!err.empty())
            return pmg_fail(err.find("Jacobian") != std::string::npos ? CGS_ERR_INVALID_MESH : CGS_ERR_INVALID_ARG,
                            err);
    }
    P->lev.resize(n_orders);
    P->host_l2g.resize(n_orders);
    for (int l = 0; l < n_orders; ++l) {
        SemHostLevel& h = H[l];
        SemDevLevel& d = P->lev[l];
        d.n = h.n;
        d.p = h.p;
        d.ng = h.ng;
        d.nfree = h.nfree;
        std::vector<int32_t> enc(h.l2g.size());
        for (size_t q = 0; q < enc.size(); ++q) enc[q] = h.dir[h.l2g[q]] ? -(h.l2g[q] + 1) : h.l2g[q];
        PMG_CUDA(upload(P.get(), &d.l2g, enc.data(), enc.size()));
        if (f32) {   // the operator in float pairs: the metric and D as (hi, lo)
            auto pairs = [](const std::vector<double>& v) {
                std::vector<float2> out(v.size());
                for (size_t q = 0; q < v.size(); ++q) {
                    const float hi = (float)v[q];
                    out[q] = make_float2(hi, (float)(v[q] - (double)hi));
                }
                return out;
            };
            const std::vector<float2> Gp = pairs(h.G), Dp = pairs(h.D);
            PMG_CUDA(upload(P.get(), &d.Gp, Gp.data(), Gp.size()));
            PMG_CUDA(upload(P.get(), &d.Dp, Dp.data(), Dp.size()));
        } else {
            PMG_CUDA(upload(P.get(), &d.G, h.G.data(), h.G.size()));
        }
        PMG_CUDA(upload(P.get(), &d.dir, h.dir.data(), h.dir.size()));
        PMG_CUDA(upload(P.get(), &d.inv_mult, h.inv_mult.data(), h.inv_mult.size()));
        PMG_CUDA(upload(P.get(), &d.S, h.S.data(), h.S.size()));
        PMG_CUDA(upload(P.get(), &d.lam, h.lam.data(), h.lam.size()));
        PMG_CUDA(upload(P.get(), &d.D, h.D.data(), h.D.size()));
        // interpolation to the next coarser level
        std::vector<double> xc, I;
        if (l + 1 < n_orders)
            xc = H[l + 1].x;
        else
            xc = {-1.0, 1.0};
        lagrange_interp(xc, h.x, I);
        PMG_CUDA(upload(P.get(), &d.I_next, I.data(), I.size()));
        d.f32 = f32;
        if (f32) {
            auto to_f = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
            const std::vector<float> S32 = to_f(h.S), lam32 = to_f(h.lam), w32 = to_f(h.inv_mult), I32 = to_f(I);
            PMG_CUDA(upload(P.get(), &d.S32, S32.data(), S32.size()));
            PMG_CUDA(upload(P.get(), &d.lam32, lam32.data(), lam32.size()));
            PMG_CUDA(upload(P.get(), &d.inv_mult32, w32.data(), w32.size()));
            PMG_CUDA(upload(P.get(), &d.I_next32, I32.data(), I32.size()));
        }
        if (l > 0) {
            if (f32) {
                float *r, *z;
                PMG_CUDA(upload<float>(P.get(), &r, nullptr, (size_t)h.ng));
                PMG_CUDA(upload<float>(P.get(), &z, nullptr, (size_t)h.ng));
                d.r = r;
                d.z = z;
            } else {
                double *r, *z;
                PMG_CUDA(upload<double>(P.get(), &r, nullptr, (size_t)h.ng));
                PMG_CUDA(upload<double>(P.get(), &z, nullptr, (size_t)h.ng));
                d.r = r;
                d.z = z;
            }
        }
        P->host_l2g[l] = std::move(h.l2g);
        h = SemHostLevel();   // release the host copies level by level
    }
    std::vector<int32_t> enc1((size_t)ne * 8);
    for (size_t q = 0; q < enc1.size(); ++q) enc1[q] = mdir[conn[q]] ? -(conn[q] + 1) : conn[q];
    PMG_CUDA(upload(P.get(), &P->l2g1, enc1.data(), enc1.size()));
    for (int64_t v = 0; v < nv; ++v) P->nfree1 += !mdir[v];
    PMG_CUDA(upload<double>(P.get(), &P->r1, nullptr, (size_t)nv));
    PMG_CUDA(upload<double>(P.get(), &P->z1, nullptr, (size_t)nv));
    *out = P.release();
    return CGS_OK;
}

cgs_status cgs_pmg_free(cgs_pmg* pmg) {
    if (!pmg) return pmg_fail(CGS_ERR_INVALID_ARG, "null pmg");
    cudaSetDevice(pmg->device);
    cudaDeviceSynchronize();
    delete pmg;
    return CGS_OK;
}

cgs_status cgs_pmg_info(const cgs_pmg* pmg, int level, int* order, int64_t* n_nodes, int64_t* n_free) {
    if (!pmg || level < 0 || level > n_levels(pmg)) return pmg_fail(CGS_ERR_INVALID_ARG, "bad pmg or level");
    if (level == n_levels(pmg)) {
        if (order) *order = 1;
        if (n_nodes) *n_nodes = pmg->nv;
        if (n_free) *n_free = pmg->nfree1;
        return CGS_OK;
    }
    const SemDevLevel& L = pmg->lev[level];
    if (order) *order = L.n;
    if (n_nodes) *n_nodes = L.ng;
    if (n_free) *n_free = L.nfree;
    return CGS_OK;
}

cgs_status cgs_pmg_node_map(const cgs_pmg* pmg, int level, int32_t* l2g) {
    if (!pmg || !l2g || level < 0 || level > n_levels(pmg)) return pmg_fail(CGS_ERR_INVALID_ARG, "bad argument");
    if (level == n_levels(pmg)) {
        std::memcpy(l2g, pmg->conn.data(), pmg->conn.size() * sizeof(int32_t));
        return CGS_OK;
    }
    const auto& h = pmg->host_l2g[level];
    std::memcpy(l2g, h.data(), h.size() * sizeof(int32_t));
    return CGS_OK;
}

cgs_status cgs_pmg_node_coords(const cgs_pmg* pmg, int level, double* xyz) {
    if (!pmg || !xyz || level < 0 || level > n_levels(pmg)) return pmg_fail(CGS_ERR_INVALID_ARG, "bad argument");
    if (level == n_levels(pmg)) {
        std::memcpy(xyz, pmg->xyz.data(), pmg->xyz.size() * sizeof(double));
        return CGS_OK;
    }
    const SemDevLevel& L = pmg->lev[level];
    sem_node_coords(L.n, pmg->xyz.data(), pmg->conn.data(), pmg->ne, pmg->host_l2g[level], L.ng, xyz);
    return CGS_OK;
}

cgs_status cgs_pmg_apply_A(cgs_pmg* pmg, int level, const double* x, double* y, void* stream) {
    if (!pmg || !x || !y || level < 0 || level >= n_levels(pmg)) return pmg_fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const SemDevLevel& L = pmg->lev[level];
    PMG_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * L.ng, st));
    launch_sem_ax(L, pmg->ne, x, y, st);
    PMG_CUDA(cudaGetLastError());
    return CGS_OK;
}

cgs_status cgs_pmg_smooth(cgs_pmg* pmg, int level, const double* r, double* z, void* stream) {
    if (!pmg || !r || !z || level < 0 || level >= n_levels(pmg)) return pmg_fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const SemDevLevel& L = pmg->lev[level];
    PMG_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * L.ng, st));
    launch_sem_fdm(L, pmg->ne, r, z, false, st);
    PMG_CUDA(cudaGetLastError());
    return CGS_OK;
}

cgs_status cgs_pmg_restrict(cgs_pmg* pmg, int level, const double* rf, double* rc, void* stream) {
    if (!pmg || !rf || !rc || level < 0 || level >= n_levels(pmg)) return pmg_fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Next c = next_level(pmg, level);
    PMG_CUDA(cudaMemsetAsync(rc, 0, sizeof(double) * c.ng, st));
    launch_sem_restrict(pmg->lev[level], c.pc, c.l2g, pmg->ne, rf, rc, false, false, st);
    PMG_CUDA(cudaGetLastError());
    return CGS_OK;
}

cgs_status cgs_pmg_prolong(cgs_pmg* pmg, int level, const double* uc, double* uf, void* stream) {
    if (!pmg || !uc || !uf || level < 0 || level >= n_levels(pmg)) return pmg_fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Next c = next_level(pmg, level);
    const SemDevLevel& L = pmg->lev[level];
    PMG_CUDA(cudaMemsetAsync(uf, 0, sizeof(double) * L.ng, st));
    launch_sem_prolong(L, c.pc, c.l2g, pmg->ne, uc, uf, false, false, st);
    PMG_CUDA(cudaGetLastError());
    return CGS_OK;
}

cgs_status cgs_pmg_apply_preconditioner(cgs_pmg* pmg, const double* r, double* z, void* stream) {
    if (!pmg || !r || !z) return pmg_fail(CGS_ERR_INVALID_ARG, "null argument");
    PMG_CUDA(cudaSetDevice(pmg->device));
    return pmg_level(pmg, 0, r, z, static_cast<cudaStream_t>(stream));
}

cgs_status cgs_pmg_solve(cgs_pmg* pmg, const double* b, double* x, double rtol, int maxit, int restart, int* iters,
                         double* relres, void* stream) {
    if (!pmg || !b || !x || !iters || !relres || maxit < 0 || !(rtol > 0.0) || restart < 1 || restart > 1024)
        return pmg_fail(CGS_ERR_INVALID_ARG, "null argument, maxit < 0, rtol <= 0 or restart outside [1, 1024]");
    PMG_CUDA(cudaSetDevice(pmg->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    KrylovOps ops;
    ops.n = pmg->lev[0].ng;
    ops.dir = pmg->lev[0].dir;
    // the workspace of the largest restart so far stays with the cgs_pmg
    const size_t need = fgmres_work_doubles(ops.n, restart);
    if (pmg->gmres_doubles < need) {
        if (pmg->gmres_work) {
            PMG_CUDA(cudaStreamSynchronize(st));
            cudaFree(pmg->gmres_work);
            pmg->gmres_work = nullptr;
            pmg->gmres_doubles = 0;
        }
        PMG_CUDA(cudaMalloc(&pmg->gmres_work, need * sizeof(double)));
        pmg->gmres_doubles = need;
    }
    ops.work = pmg->gmres_work;
    ops.work_doubles = pmg->gmres_doubles;
    ops.apply_A = [&](const double* u, double* y) { return cgs_pmg_apply_A(pmg, 0, u, y, stream); };
    ops.apply_M = [&](const double* r, double* z) { return pmg_level(pmg, 0, r, z, st); };
    const cgs_status s = fgmres_device(ops, b, x, rtol, maxit, restart, iters, relres, st);
    if (s != CGS_OK && s != CGS_ERR_NO_CONVERGENCE && s != CGS_ERR_BREAKDOWN) return s;
    const cgs_status ws = cgs_mesh_step_status(pmg->mesh, stream);
    return ws != CGS_OK ? ws : s;
}

}  // extern "C"
