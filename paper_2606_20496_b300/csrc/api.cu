// C ABI of the coarse-grid Schwarz solver (declared in include/cgs.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"

using namespace cgs;

namespace {

thread_local std::string g_err;

cgs_status fail(cgs_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

cgs_status cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CGS_ERR_OOM : CGS_ERR_CUDA;
}

#define CGS_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

}  // namespace

struct cgs_ctx {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    int live_meshes = 0;
    std::mutex mu;
};

struct cgs_mesh {
    cgs_ctx* ctx = nullptr;
    cgs_params prm{};
    cgs_form form = CGS_HYBRID;
    DevMesh d;
    cgs_mesh_info_t info{};
    std::vector<void*> allocs;
    size_t bytes = 0;
    // host copies kept for cgs_mesh_export
    std::vector<uint8_t> dir_h;
    std::vector<int64_t> box_active_h, sub_ptr_h;
    std::vector<int32_t> sub_idx_h;
    // device scratch
    uint8_t* dir = nullptr;
    double *r = nullptr, *p = nullptr, *q = nullptr, *y = nullptr, *x = nullptr;
    float2 *p2 = nullptr, *q2 = nullptr;   // float-pair p and A p of the mixed forms
    float* ur32 = nullptr;                 // float copy of u_r for the float interpolation
    // device-side PCG loop: a graph whose while node repeats one iteration
    cudaGraphExec_t gexec = nullptr;
    bool graph_failed = false;
    void* z = nullptr;   // bulk precision (double for FP64, float otherwise)
    void* s = nullptr;
    double *rr = nullptr, *ur = nullptr, *partials = nullptr, *out2 = nullptr;
    SolveScalars* S = nullptr;
    SolveScalars* S_host = nullptr;   // pinned
    double* out2_host = nullptr;      // pinned
    double *hb = nullptr, *hx = nullptr;  // device staging for cgs_solve_host
    size_t h_cap = 0;
    int last_iters = 8;
    // launch accounting and the optional event profiler
    int64_t launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, size_t>> ev_used;   // (kernel class, index of the start event)
    size_t ev_next = 0;
    double prof_ms[CGS_K_COUNT] = {0};
    int64_t prof_n[CGS_K_COUNT] = {0};

    template <typename T>
    cudaError_t alloc(T** p_out, size_t count) {
        void* p = nullptr;
        const size_t bytes_ = std::max<size_t>(count, 1) * sizeof(T);
        cudaError_t e = cudaMalloc(&p, bytes_);
        if (e != cudaSuccess) return e;
        allocs.push_back(p);
        bytes += bytes_;
        *p_out = static_cast<T*>(p);
        return cudaSuccess;
    }
    template <typename T>
    cudaError_t upload(const T** p_out, const std::vector<T>& h) {
        T* p = nullptr;
        cudaError_t e = alloc(&p, h.size());
        if (e != cudaSuccess) return e;
        if (!h.empty()) e = cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        *p_out = p;
        return e;
    }
    void release() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        ev_pool.clear();
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
        if (S_host) cudaFreeHost(S_host);
        if (out2_host) cudaFreeHost(out2_host);
        S_host = nullptr;
        out2_host = nullptr;
    }
    bool fp64() const { return prm.prec == CGS_FP64; }
};

namespace {

cgs_params default_params() {
    cgs_params p;
    p.box[0] = p.box[1] = p.box[2] = 4;
    p.box_margin = 0.0;
    p.overlap_layers = 1;
    p.prec = CGS_FP64;
    p.form = CGS_HYBRID;
    return p;
}

cgs_status check_mesh(const cgs_mesh* m) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    return CGS_OK;
}

cgs_status finish(cudaStream_t st, bool sync) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (sync) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return CGS_OK;
}

cudaEvent_t next_event(cgs_mesh* m) {
    if (m->ev_next == m->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        m->ev_pool.push_back(e);
    }
    return m->ev_pool[m->ev_next++];
}

// Run one kernel launcher, counting it and, when profiling, bracketing it by
// events on its stream.
template <typename F>
inline void launch(cgs_mesh* m, int cls, cudaStream_t st, F&& f) {
    m->launches++;
    if (!m->prof) {
        f();
        return;
    }
    const size_t i0 = m->ev_next;
    cudaEventRecord(next_event(m), st);
    f();
    cudaEventRecord(next_event(m), st);
    m->ev_used.emplace_back(cls, i0);
}

#define K(cls, call) launch(m, (cls), st, [&]() { call; })

// Fill z = 0, s = r (bulk precision), r_r = 0 before a preconditioner apply.
void precond_prep(cgs_mesh* m, const double* r, cudaStream_t st) {
    const int64_t nv = m->d.nv;
    if (m->fp64()) {
        K(CGS_K_OTHER, launch_fill_d(nv, static_cast<double*>(m->z), 0.0, st));
        K(CGS_K_OTHER, launch_copy_d(nv, r, static_cast<double*>(m->s), nullptr, st));
    } else {
        K(CGS_K_OTHER, launch_fill_f(nv, static_cast<float*>(m->z), 0.0f, st));
        K(CGS_K_OTHER, launch_convert_d2f(nv, r, static_cast<float*>(m->s), nullptr, st));
    }
    if (m->d.nr) K(CGS_K_OTHER, launch_fill_d(m->d.nr, m->rr, 0.0, st));
}

// z += J~ A_r^{-1} J~^T s (s the bulk copy of the residual or of r - A l).
void box_correction(cgs_mesh* m, const SolveScalars* S, cudaStream_t st) {
    const DevMesh& d = m->d;
    const bool f64 = m->fp64();
    K(CGS_K_RESTRICT, launch_restrict(d, f64, m->s, f64, m->rr, S, st));
    K(CGS_K_COARSE, launch_coarse(d, m->rr, m->ur, f64 ? nullptr : m->ur32, S, st));
    K(CGS_K_INTERP, launch_interp_add(d, f64, m->ur, f64 ? nullptr : m->ur32, m->z, S, st));
}

// z (bulk) = M r, assuming precond_prep (or the PCG update kernel) ran.
void precond_body(cgs_mesh* m, const double* r, const SolveScalars* S, cudaStream_t st) {
    const DevMesh& d = m->d;
    const bool f64 = m->fp64();
    if (m->form == CGS_HYBRID) {
        K(CGS_K_LOCAL, launch_local(d, m->prm.prec, m->s, m->z, true, S, st));
        if (f64)
            K(CGS_K_APPLY_A64, launch_apply64(d, static_cast<const double*>(m->z), static_cast<double*>(m->s),
                                              -1.0, nullptr, const_cast<SolveScalars*>(S), false, st));
        else
            K(CGS_K_APPLY_A32, launch_apply28f_tiled(d, static_cast<const float*>(m->z), static_cast<float*>(m->s),
                                                     -1.0f, const_cast<SolveScalars*>(S), st));
        if (d.nr) box_correction(m, S, st);
    } else {
        K(CGS_K_LOCAL, launch_local(d, m->prm.prec, m->s, m->z, false, S, st));
        if (d.nr) box_correction(m, S, st);
    }
}

void z_to_double(cgs_mesh* m, double* out, cudaStream_t st) {
    if (m->fp64())
        K(CGS_K_OTHER, launch_copy_d(m->d.nv, static_cast<const double*>(m->z), out, m->dir, st));
    else
        K(CGS_K_OTHER, launch_convert_f2d(m->d.nv, static_cast<const float*>(m->z), out, m->dir, st));
}

// One flexible-PCG iteration on mesh-owned buffers (x is the mesh's own
// iterate, so the same launches can be captured once into a graph).
template <typename Tz>
void pcg_iteration(cgs_mesh* m, cudaStream_t st, cudaGraphConditionalHandle cond, bool use_cond) {
    const DevMesh& d = m->d;
    Tz* z = static_cast<Tz*>(m->z);
    Tz* s = static_cast<Tz*>(m->s);
    if (m->fp64()) {
        K(CGS_K_APPLY_A64, launch_apply64(d, m->p, m->q, 1.0, m->partials, m->S, true, st));
        K(CGS_K_PCG_XR, (launch_pcg_update_xr<Tz, double>(d, m->x, m->r, m->p, m->q, z, s, m->rr, m->partials,
                                                           m->S, st)));
        precond_body(m, m->r, m->S, st);
        K(CGS_K_PCG_DOTS, (launch_pcg_dots<Tz, double>(d, z, m->r, m->q, m->partials, m->S, st)));
        K(CGS_K_PCG_P, (launch_pcg_update_p<Tz, double>(d, z, m->p, nullptr, m->q, m->S, cond, use_cond, st)));
    } else {
        K(CGS_K_APPLY_A64, launch_apply_pair_tiled(d, m->p2, m->q2, m->partials, m->S, st));
        K(CGS_K_PCG_XR, (launch_pcg_update_xr<Tz, float2>(d, m->x, m->r, m->p, m->q2, z, s, m->rr, m->partials,
                                                           m->S, st)));
        precond_body(m, m->r, m->S, st);
        K(CGS_K_PCG_DOTS, (launch_pcg_dots<Tz, float2>(d, z, m->r, m->q2, m->partials, m->S, st)));
        K(CGS_K_PCG_P, (launch_pcg_update_p<Tz, float2>(d, z, m->p, m->p2, m->q2, m->S, cond, use_cond, st)));
    }
}

// Build the graph: one while node whose body is one PCG iteration; the body's
// last kernel sets the loop condition from the device-side stopping test.
template <typename Tz>
cgs_status build_loop_graph(cgs_mesh* m) {
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    auto bail = [&](cudaError_t e, const char* where) {
        if (cs) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(cs, &dummy);
            cudaStreamDestroy(cs);
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(e, where);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(e, "graph stream");
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return bail(e, "cudaGraphCreate");
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return bail(e, "cudaGraphConditionalHandleCreate");
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) return bail(e, "cudaGraphAddNode");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return bail(e, "cudaStreamBeginCaptureToGraph");
    const bool prof = m->prof;
    const int64_t launches = m->launches;
    m->prof = false;
    pcg_iteration<Tz>(m, cs, h, true);
    m->prof = prof;
    m->launches = launches;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    cs = nullptr;
    if (e != cudaSuccess) return bail(e, "cudaStreamEndCapture");
    if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) return bail(e, "cudaGraphInstantiate");
    cudaGraphDestroy(g);
    m->gexec = ex;
    return CGS_OK;
}

template <typename Tz>
cgs_status solve_one(cgs_mesh* m, const double* b, double* x, double rtol, int maxit, int* iters, double* relres,
                     cudaStream_t st) {
    const DevMesh& d = m->d;
    if (m->fp64())
        K(CGS_K_OTHER, launch_pcg_init<double>(d, b, m->dir, m->x, m->r, m->q, rtol, maxit, m->partials, m->S, st));
    else
        K(CGS_K_OTHER, launch_pcg_init<float2>(d, b, m->dir, m->x, m->r, m->q2, rtol, maxit, m->partials, m->S, st));
    // z = M r, p = z, rho = r.z  (skipped when b = 0)
    if (m->fp64()) {
        K(CGS_K_OTHER, launch_fill_d(d.nv, static_cast<double*>(m->z), 0.0, st));
        K(CGS_K_OTHER, launch_copy_d(d.nv, m->r, static_cast<double*>(m->s), nullptr, st));
    } else {
        K(CGS_K_OTHER, launch_fill_f(d.nv, static_cast<float*>(m->z), 0.0f, st));
        K(CGS_K_OTHER, launch_convert_d2f(d.nv, m->r, static_cast<float*>(m->s), nullptr, st));
    }
    if (d.nr) K(CGS_K_OTHER, launch_fill_d(d.nr, m->rr, 0.0, st));
    precond_body(m, m->r, m->S, st);
    K(CGS_K_OTHER, launch_pcg_first_dir<Tz>(d, static_cast<const Tz*>(m->z), m->r, m->p, m->p2, m->partials, m->S,
                                            st));
    const bool use_graph = !m->prof && !m->graph_failed;
    if (use_graph && !m->gexec) {
        if (build_loop_graph<Tz>(m) != CGS_OK) m->graph_failed = true;
    }
    if (use_graph && m->gexec) {
        // the whole iteration loop runs on the device
        CGS_CUDA(cudaGraphLaunch(m->gexec, st));
        m->launches += 1;
        CGS_CUDA(cudaMemcpyAsync(m->S_host, m->S, sizeof(SolveScalars), cudaMemcpyDeviceToHost, st));
    } else {
        int enqueued = 0;
        int chunk = std::max(2, m->last_iters);
        for (;;) {
            const int n = std::min(chunk, maxit - enqueued);
            for (int i = 0; i < n; ++i) pcg_iteration<Tz>(m, st, cudaGraphConditionalHandle(), false);
            enqueued += n;
            CGS_CUDA(cudaMemcpyAsync(m->S_host, m->S, sizeof(SolveScalars), cudaMemcpyDeviceToHost, st));
            CGS_CUDA(cudaStreamSynchronize(st));
            if (m->S_host->done || enqueued >= maxit) break;
            chunk = 4;
        }
    }
    // x out, then the true residual ||b - A x|| / ||b|| over the free entries
    K(CGS_K_OTHER, launch_copy_d(d.nv, m->x, x, nullptr, st));
    K(CGS_K_OTHER, launch_fill_d(d.nv, m->y, 0.0, st));
    K(CGS_K_APPLY_A64, launch_apply64(d, m->x, m->y, 1.0, nullptr, nullptr, false, st));
    K(CGS_K_OTHER, launch_resid_norm(d, b, m->y, m->dir, m->partials, &m->S->ticket[1], m->out2, st));
    CGS_CUDA(cudaMemcpyAsync(m->out2_host, m->out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    cgs_status fs = finish(st, true);
    if (fs != CGS_OK) return fs;
    const SolveScalars h = *m->S_host;
    const int status = h.done ? h.status : CGS_ERR_NO_CONVERGENCE;
    *iters = h.iters;
    if (h.iters > 0) m->last_iters = h.iters;
    *relres = m->out2_host[1] > 0 ? std::sqrt(m->out2_host[0] / m->out2_host[1]) : 0.0;
    if (status == CGS_ERR_NO_CONVERGENCE) g_err = "maxit reached before the tolerance";
    if (status == CGS_ERR_BREAKDOWN) g_err = "breakdown in the PCG iteration";
    return (cgs_status)status;
}

}  // namespace

namespace cgs {
// Read-only views of a mesh for entry points defined in other files.
const DevMesh& mesh_dev(const cgs_mesh* m) { return m->d; }
cgs_precision mesh_prec(const cgs_mesh* m) { return m->prm.prec; }
cgs_form mesh_form(const cgs_mesh* m) { return m->form; }
const uint8_t* mesh_dir(const cgs_mesh* m) { return m->dir; }
int mesh_device(const cgs_mesh* m) { return m->ctx->device; }
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace cgs

extern "C" {

const char* cgs_status_string(cgs_status s) {
    switch (s) {
        case CGS_OK: return "ok";
        case CGS_ERR_INVALID_ARG: return "invalid argument";
        case CGS_ERR_INVALID_MESH: return "invalid mesh";
        case CGS_ERR_NOT_SPD: return "matrix not SPD";
        case CGS_ERR_NO_CONVERGENCE: return "no convergence";
        case CGS_ERR_BREAKDOWN: return "breakdown";
        case CGS_ERR_OOM: return "out of device memory";
        case CGS_ERR_ADMISSION: return "HBM budget exceeded";
        case CGS_ERR_TIMEOUT: return "device wait timed out";
        case CGS_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

const char* cgs_last_error(void) { return g_err.c_str(); }

cgs_status cgs_create(cgs_ctx** ctx, int device, size_t hbm_budget_bytes) {
    if (!ctx) return fail(CGS_ERR_INVALID_ARG, "null ctx");
    *ctx = nullptr;
    int n = 0;
    CGS_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(CGS_ERR_INVALID_ARG, "no such CUDA device");
    CGS_CUDA(cudaSetDevice(device));
    cgs_ctx* c = new (std::nothrow) cgs_ctx;
    if (!c) return fail(CGS_ERR_INVALID_ARG, "host allocation failed");
    c->device = device;
    c->budget = hbm_budget_bytes;
    *ctx = c;
    return CGS_OK;
}

cgs_status cgs_destroy(cgs_ctx* ctx) {
    if (!ctx) return fail(CGS_ERR_INVALID_ARG, "null ctx");
    if (ctx->live_meshes != 0) return fail(CGS_ERR_INVALID_ARG, "meshes still alive");
    delete ctx;
    return CGS_OK;
}

size_t cgs_ctx_bytes_in_use(const cgs_ctx* ctx) { return ctx ? ctx->in_use : 0; }

cgs_status cgs_mesh_setup(cgs_ctx* ctx, const double* xyz, int64_t nv, const int32_t* conn, int64_t ne,
                          const uint8_t* dirichlet, const int32_t* elem_part, const cgs_params* params,
                          cgs_mesh** out) {
    if (!out) return fail(CGS_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (!ctx) return fail(CGS_ERR_INVALID_ARG, "null ctx");
    const auto t0 = std::chrono::steady_clock::now();
    const cgs_params prm = params ? *params : default_params();
    if (prm.prec < CGS_FP64 || prm.prec > CGS_FP16_LOCAL || prm.form < CGS_HYBRID || prm.form > CGS_ADDITIVE)
        return fail(CGS_ERR_INVALID_ARG, "unknown precision or form");
    CGS_CUDA(cudaSetDevice(ctx->device));
    HostSetup hs;
    std::string err;
    cgs_status st = host_setup(xyz, nv, conn, ne, dirichlet, elem_part, prm, hs, err);
    if (st != CGS_OK) return fail(st, err);

    cgs_mesh* m = new (std::nothrow) cgs_mesh;
    if (!m) return fail(CGS_ERR_INVALID_ARG, "host allocation failed");
    m->ctx = ctx;
    m->prm = prm;
    m->form = prm.form;
    DevMesh& d = m->d;
    d.nv = nv;
    d.ne = ne;
    d.n_sub = hs.n_sub;
    d.nr = hs.nr;
    for (int k = 0; k < 3; ++k) {
        d.b[k] = hs.b[k];
        d.lo[k] = 0.0;   // coordinates are stored relative to the box origin
        d.H[k] = hs.H[k];
    }
    d.max_m = (int)hs.max_m;

    // estimated footprint for admission before allocating
    const bool f64 = prm.prec == CGS_FP64;
    const size_t bulk = f64 ? 8 : 4;
    size_t est = (size_t)ne * (8 * 4 + kUpper * 8 + kOff * 4 + 4) + (size_t)nv * (32 + 16 + 1 + 8 + 4) +
                 hs.sub_idx.size() * 4 + hs.inv.size() * (prm.prec == CGS_FP64 ? 8 : prm.prec == CGS_FP32_BULK ? 4 : 2) +
                 hs.ar_inv.size() * 8 + (size_t)nv * (4 * 8 + 2 * bulk);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->budget && ctx->in_use + est > ctx->budget) {
            delete m;
            return fail(CGS_ERR_ADMISSION, "mesh footprint exceeds the context's HBM budget");
        }
    }

    auto cleanup = [&](cgs_status s) {
        m->release();
        delete m;
        return s;
    };
#define UP(ptr, vec)                                                   \
    do {                                                               \
        cudaError_t e_ = m->upload(&(ptr), (vec));                     \
        if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, "upload")); \
    } while (0)
#define AL(ptr, n)                                                     \
    do {                                                               \
        cudaError_t e_ = m->alloc(&(ptr), (n));                        \
        if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, "alloc"));  \
    } while (0)

    UP(d.conn, hs.conn);
    UP(d.a36, hs.a36);
    if (!f64) {
        UP(d.at_hi, hs.at_hi);
        UP(d.at_lo, hs.at_lo);
    }
    UP(d.cell, hs.cell);
    if (!f64) {
        d.ntiles = (int64_t)hs.tile_ptr.size() - 1;
        UP(d.tile_ptr, hs.tile_ptr);
        UP(d.tile_vptr, hs.tile_vptr);
        UP(d.tile_verts, hs.tile_verts);
        UP(d.eloc, hs.eloc);
    }
    UP(d.cell_cols, hs.cell_cols);
    {
        std::vector<int32_t> sp(hs.sub_ptr.begin(), hs.sub_ptr.end());
        UP(d.sub_ptr, sp);
    }
    UP(d.sub_idx, hs.sub_idx);
    UP(d.inv_ptr, hs.inv_ptr);
    if (prm.prec == CGS_FP64) {
        UP(d.inv64, hs.inv);
    } else if (prm.prec == CGS_FP32_BULK) {
        std::vector<float> f(hs.inv.begin(), hs.inv.end());
        UP(d.inv32, f);
    } else {
        std::vector<__half> h(hs.inv.size());
        std::vector<float> sc(hs.n_sub, 1.0f);
        for (int64_t p = 0; p < hs.n_sub; ++p) {
            double mx = 0.0;
            for (int64_t i = hs.inv_ptr[p]; i < hs.inv_ptr[p + 1]; ++i) mx = std::max(mx, std::fabs(hs.inv[i]));
            const double s = mx > 0 ? mx : 1.0;
            sc[p] = (float)s;
            for (int64_t i = hs.inv_ptr[p]; i < hs.inv_ptr[p + 1]; ++i) h[i] = __float2half_rn((float)(hs.inv[i] / s));
        }
        UP(d.inv16, h);
        UP(d.inv16_scale, sc);
    }
    UP(d.wov64, hs.wov);
    if (!f64) {
        std::vector<float> w(hs.wov.begin(), hs.wov.end());
        UP(d.wov32, w);
    }
    {
        // vertex coordinates relative to the box origin, with 1/count
        std::vector<double> v64((size_t)nv * 4);
        std::vector<float> v32(f64 ? 0 : (size_t)nv * 4);
        for (int64_t v = 0; v < nv; ++v) {
            for (int k = 0; k < 3; ++k) v64[(size_t)v * 4 + k] = xyz[(size_t)v * 3 + k] - hs.lo[k];
            v64[(size_t)v * 4 + 3] = hs.invcnt[v];
            if (!f64)
                for (int k = 0; k < 4; ++k) v32[(size_t)v * 4 + k] = (float)v64[(size_t)v * 4 + k];
        }
        if (f64) {
            const double* p = nullptr;
            UP(p, v64);
            d.xyzw = reinterpret_cast<const double2*>(p);
        } else {
            const float* p = nullptr;
            UP(p, v32);
            d.xyzwf = reinterpret_cast<const float4*>(p);
        }
    }
    if (hs.nr) UP(d.ar_inv, hs.ar_inv);
    {
        const uint8_t* dp = nullptr;
        UP(dp, hs.dir);
        m->dir = const_cast<uint8_t*>(dp);
    }
    AL(m->r, nv);
    AL(m->p, nv);
    AL(m->y, nv);
    AL(m->x, nv);
    if (f64) {
        AL(m->q, nv);
    } else {
        AL(m->q2, nv);
        AL(m->p2, nv);
    }
    if (f64) {
        double* z = nullptr;
        double* s = nullptr;
        AL(z, nv);
        AL(s, nv);
        m->z = z;
        m->s = s;
    } else {
        float* z = nullptr;
        float* s = nullptr;
        AL(z, nv);
        AL(s, nv);
        m->z = z;
        m->s = s;
    }
    AL(m->rr, std::max<int64_t>(hs.nr, 1));
    if (!f64) AL(m->ur32, std::max<int64_t>(hs.nr, 1));
    AL(m->ur, std::max<int64_t>(hs.nr, 1));
    AL(m->partials, 2 * (size_t)partial_slots(d));
    AL(m->out2, 2);
    AL(m->S, 1);
    CGS_CUDA(cudaMemset(m->S, 0, sizeof(SolveScalars)));
    {
        cudaError_t e = cudaMallocHost(&m->S_host, sizeof(SolveScalars));
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMallocHost"));
        e = cudaMallocHost(&m->out2_host, 2 * sizeof(double));
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMallocHost"));
    }
    {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "setup upload"));
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->budget && ctx->in_use + m->bytes > ctx->budget) {
            return cleanup(fail(CGS_ERR_ADMISSION, "mesh footprint exceeds the context's HBM budget"));
        }
        ctx->in_use += m->bytes;
        ctx->live_meshes++;
    }
    m->dir_h = std::move(hs.dir);
    m->box_active_h = std::move(hs.box_active);
    m->sub_ptr_h = std::move(hs.sub_ptr);
    m->sub_idx_h = std::move(hs.sub_idx);
    m->info.nv = nv;
    m->info.ne = ne;
    m->info.n_free = hs.n_free;
    m->info.n_sub = hs.n_sub;
    m->info.n_r = hs.nr;
    m->info.max_sub_dofs = hs.max_m;
    m->info.sum_sub_dofs = hs.sum_m;
    m->info.footprint_bytes = m->bytes;
    m->info.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = m;
#undef UP
#undef AL
    return CGS_OK;
}

cgs_status cgs_mesh_free(cgs_mesh* m) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    cudaSetDevice(m->ctx->device);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> lk(m->ctx->mu);
        m->ctx->in_use -= m->bytes;
        m->ctx->live_meshes--;
    }
    m->release();
    delete m;
    return CGS_OK;
}

cgs_status cgs_mesh_info(const cgs_mesh* m, cgs_mesh_info_t* info) {
    if (!m || !info) return fail(CGS_ERR_INVALID_ARG, "null argument");
    *info = m->info;
    info->kernel_launches = m->launches;
    return CGS_OK;
}

cgs_status cgs_profile_enable(cgs_mesh* m, int enable) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    m->prof = enable != 0;
    return CGS_OK;
}

cgs_status cgs_profile_read(cgs_mesh* m, double* ms, int64_t* launches) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    if (!m->ev_used.empty()) {
        CGS_CUDA(cudaEventSynchronize(m->ev_pool[m->ev_used.back().second + 1]));
        for (const auto& u : m->ev_used) {
            float t = 0.0f;
            CGS_CUDA(cudaEventElapsedTime(&t, m->ev_pool[u.second], m->ev_pool[u.second + 1]));
            m->prof_ms[u.first] += t;
            m->prof_n[u.first] += 1;
        }
    }
    m->ev_used.clear();
    m->ev_next = 0;
    for (int k = 0; k < CGS_K_COUNT; ++k) {
        if (ms) ms[k] = m->prof_ms[k];
        if (launches) launches[k] = m->prof_n[k];
        m->prof_ms[k] = 0.0;
        m->prof_n[k] = 0;
    }
    return CGS_OK;
}

cgs_status cgs_mesh_set_form(cgs_mesh* m, cgs_form form) {
    if (!m || form < CGS_HYBRID || form > CGS_ADDITIVE) return fail(CGS_ERR_INVALID_ARG, "bad mesh or form");
    m->form = form;
    return CGS_OK;
}

cgs_status cgs_mesh_export(const cgs_mesh* m, uint8_t* dirichlet, int64_t* box_active, int64_t* sub_ptr,
                           int32_t* sub_idx) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    if (dirichlet) std::copy(m->dir_h.begin(), m->dir_h.end(), dirichlet);
    if (box_active) std::copy(m->box_active_h.begin(), m->box_active_h.end(), box_active);
    if (sub_ptr) std::copy(m->sub_ptr_h.begin(), m->sub_ptr_h.end(), sub_ptr);
    if (sub_idx) std::copy(m->sub_idx_h.begin(), m->sub_idx_h.end(), sub_idx);
    return CGS_OK;
}

cgs_status cgs_apply_A(cgs_mesh* m, const double* x, double* y, void* stream) {
    if (check_mesh(m) != CGS_OK || !x || !y) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    K(CGS_K_OTHER, launch_fill_d(m->d.nv, y, 0.0, st));
    K(CGS_K_APPLY_A64, launch_apply64(m->d, x, y, 1.0, nullptr, nullptr, false, st));
    return finish(st, false);
}

cgs_status cgs_apply_local(cgs_mesh* m, const double* r, double* l, int weighted, void* stream) {
    if (check_mesh(m) != CGS_OK || !r || !l) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m->fp64())
        K(CGS_K_OTHER, launch_fill_d(m->d.nv, static_cast<double*>(m->z), 0.0, st));
    else
        K(CGS_K_OTHER, launch_fill_f(m->d.nv, static_cast<float*>(m->z), 0.0f, st));
    const void* rin = r;
    if (!m->fp64()) {   // the float kernels read the residual in the bulk precision
        K(CGS_K_OTHER, launch_convert_d2f(m->d.nv, r, static_cast<float*>(m->s), nullptr, st));
        rin = m->s;
    }
    K(CGS_K_LOCAL, launch_local(m->d, m->prm.prec, rin, m->z, weighted != 0, nullptr, st));
    z_to_double(m, l, st);
    return finish(st, false);
}

cgs_status cgs_restrict(cgs_mesh* m, const double* s, double* rr, void* stream) {
    if (check_mesh(m) != CGS_OK || !s || (!rr && m->d.nr)) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m->d.nr == 0) return CGS_OK;
    K(CGS_K_OTHER, launch_fill_d(m->d.nr, rr, 0.0, st));
    K(CGS_K_RESTRICT, launch_restrict(m->d, m->fp64(), s, true, rr, nullptr, st));
    return finish(st, false);
}

cgs_status cgs_coarse_solve(cgs_mesh* m, const double* rr, double* ur, void* stream) {
    if (check_mesh(m) != CGS_OK || ((!rr || !ur) && m->d.nr)) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    K(CGS_K_COARSE, launch_coarse(m->d, rr, ur, nullptr, nullptr, st));
    return finish(st, false);
}

cgs_status cgs_interp(cgs_mesh* m, const double* ur, double* z, void* stream) {
    if (check_mesh(m) != CGS_OK || !z || (!ur && m->d.nr)) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m->fp64())
        K(CGS_K_OTHER, launch_fill_d(m->d.nv, static_cast<double*>(m->z), 0.0, st));
    else
        K(CGS_K_OTHER, launch_fill_f(m->d.nv, static_cast<float*>(m->z), 0.0f, st));
    if (m->d.nr) {
        K(CGS_K_INTERP, launch_interp_add(m->d, m->fp64(), ur, nullptr, m->z, nullptr, st));
    }
    z_to_double(m, z, st);
    return finish(st, false);
}

cgs_status cgs_apply_preconditioner(cgs_mesh* m, const double* r, double* z, void* stream) {
    if (check_mesh(m) != CGS_OK || !r || !z) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    precond_prep(m, r, st);
    precond_body(m, r, nullptr, st);
    z_to_double(m, z, st);
    return finish(st, false);
}

cgs_status cgs_solve(cgs_mesh* m, const double* b, double* x, int nrhs, double rtol, int maxit, int* iters,
                     double* relres, void* stream) {
    if (check_mesh(m) != CGS_OK || !b || !x || !iters || !relres || nrhs < 0 || !(rtol >= 0.0))
        return fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cgs_status first_bad = CGS_OK;
    for (int k = 0; k < nrhs; ++k) {
        const double* bk = b + (size_t)k * m->d.nv;
        double* xk = x + (size_t)k * m->d.nv;
        iters[k] = 0;
        relres[k] = 0.0;
        cgs_status s = m->fp64() ? solve_one<double>(m, bk, xk, rtol, maxit, &iters[k], &relres[k], st)
                                 : solve_one<float>(m, bk, xk, rtol, maxit, &iters[k], &relres[k], st);
        if (s == CGS_ERR_CUDA || s == CGS_ERR_OOM) return s;
        if (s != CGS_OK && first_bad == CGS_OK) first_bad = s;
    }
    return first_bad;
}

cgs_status cgs_solve_host(cgs_mesh* m, const double* b_host, double* x_host, int nrhs, double rtol, int maxit,
                          int* iters, double* relres, void* stream) {
    if (check_mesh(m) != CGS_OK || !b_host || !x_host || nrhs < 0) return fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)nrhs * m->d.nv;
    if (n > m->h_cap) {
        if (m->hb) {
            cudaFree(m->hb);
            cudaFree(m->hx);
            m->allocs.erase(std::remove(m->allocs.begin(), m->allocs.end(), (void*)m->hb), m->allocs.end());
            m->allocs.erase(std::remove(m->allocs.begin(), m->allocs.end(), (void*)m->hx), m->allocs.end());
            m->hb = m->hx = nullptr;
            m->h_cap = 0;
        }
        CGS_CUDA(m->alloc(&m->hb, n));
        CGS_CUDA(m->alloc(&m->hx, n));
        m->h_cap = n;
    }
    CGS_CUDA(cudaMemcpyAsync(m->hb, b_host, n * sizeof(double), cudaMemcpyHostToDevice, st));
    cgs_status s = cgs_solve(m, m->hb, m->hx, nrhs, rtol, maxit, iters, relres, stream);
    if (s == CGS_ERR_CUDA || s == CGS_ERR_OOM) return s;
    CGS_CUDA(cudaMemcpyAsync(x_host, m->hx, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CGS_CUDA(cudaStreamSynchronize(st));
    return s;
}

}  // extern "C"
