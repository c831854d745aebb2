// C ABI of the coarse-grid Schwarz solver (declared in include/cgs.h).
//
// A mesh owns its device data, one solve slot (scratch vectors, scalars) and
// an Engine: the work tables of that slot, the device-side PCG loop graph and
// launch accounting.  A batch is an Engine over many slots (meshes x
// right-hand sides) whose kernels cover all slots in each launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>
#include <iterator>
#include <map>
#include <unordered_map>
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

// Device allocations owned by one object, freed together.
struct DevAllocs {
    std::vector<void*> ptrs;
    size_t bytes = 0;
    template <typename T>
    cudaError_t alloc(T** out, size_t count) {
        void* p = nullptr;
        const size_t b = std::max<size_t>(count, 1) * sizeof(T);
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        bytes += b;
        *out = static_cast<T*>(p);
        return cudaSuccess;
    }
    template <typename T>
    cudaError_t upload(const T** out, const std::vector<T>& h) {
        T* p = nullptr;
        cudaError_t e = alloc(&p, h.size());
        if (e != cudaSuccess) return e;
        if (!h.empty()) e = cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        *out = p;
        return e;
    }
    void release() {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
        bytes = 0;
    }
};

// Shared solve machinery of a mesh (one slot) or a batch (many slots).
struct Engine {
    Plan P;
    Vecs V;                    // pools of the solve slots
    Schedule sch;              // block sizes of the work tables
    DevAllocs tables;          // the work tables (rebuilt by the tuner)
    // host-side builder of the work tables for a schedule
    std::function<void(const Schedule&, std::vector<Work> (&)[kWorkKinds])> build;
    bool f64 = true;
    cgs_precision prec = CGS_FP64;
    cgs_form form = CGS_HYBRID;
    int64_t total_v = 0;       // vertex entries over all slots
    SolveScalars* S_host = nullptr;   // pinned copy of the slot scalars
    cudaGraphExec_t gexec = nullptr;
    bool graph_failed = false;
    int last_iters = 8;
    // persistent loop (mixed forms, schedule.persistent): its grid barrier
    // and the resident block count
    GridBar* bar = nullptr;
    int pblocks_of[2] = {0, 0};   // persistent-loop blocks without / with packs above 32 dofs
    // launch accounting and the optional event profiler
    int64_t launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, size_t>> ev_used;
    size_t ev_next = 0;
    double prof_ms[CGS_K_COUNT] = {0};
    int64_t prof_n[CGS_K_COUNT] = {0};

    void release() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        if (bar) cudaFree(bar);
        bar = nullptr;
        tables.release();
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        ev_pool.clear();
        if (S_host) cudaFreeHost(S_host);
        S_host = nullptr;
    }
    cudaEvent_t next_event() {
        if (ev_next == ev_pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ev_pool.push_back(e);
        }
        return ev_pool[ev_next++];
    }
};

// Run one kernel launcher, counting it and, when profiling, bracketing it by
// events on its stream.
template <typename F>
inline void launch(Engine& E, int cls, cudaStream_t st, F&& f) {
    E.launches++;
    if (!E.prof) {
        f();
        return;
    }
    const size_t i0 = E.ev_next;
    cudaEventRecord(E.next_event(), st);
    f();
    cudaEventRecord(E.next_event(), st);
    E.ev_used.emplace_back(cls, i0);
}
#define K(cls, call) launch(E, (cls), st, [&]() { call; })

// Vecs for steps that must not stop early (no scalars).
Vecs no_stop(Vecs V) {
    V.S = nullptr;
    return V;
}

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
    DevMesh d;                 // host copy of the descriptor
    DevMesh* d_dev = nullptr;  // device copy
    MeshSizes sizes{};
    cgs_mesh_info_t info{};
    DevAllocs mem;
    Engine E;
    // host copies kept for cgs_mesh_export
    std::vector<uint8_t> dir_h;
    std::vector<int64_t> box_active_h, sub_ptr_h;
    std::vector<int32_t> sub_idx_h;
    double *hb = nullptr, *hx = nullptr;  // device staging for cgs_solve_host
    // status of the single-step calls (cgs_apply_*, cgs_restrict, ..., and
    // cgs_apply_preconditioner_noalloc): a bounded device wait that expired
    // leaves CGS_ERR_TIMEOUT here until cgs_mesh_step_status reads it
    SolveScalars* step_S = nullptr;
    size_t h_cap = 0;
    // projection onto prior solutions (cgs_mesh_set_projection): l x nv rows
    // of the A-orthonormal basis X and of A X, work vectors, dot results
    struct Projection {
        int l = 0, k = 0;
        double *X = nullptr, *AX = nullptr, *ubar = nullptr, *bp = nullptr;
        double *coef = nullptr, *partial = nullptr;
        double* host = nullptr;   // pinned copy of coef
        void release() {
            for (double* p : {X, AX, ubar, bp, coef, partial}) if (p) cudaFree(p);
            if (host) cudaFreeHost(host);
            *this = Projection();
        }
    } proj;
    bool fp64() const { return prm.prec == CGS_FP64; }
};

struct cgs_batch {
    cgs_ctx* ctx = nullptr;
    std::vector<cgs_mesh*> meshes;
    int nrhs = 1;
    DevAllocs mem;
    Engine E;
    const double** bptr_h = nullptr;   // pinned staging of the per-slot pointers
    double** xptr_h = nullptr;
    const double** bptr_d = nullptr;
    double** xptr_d = nullptr;
    int64_t max_nv = 0;
};

namespace {

cgs_params default_params() {
    cgs_params p{};
    p.box[0] = p.box[1] = p.box[2] = 4;
    p.box_margin = 0.0;
    p.overlap_layers = 1;
    p.prec = CGS_FP64;
    p.form = CGS_HYBRID;
    return p;
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

// z += J A_r^{-1} J^T s (s: the bulk copy of the residual or of r - A l;
// r_r = 0 on entry; restricted already when `restricted`).  dots: the
// per-vertex interpolation also forms the PCG dots z.r, z.q and beta;
// returns whether it did (the interpolation by cells leaves them to the
// dots kernel).
bool box_correction(Engine& E, const Vecs& V, bool dots, cudaStream_t st, bool restricted = false,
                    const cudaGraphConditionalHandle* cond = nullptr) {
    const Plan& P = E.P;
    if (E.f64) {
        if (!restricted) K(CGS_K_RESTRICT, launch_restrict(P, V, true, V.s, true, V.rr, false, st));
        if (P.any_xxt) K(CGS_K_COARSE, launch_xxt_pass1(P, V, false, V.rr, st));
        K(CGS_K_COARSE, launch_coarse(P, V, V.rr, V.ur, nullptr, st));
    } else {
        // r_r and the reduced product in float pairs, u_r rounded to float
        if (!restricted) K(CGS_K_RESTRICT, launch_restrict(P, V, false, V.s, false, V.rr, true, st));
        if (P.any_xxt) K(CGS_K_COARSE, launch_xxt_pass1(P, V, true, V.rr, st));
        K(CGS_K_COARSE, launch_coarse_pair(P, V, reinterpret_cast<const float2*>(V.rr), nullptr, V.ur32, st));
    }
    bool fused = false;
    K(CGS_K_INTERP, fused = launch_interp_add(P, V, E.f64, V.ur, E.f64 ? nullptr : V.ur32, V.z, dots, cond, st));
    return fused;
}

// z (bulk) = M r, with z = 0, s = r (bulk) and r_r = 0 on entry.  dots: also
// the PCG dots (fused into the per-vertex interpolation when there is a
// reduced space); returns whether they were formed.
bool precond_body(Engine& E, const Vecs& V, cudaStream_t st, bool dots = false,
                  const cudaGraphConditionalHandle* cond = nullptr) {
    const Plan& P = E.P;
    if (E.form == CGS_HYBRID) {
        K(CGS_K_LOCAL, launch_local(P, V, E.prec, V.s, V.z, 1, st));
        if (P.hyb_restrict) {
            // r_r = J~^T r - (A J~)^T l: s = r - A l is never formed
            K(CGS_K_RESTRICT, launch_restrict_hybrid(P, V, E.f64, V.s, V.z, V.rr, st));
            return box_correction(E, V, dots, st, true, cond);
        }
        if (E.f64)
            K(CGS_K_APPLY_A64, launch_apply64(P, V, static_cast<const double*>(V.z), static_cast<double*>(V.s), -1.0,
                                              false, st));
        else
            K(CGS_K_APPLY_A32,
              launch_apply28f_tiled(P, V, static_cast<const float*>(V.z), static_cast<float*>(V.s), -1.0f, st));
    } else if (E.form == CGS_RAS) {
        // restricted prolongation: a weight per subdomain entry
        K(CGS_K_LOCAL, launch_local(P, V, E.prec, V.s, V.z, 2, st));
    } else {
        // the restriction of s fused with the local solves when every
        // subdomain is in packs of at most 32 dofs (the conditions under
        // which launch_local_restrict launches)
        if (!E.f64 && !P.nwork[kWorkSub] && !P.lane_big && P.any_nr && P.nwork[kWorkBoxEnt]) {
            K(CGS_K_LOCAL, launch_local_restrict(P, V, E.prec, static_cast<const float*>(V.s),
                                                 static_cast<float*>(V.z), V.rr, st));
            return box_correction(E, V, dots, st, true, cond);
        }
        K(CGS_K_LOCAL, launch_local(P, V, E.prec, V.s, V.z, 0, st));
    }
    if (!P.any_nr) return false;
    return box_correction(E, V, dots, st, false, cond);
}

// One flexible-PCG iteration over every slot of the engine: float64 vectors
// in the FP64 form, float-pair vectors in the mixed forms.
void pcg_iteration(Engine& E, cudaStream_t st, const cudaGraphConditionalHandle* cond = nullptr) {
    const Plan& P = E.P;
    const Vecs& V = E.V;
    if (E.f64) {
        // the preconditioner reads its input without changing it unless the
        // hybrid step forms s = r - A l in place: then s must be a copy of r,
        // otherwise it is r itself (no copy written by the x, r update)
        Vecs Vi = V;
        if (P.hyb_restrict || E.form != CGS_HYBRID) Vi.s = V.r;
        K(CGS_K_APPLY_A64, launch_apply64(P, V, V.p, V.q, 1.0, true, st));
        K(CGS_K_PCG_XR, (launch_pcg_update_xr<double, double>(P, Vi, V.q, st)));
        if (!precond_body(E, Vi, st, true)) K(CGS_K_PCG_DOTS, (launch_pcg_dots<double, double>(P, Vi, V.q, st)));
        K(CGS_K_PCG_P, (launch_pcg_update_p<double, double>(P, Vi, V.q, cond, st)));
    } else {
        if (rows_outer(P)) {
            // q = A p by rows of the assembled A (p stored by the previous
            // iteration's p update), x and r, the preconditioner and the dots;
            // the p update closes the iteration and sets the loop condition
            K(CGS_K_APPLY_A64, launch_apply_outer(P, V, st));
            K(CGS_K_PCG_XR, launch_pcg_update_xr_pair(P, V, st, false));
            if (!precond_body(E, V, st, true, nullptr)) K(CGS_K_PCG_DOTS, launch_pcg_dots_pair(P, V, nullptr, st));
            K(CGS_K_PCG_P, launch_pcg_update_p_pair(P, V, cond, st));
        } else {
            // p = z + beta p is formed by the tiled apply and stored by the x,
            // r update; the interpolation (or the dots) closes the iteration
            // and sets the loop condition
            K(CGS_K_APPLY_A64, launch_apply_pair_tiled(P, V, st));
            K(CGS_K_PCG_XR, launch_pcg_update_xr_pair(P, V, st));
            if (!precond_body(E, V, st, true, cond)) K(CGS_K_PCG_DOTS, launch_pcg_dots_pair(P, V, cond, st));
        }
    }
}

// Start every slot of the plan: r = b, x = 0, z = M r, p = z, rho = r.z.
void pcg_start(Engine& E, const Plan& P, double rtol, int maxit, cudaStream_t st) {
    const Vecs& V = E.V;
    if (E.f64) {
        K(CGS_K_OTHER, launch_pcg_init<double>(P, V, V.q, rtol, maxit, st));
        K(CGS_K_OTHER, launch_precond_prep<double>(P, V, V.r, st));
    } else {
        K(CGS_K_OTHER, launch_pcg_init_pair(P, V, rtol, maxit, st));
        K(CGS_K_OTHER, launch_precond_prep_pair(P, V, st));
    }
    precond_body(E, V, st);
    if (E.f64)
        K(CGS_K_OTHER, launch_pcg_first_dir<double>(P, V, st));
    else
        K(CGS_K_OTHER, launch_pcg_first_dir_pair(P, V, st));
}

// Build the graph: one while node whose body is one PCG iteration over all
// slots plus the condition kernel (continue while some slot runs).
cgs_status build_loop_graph(Engine& E) {
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
    const bool prof = E.prof;
    const int64_t launches = E.launches;
    E.prof = false;
    {
        cudaStream_t st = cs;
        pcg_iteration(E, st, &h);   // its last kernel sets the loop condition
    }
    E.prof = prof;
    E.launches = launches;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    cs = nullptr;
    if (e != cudaSuccess) return bail(e, "cudaStreamEndCapture");
    if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) return bail(e, "cudaGraphInstantiate");
    cudaGraphDestroy(g);
    E.gexec = ex;
    return CGS_OK;
}

// Whether the engine runs its iterations in the persistent loop (mixed forms
// only): by the schedule, or (auto) when the element tiles of a launch fit
// about two per resident block.
// Resident blocks of the persistent loop for the engine's current plan (the
// variant with packs above 32 dofs holds one block per SM), cached.
int pblocks(Engine& E) {
    int& b = E.pblocks_of[E.P.lane_big ? 1 : 0];
    if (!b) b = persistent_blocks(E.prec, E.P.lane_big);
    return b;
}

bool use_persistent(Engine& E, const Schedule& sch) {
    // the persistent loop runs the dense reduced product only
    if (E.f64 || sch.persistent == 0 || E.P.any_xxt) return false;
    if (pblocks(E) <= 0) return false;
    return sch.persistent == 1;
}

// Launch the persistent loop for up to max_iters iterations of every slot.
cudaError_t persistent_launch(Engine& E, int max_iters, cudaStream_t st) {
    if (!E.bar) {
        cudaError_t e = cudaMalloc(&E.bar, sizeof(GridBar));
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemsetAsync(E.bar, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    K(CGS_K_LOOP, e = launch_pcg_persistent(E.P, E.V, E.prec, E.form == CGS_HYBRID, E.bar, max_iters, pblocks(E), st));
    return e;
}

// Solve every slot of the engine: V.b / V.bptr give the right-hand sides,
// the iterates stay in V.x (copied out through V.xptr when set).  On return
// E.S_host holds every slot's scalars (iters, status, res2, b2).
cgs_status engine_solve(Engine& E, double rtol, int maxit, cudaStream_t st) {
    const Plan& P = E.P;
    const Vecs& V = E.V;
    pcg_start(E, P, rtol, maxit, st);
    const bool persistent = use_persistent(E, E.sch);
    const bool use_graph = !E.prof && !E.graph_failed && !persistent;
    if (use_graph && !E.gexec) {
        if (build_loop_graph(E) != CGS_OK) E.graph_failed = true;
    }
    const size_t sbytes = sizeof(SolveScalars) * (size_t)P.nslots;
    if (persistent) {
        // every iteration in one cooperative launch
        CGS_CUDA(persistent_launch(E, maxit + 2, st));
    } else if (use_graph && E.gexec) {
        // the whole iteration loop runs on the device
        CGS_CUDA(cudaGraphLaunch(E.gexec, st));
        E.launches += 1;
    } else {
        int enqueued = 0;
        int chunk = std::max(2, E.last_iters);
        for (;;) {
            const int n = std::min(chunk, maxit - enqueued);
            for (int i = 0; i < n; ++i) pcg_iteration(E, st);
            enqueued += n;
            CGS_CUDA(cudaMemcpyAsync(E.S_host, V.S, sbytes, cudaMemcpyDeviceToHost, st));
            CGS_CUDA(cudaStreamSynchronize(st));
            bool all = true;
            for (int s = 0; s < P.nslots; ++s) all = all && E.S_host[s].done;
            if (all || enqueued >= maxit) break;
            chunk = 4;
        }
    }
    // the true residual ||b - A x|| over the free entries (and copy-out)
    const Vecs Vn = no_stop(V);
    if (!E.f64) K(CGS_K_OTHER, launch_finalize_x_pair(P, V, st));
    launch_fill_d(E.total_v, V.y, 0.0, st);
    K(CGS_K_OTHER, launch_apply64(P, Vn, V.x, V.y, 1.0, false, st));
    K(CGS_K_OTHER, launch_resid_norm(P, V, st));
    CGS_CUDA(cudaMemcpyAsync(E.S_host, V.S, sbytes, cudaMemcpyDeviceToHost, st));
    cgs_status fs = finish(st, true);
    if (fs != CGS_OK) return fs;
    int most = 0;
    for (int s = 0; s < P.nslots; ++s) most = std::max(most, E.S_host[s].iters);
    if (most > 0) E.last_iters = most;
    return CGS_OK;
}

cgs_status slot_status(const SolveScalars& h) {
    const int status = h.done ? h.status : CGS_ERR_NO_CONVERGENCE;
    if (status == CGS_ERR_NO_CONVERGENCE) g_err = "maxit reached before the tolerance";
    if (status == CGS_ERR_BREAKDOWN) g_err = "breakdown in the PCG iteration";
    if (status == CGS_ERR_TIMEOUT) g_err = "a bounded device wait expired";
    return (cgs_status)status;
}

double slot_relres(const SolveScalars& h) { return h.b2 > 0 ? std::sqrt(h.res2 / h.b2) : 0.0; }

// Allocate the pooled vectors of `nslots` slots with `total_v` vertex and
// `total_r` reduced entries, `total_p` partials.
cudaError_t alloc_pools(DevAllocs& mem, Engine& E, int64_t total_v, int64_t total_r, int64_t total_p, int nslots) {
    cudaError_t e;
    Vecs& V = E.V;
#define TRY(x)                          \
    if ((e = (x)) != cudaSuccess) return e;
    TRY(mem.alloc(&V.x, total_v));
    TRY(mem.alloc(&V.r, total_v));
    TRY(mem.alloc(&V.p, total_v));
    TRY(mem.alloc(&V.y, total_v));
    if (E.f64) {
        TRY(mem.alloc(&V.q, total_v));
        double *z, *s;
        TRY(mem.alloc(&z, total_v));
        TRY(mem.alloc(&s, total_v));
        V.z = z;
        V.s = s;
    } else {
        TRY(mem.alloc(&V.q2, total_v));
        V.p2 = reinterpret_cast<float2*>(V.p);   // p is a float pair in the mixed forms
        float *z, *s;
        TRY(mem.alloc(&z, total_v));
        TRY(mem.alloc(&s, total_v));
        V.z = z;
        V.s = s;
        TRY(mem.alloc(&V.ur32, std::max<int64_t>(total_r, 1)));
    }
    TRY(mem.alloc(&V.rr, std::max<int64_t>(total_r, 1)));
    TRY(mem.alloc(&V.ur, std::max<int64_t>(total_r, 1)));
    TRY(mem.alloc(&V.rt, std::max<int64_t>(total_r, 1)));
    TRY(mem.alloc(&V.partials, std::max<int64_t>(total_p, 2)));
    TRY(mem.alloc(&V.S, nslots));
    TRY(cudaMemset(V.S, 0, sizeof(SolveScalars) * nslots));
    TRY(cudaMallocHost(&E.S_host, sizeof(SolveScalars) * nslots));
#undef TRY
    E.total_v = total_v;
    return cudaSuccess;
}

// Whether every slot with a reduced space has hybrid-restriction ranges
// (then the hybrid step restricts r and l directly, without s = r - A l).
bool hyb_restrict_ok(const Plan& P, const std::vector<Work> (&tabs)[kWorkKinds]) {
    if (!P.any_nr || tabs[kWorkHybR].empty()) return false;
    std::vector<char> with_box, with_hr;
    for (const Work& w : tabs[kWorkBoxEnt]) {
        if ((size_t)w.slot >= with_box.size()) with_box.resize(w.slot + 1, 0);
        with_box[w.slot] = 1;
    }
    for (const Work& w : tabs[kWorkHybR]) {
        if ((size_t)w.slot >= with_hr.size()) with_hr.resize(w.slot + 1, 0);
        with_hr[w.slot] = 1;
    }
    for (size_t k = 0; k < with_box.size(); ++k)
        if (with_box[k] && (k >= with_hr.size() || !with_hr[k])) return false;
    return true;
}

// (Re)build the work tables of an engine for a schedule and upload them.
cudaError_t set_schedule(Engine& E, const Schedule& sch) {
    std::vector<Work> tabs[kWorkKinds];
    E.build(sch, tabs);
    DevAllocs fresh;
    Plan P = E.P;
    for (int k = 0; k < kWorkKinds; ++k) {
        const Work* p = nullptr;
        cudaError_t e = fresh.upload(&p, tabs[k]);
        if (e != cudaSuccess) {
            fresh.release();
            return e;
        }
        P.work[k] = p;
        P.nwork[k] = (unsigned int)tabs[k].size();
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fresh.release();
        return e;
    }
    E.tables.release();
    E.tables = fresh;
    P.tile_tma = sch.tile_tma != 0;
    P.pack_chunk = sch.pack_chunk;
    P.pdl = sch.pdl != 0;
    P.interp_cells = sch.interp_cells != 0;
    P.any_xxt = P.nwork[kWorkXSeg] > 0;
    P.hyb_restrict = hyb_restrict_ok(P, tabs);
    E.P = P;
    E.sch = sch;
    if (E.gexec) {   // the captured loop holds the old grid sizes
        cudaGraphExecDestroy(E.gexec);
        E.gexec = nullptr;
    }
    return cudaSuccess;
}

bool P_any_nr(const Engine& E) { return E.P.any_nr; }

// Autotuner: time the local solves for each subdomain chunk and a vertex
// kernel for each vertex chunk on the engine's own data, keep the fastest.
cgs_status tune_engine(Engine& E, cudaStream_t st) {
    const int verts[] = {256, 512, 1024, 2048};
    const int subs[] = {8, 16, 32, 64};
    cudaEvent_t a, b;
    CGS_CUDA(cudaEventCreate(&a));
    CGS_CUDA(cudaEventCreate(&b));
    const Vecs V = no_stop(E.V);
    auto time_it = [&](auto&& body) -> float {
        body();   // warm-up
        cudaEventRecord(a, st);
        for (int r = 0; r < 3; ++r) body();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    };
    Schedule best = E.sch;
    float best_sub = 1e30f, best_vert = 1e30f;
    for (int sc : subs) {
        Schedule t = E.sch;
        t.sub_chunk = sc;
        if (set_schedule(E, t) != cudaSuccess) continue;
        const float ms = time_it([&]() { launch_local(E.P, V, E.prec, V.s, V.z, true, st); });
        if (ms < best_sub) {
            best_sub = ms;
            best.sub_chunk = sc;
        }
    }
    for (int vc : verts) {
        Schedule t = E.sch;
        t.vert_chunk = vc;
        if (set_schedule(E, t) != cudaSuccess) continue;
        const float ms = time_it([&]() {
            if (E.f64)
                launch_precond_prep<double>(E.P, V, V.r, st);
            else
                launch_precond_prep_pair(E.P, V, st);
        });
        if (ms < best_vert) {
            best_vert = ms;
            best.vert_chunk = vc;
        }
    }
    // box-list vertices per interpolation block (mixed forms; the FP64
    // form's interpolation by rows closes with the PCG dots, whose per-slot
    // reduction a timing run without slot scalars cannot include, so it keeps
    // the default of about seven blocks per SM)
    if (P_any_nr(E) && !E.f64) {
        float best_box = 1e30f;
        for (int bc : {256, 512, 768, 1024, 2048}) {
            Schedule t = best;
            t.box_chunk = bc;
            if (set_schedule(E, t) != cudaSuccess) continue;
            const float ms = time_it([&]() {
                launch_interp_add(E.P, V, E.f64, V.ur, E.f64 ? nullptr : V.ur32, V.z, false, nullptr, st);
            });
            if (ms < best_box) {
                best_box = ms;
                best.box_chunk = bc;
            }
        }
    }
    // interpolation by vertex with the dots fused, or by cells followed by
    // the dots kernel (mixed forms; the FP64 form interpolates by rows)
    if (P_any_nr(E) && !E.f64) {
        float best_ip = 1e30f;
        for (int ic = 0; ic < 2; ++ic) {
            Schedule t = best;
            t.interp_cells = ic;
            if (set_schedule(E, t) != cudaSuccess) continue;
            const float ms = time_it([&]() {
                if (!launch_interp_add(E.P, V, E.f64, V.ur, E.f64 ? nullptr : V.ur32, V.z, true, nullptr, st)) {
                    if (E.f64)
                        launch_pcg_dots<double, double>(E.P, V, V.q, st);
                    else
                        launch_pcg_dots_pair(E.P, V, nullptr, st);
                }
            });
            if (ms < best_ip) {
                best_ip = ms;
                best.interp_cells = ic;
            }
        }
    }
    // mixed forms: element tiles staged by TMA or streamed by the threads
    if (!E.f64) {
        float best_tile = 1e30f;
        for (int tma = 0; tma < 2; ++tma) {
            Schedule t = best;
            t.tile_tma = tma;
            if (set_schedule(E, t) != cudaSuccess) continue;
            const float ms = time_it([&]() {
                launch_apply_outer(E.P, V, st);
                launch_apply28f_tiled(E.P, V, static_cast<const float*>(V.z), static_cast<float*>(V.s), -1.0f, st);
            });
            if (ms < best_tile) {
                best_tile = ms;
                best.tile_tma = tma;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CGS_CUDA(set_schedule(E, best));
    return finish(st, true);
}

}  // namespace

namespace cgs {
// Read-only views of a mesh for entry points defined in other files.
const DevMesh& mesh_dev(const cgs_mesh* m) { return m->d; }
const Plan& mesh_plan(const cgs_mesh* m) { return m->E.P; }
cgs_precision mesh_prec(const cgs_mesh* m) { return m->prm.prec; }
cgs_form mesh_form(const cgs_mesh* m) { return m->E.form; }
const uint8_t* mesh_dir(const cgs_mesh* m) { return m->d.dir; }
int mesh_device(const cgs_mesh* m) { return m->ctx->device; }
SolveScalars* mesh_step_status_word(cgs_mesh* m, cudaStream_t st) {
    cudaMemsetAsync(&m->step_S->done, 0, sizeof(int), st);
    return m->step_S;
}
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
    if (prm.prec < CGS_FP64 || prm.prec > CGS_FP16_LOCAL || prm.form < CGS_HYBRID || prm.form > CGS_RAS)
        return fail(CGS_ERR_INVALID_ARG, "unknown precision or form");
    if (prm.local_cg_steps < 0 || prm.local_cg_steps > 1024 ||
        (prm.local_cg_steps > 0 && prm.prec == CGS_FP16_LOCAL))
        return fail(CGS_ERR_INVALID_ARG, "local_cg_steps must be in [0, 1024], and 0 in the FP16-local form");
    if (prm.fault_negate_subdomain < 0) return fail(CGS_ERR_INVALID_ARG, "fault_negate_subdomain must be >= 0");
    CGS_CUDA(cudaSetDevice(ctx->device));
    HostSetup hs;
    std::string err;
    cgs_status st = host_setup(xyz, nv, conn, ne, dirichlet, elem_part, prm, hs, err);
    if (st != CGS_OK) return fail(st, err);

    const bool f64 = prm.prec == CGS_FP64;
    // estimated footprint for admission before allocating
    const size_t bulk = f64 ? 8 : 4;
    const size_t est = (size_t)ne * (8 * 4 + kUpper * 8 + 4) + (f64 ? 0 : hs.at_hi.size() * 8 + (size_t)ne * 16) +
                       (size_t)nv * (32 + 16 + 1 + 8 + 4) + hs.sub_idx.size() * 4 +
                       (hs.inv.size() + hs.pack_inv.size() + hs.rpack_inv.size()) *
                           (f64 ? 8 : prm.prec == CGS_FP32_BULK ? 4 : 2) +
                       (hs.pack_idx.size() + hs.rpack_idx.size()) * 4 + hs.ar_inv.size() * 8 +
                       hs.xc_idx.size() * 20 + hs.xs_seg.size() * 4 + hs.xr_ptr.size() * 4 +
                       (size_t)nv * (5 * 8 + 2 * bulk);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->budget && ctx->in_use + est > ctx->budget)
            return fail(CGS_ERR_ADMISSION, "mesh footprint exceeds the context's HBM budget");
    }

    cgs_mesh* m = new (std::nothrow) cgs_mesh;
    if (!m) return fail(CGS_ERR_INVALID_ARG, "host allocation failed");
    m->ctx = ctx;
    m->prm = prm;
    DevMesh& d = m->d;
    d.nv = nv;
    d.ne = ne;
    d.n_sub = hs.n_wsub;
    d.n_pack = (int64_t)hs.pack_m.size();
    for (int c : hs.pack_m) d.max_pack_m = std::max(d.max_pack_m, c);
    for (int c : hs.rpack_m) d.max_pack_m = std::max(d.max_pack_m, c);
    d.nr = hs.nr;
    for (int k = 0; k < 3; ++k) {
        d.b[k] = hs.b[k];
        d.lo[k] = 0.0;   // coordinates are stored relative to the box origin
        d.H[k] = hs.H[k];
        d.iH[k] = 1.0 / hs.H[k];
        d.Hf[k] = (float)d.H[k];
        d.iHf[k] = (float)d.iH[k];
    }
    d.max_m = (int)hs.max_wm;

    auto cleanup = [&](cgs_status s) {
        m->E.release();
        m->mem.release();
        delete m;
        return s;
    };
#define UP(ptr, vec)                                                      \
    do {                                                                  \
        cudaError_t e_ = m->mem.upload(&(ptr), (vec));                    \
        if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, "upload"));    \
    } while (0)

    UP(d.conn, hs.conn);
    UP(d.a36, hs.a36);
    if (!hs.ell_ptr.empty()) {
        d.nslice = (int64_t)hs.ell_ptr.size() - 1;
        d.ell_w = hs.ell_w;
        UP(d.ell_ptr, hs.ell_ptr);
        UP(d.ell_col, hs.ell_col);
        if (!hs.ell_val.empty()) UP(d.ell_val, hs.ell_val);
        if (!hs.ell_pair.empty()) {
            const float* pp = nullptr;
            UP(pp, hs.ell_pair);
            d.ell_pair = reinterpret_cast<const float2*>(pp);
        }
    }
    UP(d.cell, hs.cell);
    if (!f64) {
        d.ntiles = (int64_t)hs.tile_ptr.size() - 1;
        UP(d.tile_ptr, hs.tile_ptr);
        UP(d.tile_vptr, hs.tile_vptr);
        UP(d.tile_verts, hs.tile_verts);
        UP(d.eloc, hs.eloc);
        UP(d.at_hi, hs.at_hi);
        UP(d.at_lo, hs.at_lo);
    }
    UP(d.cell_cols, hs.cell_cols);
    d.nvb = (int64_t)hs.vb_vert.size();
    if (d.nvb) {
        UP(d.vb_vert, hs.vb_vert);
        UP(d.vb_ptr, hs.vb_ptr);
        UP(d.vb_cell, hs.vb_cell);
        d.nre = (int64_t)hs.re_vert.size();
        UP(d.re_vert, hs.re_vert);
        UP(d.re_cell, hs.re_cell);
        d.nrng = (int64_t)hs.re_rng.size() / 2;
        {
            const int32_t* rp = nullptr;
            UP(rp, hs.re_rng);
            d.re_rng = reinterpret_cast<const int2*>(rp);
        }
        if (f64) {
            UP(d.vb_w64, hs.vb_w);
            UP(d.re_w64, hs.re_w);
            // explicit rows of J~ for the float64 interpolation
            UP(d.jt_vert, hs.jt_vert);
            UP(d.jt_ptr, hs.jt_ptr);
            UP(d.jt_col, hs.jt_col);
            UP(d.jt_val, hs.jt_val);
        } else {
            UP(d.vb_w32, std::vector<float>(hs.vb_w.begin(), hs.vb_w.end()));
            UP(d.re_w32, std::vector<float>(hs.re_w.begin(), hs.re_w.end()));
        }
    }
    d.nhr = (int64_t)hs.hr_rng.size() / 4;
    if (d.nhr) {
        const int32_t* rp = nullptr;
        UP(rp, hs.hr_rng);
        d.hr_rng = reinterpret_cast<const int4*>(rp);
        UP(d.hr_vert, hs.hr_vert);
        const size_t nh = hs.hr_vert.size();
        if (f64) {
            std::vector<double2> jg(nh);
            for (size_t i = 0; i < nh; ++i) jg[i] = make_double2(hs.hr_j[i], hs.hr_g[i]);
            UP(d.hr_jg64, jg);
        } else {
            std::vector<float2> jg(nh);
            for (size_t i = 0; i < nh; ++i) jg[i] = make_float2((float)hs.hr_j[i], (float)hs.hr_g[i]);
            UP(d.hr_jg32, jg);
        }
    }
    {
        std::vector<int32_t> sp(hs.wsub_ptr.begin(), hs.wsub_ptr.end());
        UP(d.sub_ptr, sp);
    }
    UP(d.sub_idx, hs.wsub_idx);
    UP(d.inv_ptr, hs.inv_ptr);
    d.cg_steps = prm.local_cg_steps;
    if (prm.prec == CGS_FP64) {
        UP(d.inv64, hs.inv);
        UP(d.went64, hs.wsub_ras);
        if (d.cg_steps) UP(d.ap64, hs.ap);
    } else if (prm.prec == CGS_FP32_BULK) {
        std::vector<float> f(hs.inv.begin(), hs.inv.end());
        UP(d.inv32, f);
        UP(d.went32, std::vector<float>(hs.wsub_ras.begin(), hs.wsub_ras.end()));
        if (d.cg_steps) UP(d.ap32, std::vector<float>(hs.ap.begin(), hs.ap.end()));
    } else {
        UP(d.went32, std::vector<float>(hs.wsub_ras.begin(), hs.wsub_ras.end()));
        std::vector<__half> h(hs.inv.size());
        std::vector<float> sc(hs.n_wsub, 1.0f);
        for (int64_t p = 0; p < hs.n_wsub; ++p) {
            double mx = 0.0;
            for (int64_t i = hs.inv_ptr[p]; i < hs.inv_ptr[p + 1]; ++i) mx = std::max(mx, std::fabs(hs.inv[i]));
            const double s = mx > 0 ? mx : 1.0;
            sc[p] = (float)s;
            for (int64_t i = hs.inv_ptr[p]; i < hs.inv_ptr[p + 1]; ++i) h[i] = __float2half_rn((float)(hs.inv[i] / s));
        }
        UP(d.inv16, h);
        UP(d.inv16_scale, sc);
    }
    if (d.n_pack) {
        // lane packs: host [pack][lane][entry] -> device groups across lanes
        const int64_t np = d.n_pack;
        UP(d.pack_m, hs.pack_m);
        UP(d.pack_idx_off, std::vector<int64_t>(hs.pack_idx_off.begin(), hs.pack_idx_off.end() - 1));
        UP(d.pack_inv_off, std::vector<int64_t>(hs.pack_inv_off.begin(), hs.pack_inv_off.end() - 1));
        UP(d.pack_idx, hs.pack_idx);
        if (f64)
            UP(d.pack_went64, hs.pack_ras);
        else
            UP(d.pack_went32, std::vector<float>(hs.pack_ras.begin(), hs.pack_ras.end()));
        const size_t total = hs.pack_inv.size();
        if (prm.prec == CGS_FP64) {
            // 16-byte groups of two entries across the 32 lanes
            std::vector<double> f(total);
            for (int64_t P = 0; P < np; ++P) {
                const int64_t ao = hs.pack_inv_off[P], T = lane_entries(hs.pack_m[P]);
                for (int l = 0; l < 32; ++l)
                    for (int64_t e = 0; e < T; ++e)
                        f[ao + (e / 2) * 64 + l * 2 + e % 2] = hs.pack_inv[ao + l * T + e];
            }
            UP(d.pack_inv64, f);
        } else if (prm.prec == CGS_FP32_BULK) {
            std::vector<float> f(total);
            for (int64_t P = 0; P < np; ++P) {
                const int64_t ao = hs.pack_inv_off[P], T = lane_entries(hs.pack_m[P]);
                for (int l = 0; l < 32; ++l)
                    for (int64_t e = 0; e < T; ++e)
                        f[ao + (e / 4) * 128 + l * 4 + e % 4] = (float)hs.pack_inv[ao + l * T + e];
            }
            UP(d.pack_inv32, f);
        } else {
            std::vector<__half> h(total);
            std::vector<float> sc((size_t)np * 32, 1.0f);
            for (int64_t P = 0; P < np; ++P) {
                const int64_t ao = hs.pack_inv_off[P], T = lane_entries(hs.pack_m[P]);
                for (int l = 0; l < 32; ++l) {
                    double mx = 0.0;
                    for (int64_t e = 0; e < T; ++e) mx = std::max(mx, std::fabs(hs.pack_inv[ao + l * T + e]));
                    const double s = mx > 0 ? mx : 1.0;
                    sc[(size_t)P * 32 + l] = (float)s;
                    for (int64_t e = 0; e < T; ++e)
                        h[ao + (e / 8) * 256 + l * 8 + e % 8] =
                            __float2half_rn((float)(hs.pack_inv[ao + l * T + e] / s));
                }
            }
            UP(d.pack_inv16, h);
            UP(d.pack_scale, sc);
        }
    }
    if (!hs.rpack_m.empty()) {
        // row packs: host [pack][lane][entry] -> device groups across lanes
        d.n_rpack = (int64_t)hs.rpack_m.size();
        UP(d.rpack_m, hs.rpack_m);
        UP(d.rpack_idx_off, std::vector<int64_t>(hs.rpack_idx_off.begin(), hs.rpack_idx_off.end() - 1));
        UP(d.rpack_inv_off, std::vector<int64_t>(hs.rpack_inv_off.begin(), hs.rpack_inv_off.end() - 1));
        UP(d.rpack_idx, hs.rpack_idx);
        UP(d.rpack_went32, std::vector<float>(hs.rpack_ras.begin(), hs.rpack_ras.end()));
        const size_t total = hs.rpack_inv.size();
        if (prm.prec == CGS_FP32_BULK) {
            std::vector<float> f(total);
            for (int64_t P = 0; P < d.n_rpack; ++P) {
                const int64_t ao = hs.rpack_inv_off[P], T = row_entries(hs.rpack_m[P]);
                for (int l = 0; l < 32; ++l)
                    for (int64_t e = 0; e < T; ++e)
                        f[ao + (e / 4) * 128 + l * 4 + e % 4] = (float)hs.rpack_inv[ao + l * T + e];
            }
            UP(d.rpack_inv32, f);
        } else {
            std::vector<__half> h(total);
            std::vector<float> sc((size_t)d.n_rpack * 32, 1.0f);
            for (int64_t P = 0; P < d.n_rpack; ++P) {
                const int64_t ao = hs.rpack_inv_off[P], T = row_entries(hs.rpack_m[P]);
                for (int l = 0; l < 32; ++l) {
                    double mx = 0.0;
                    for (int64_t e = 0; e < T; ++e) mx = std::max(mx, std::fabs(hs.rpack_inv[ao + l * T + e]));
                    const double sv = mx > 0 ? mx : 1.0;
                    sc[(size_t)P * 32 + l] = (float)sv;
                    for (int64_t e = 0; e < T; ++e)
                        h[ao + (e / 8) * 256 + l * 8 + e % 8] =
                            __float2half_rn((float)(hs.rpack_inv[ao + l * T + e] / sv));
                }
            }
            UP(d.rpack_inv16, h);
            UP(d.rpack_scale, sc);
        }
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
    if (hs.nr && hs.coarse == CGS_COARSE_XXT) {
        // X by columns (segmented) and by rows; values float64 (FP64 form) or
        // hi/lo float pairs (mixed forms), 8 bytes either way
        d.xxt = 1;
        d.nxseg = (int64_t)hs.xs_seg.size() / 4;
        const int32_t* seg = nullptr;
        UP(seg, hs.xs_seg);
        d.xs_seg = reinterpret_cast<const int4*>(seg);
        UP(d.xc_idx, hs.xc_idx);
        UP(d.xr_idx, hs.xr_idx);
        UP(d.xr_ptr, hs.xr_ptr);
        auto vals = [&](const std::vector<double>& v, const void** out) -> cudaError_t {
            if (f64) {
                const double* p = nullptr;
                cudaError_t e = m->mem.upload(&p, v);
                *out = p;
                return e;
            }
            std::vector<float2> v2(v.size());
            for (size_t i = 0; i < v.size(); ++i) {
                const float h = (float)v[i];
                v2[i] = make_float2(h, (float)(v[i] - (double)h));
            }
            const float2* p = nullptr;
            cudaError_t e = m->mem.upload(&p, v2);
            *out = p;
            return e;
        };
        cudaError_t e1 = vals(hs.xc_val, &d.xc_val);
        if (e1 == cudaSuccess) e1 = vals(hs.xr_val, &d.xr_val);
        if (e1 != cudaSuccess) return cleanup(cuda_fail(e1, "upload"));
    } else if (hs.nr && f64) {
        UP(d.ar_inv, hs.ar_inv);
    } else if (hs.nr) {
        // hi = entry rounded to float, lo = the rounded remainder; rows padded
        // to an even length (16-byte aligned row starts)
        const int64_t nr = hs.nr, nr2 = (nr + 1) / 2 * 2;
        std::vector<float2> a2((size_t)nr * nr2, make_float2(0.0f, 0.0f));
        for (int64_t i = 0; i < nr; ++i)
            for (int64_t j = 0; j < nr; ++j) {
                const double a = hs.ar_inv[(size_t)i * nr + j];
                const float h = (float)a;
                a2[(size_t)i * nr2 + j] = make_float2(h, (float)(a - (double)h));
            }
        d.nr2 = nr2;
        UP(d.ar_inv2, a2);
    }
    UP(d.dir, hs.dir);
    {
        cudaError_t e_ = m->mem.alloc(&m->step_S, 1);
        if (e_ == cudaSuccess) e_ = cudaMemset(m->step_S, 0, sizeof(SolveScalars));
        if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, "step status"));
    }
    {
        const DevMesh* dd = nullptr;
        UP(dd, std::vector<DevMesh>{d});
        m->d_dev = const_cast<DevMesh*>(dd);
    }
    // one solve slot and its work tables
    m->sizes = MeshSizes{nv, ne, d.ntiles, hs.n_wsub, hs.nr, d.n_pack, d.nvb, d.nrng, d.n_rpack, d.nxseg, d.nhr};
    Engine& E = m->E;
    E.f64 = f64;
    E.prec = prm.prec;
    E.form = prm.form;
    E.P.meshes = m->d_dev;
    E.P.nslots = 1;
    E.P.max_m = d.max_m;
    E.P.any_nr = hs.nr > 0;
    E.P.hyb_restrict = d.nhr > 0;
    E.P.lane_big = d.max_pack_m > 32;
    E.P.ell = d.nslice > 0 && d.ell_val;
    E.P.ell_pair = d.nslice > 0 && d.ell_pair;
    {
        const MeshSizes sz = m->sizes;
        E.build = [sz](const Schedule& sch, std::vector<Work> (&tabs)[kWorkKinds]) {
            append_mesh_work(tabs, 0, 0, 0, 0, 0, sz, sch);
        };
        Schedule smallest;
        smallest.vert_chunk = 256;
        smallest.sub_chunk = 8;
        smallest.box_chunk = 256;
        cudaError_t e = alloc_pools(m->mem, E, nv, hs.nr, mesh_partial_slots(sz, smallest), 1);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "scratch"));
        e = set_schedule(E, default_schedule(nv, hs.n_wsub, d.n_pack, d.n_pack * 32));
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "work tables"));
    }
    {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "setup upload"));
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->budget && ctx->in_use + m->mem.bytes > ctx->budget)
            return cleanup(fail(CGS_ERR_ADMISSION, "mesh footprint exceeds the context's HBM budget"));
        ctx->in_use += m->mem.bytes;
        ctx->live_meshes++;
    }
#undef UP
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
    m->info.sum_sub_tri = 0;
    for (size_t p = 0; p + 1 < m->sub_ptr_h.size(); ++p) {   // hs.sub_ptr was moved to the export copy
        const int64_t mp = m->sub_ptr_h[p + 1] - m->sub_ptr_h[p];
        m->info.sum_sub_tri += mp * (mp + 1) / 2;
    }
    m->info.n_box_entries = (int64_t)hs.vb_cell.size();
    m->info.n_lane_packs = (int64_t)hs.pack_m.size();
    m->info.coarse_solver = hs.coarse;
    m->info.ar_nnz = hs.ar_nnz;
    m->info.coarse_operator = prm.coarse_operator;
    m->info.xxt_nnz = (int64_t)hs.xc_idx.size();
    m->info.n_hyb_entries = (int64_t)hs.hr_vert.size();
    m->info.n_jt_entries = f64 ? hs.jt_nnz : 0;
    m->info.ell_slots = (int64_t)hs.ell_col.size();
    m->info.ell_nnz = 0;
    for (int32_t c : hs.ell_col) m->info.ell_nnz += c >= 0;
    m->info.footprint_bytes = m->mem.bytes;
    m->info.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = m;
    return CGS_OK;
}

cgs_status cgs_mesh_free(cgs_mesh* m) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    cudaSetDevice(m->ctx->device);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> lk(m->ctx->mu);
        m->ctx->in_use -= m->info.footprint_bytes;
        m->ctx->live_meshes--;
    }
    if (m->hb) cudaFree(m->hb);
    if (m->hx) cudaFree(m->hx);
    m->proj.release();
    m->E.release();
    m->mem.release();
    delete m;
    return CGS_OK;
}

cgs_status cgs_mesh_info(const cgs_mesh* m, cgs_mesh_info_t* info) {
    if (!m || !info) return fail(CGS_ERR_INVALID_ARG, "null argument");
    *info = m->info;
    info->kernel_launches = m->E.launches;
    {
        Engine& E = const_cast<Engine&>(m->E);
        info->loop = use_persistent(E, E.sch) ? 2 : (E.graph_failed ? 0 : 1);
    }
    return CGS_OK;
}

cgs_status cgs_mesh_set_form(cgs_mesh* m, cgs_form form) {
    if (!m || form < CGS_HYBRID || form > CGS_RAS) return fail(CGS_ERR_INVALID_ARG, "bad mesh or form");
    if (form != m->E.form && m->E.gexec) {   // the captured loop holds the old form
        cudaDeviceSynchronize();
        cudaGraphExecDestroy(m->E.gexec);
        m->E.gexec = nullptr;
    }
    m->E.form = form;
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

cgs_status cgs_profile_enable(cgs_mesh* m, int enable) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    m->E.prof = enable != 0;
    return CGS_OK;
}

cgs_status cgs_profile_read(cgs_mesh* m, double* ms, int64_t* launches) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    Engine& E = m->E;
    if (!E.ev_used.empty()) {
        CGS_CUDA(cudaEventSynchronize(E.ev_pool[E.ev_used.back().second + 1]));
        for (const auto& u : E.ev_used) {
            float t = 0.0f;
            CGS_CUDA(cudaEventElapsedTime(&t, E.ev_pool[u.second], E.ev_pool[u.second + 1]));
            E.prof_ms[u.first] += t;
            E.prof_n[u.first] += 1;
        }
    }
    E.ev_used.clear();
    E.ev_next = 0;
    for (int k = 0; k < CGS_K_COUNT; ++k) {
        if (ms) ms[k] = E.prof_ms[k];
        if (launches) launches[k] = E.prof_n[k];
        E.prof_ms[k] = 0.0;
        E.prof_n[k] = 0;
    }
    return CGS_OK;
}

// ---- single steps: user buffers take the place of the slot's vectors -------

namespace {
// Vecs of a single-step call: the slot scalars are the mesh's step status
// word, which only bounded waits write.  Its stop flag is cleared first, so
// a wait that expired in an earlier call does not skip this call's work; the
// recorded timeout stays until cgs_mesh_step_status reads it.
Vecs step_vecs(cgs_mesh* m, cudaStream_t st) {
    Vecs V = m->E.V;
    V.S = m->step_S;
    V.step = 1;
    cudaMemsetAsync(&m->step_S->done, 0, sizeof(int), st);
    return V;
}
}  // namespace

cgs_status cgs_apply_A(cgs_mesh* m, const double* x, double* y, void* stream) {
    if (!m || !x || !y) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = m->E;
    const Vecs V = step_vecs(m, st);
    K(CGS_K_OTHER, launch_fill_d(m->d.nv, y, 0.0, st));
    K(CGS_K_APPLY_A64, launch_apply64(E.P, V, x, y, 1.0, false, st));
    return finish(st, false);
}

cgs_status cgs_apply_A_prec(cgs_mesh* m, const double* x, double* y, int op, void* stream) {
    if (!m || !x || !y) return fail(CGS_ERR_INVALID_ARG, "null argument");
    if (op < CGS_OP_FP64 || op > CGS_OP_OUTER) return fail(CGS_ERR_INVALID_ARG, "unknown operator");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = m->E;
    const Vecs V = step_vecs(m, st);
    const int64_t nv = m->d.nv;
    if (m->fp64() || op == CGS_OP_FP64) {
        K(CGS_K_OTHER, launch_fill_d(nv, y, 0.0, st));
        K(CGS_K_APPLY_A64, launch_apply64(E.P, V, x, y, 1.0, false, st));
    } else if (op == CGS_OP_INNER) {
        // x rounded to float, y = A x accumulated in float, then widened
        float* xf = static_cast<float*>(V.z);
        float* yf = static_cast<float*>(V.s);
        K(CGS_K_OTHER, launch_convert_d2f(E.P, x, xf, true, st));
        K(CGS_K_OTHER, launch_fill_f(nv, yf, 0.0f, st));
        K(CGS_K_APPLY_A32, launch_apply28f_tiled(E.P, V, xf, yf, 1.0f, st));
        K(CGS_K_OTHER, launch_convert_f2d(E.P, yf, y, true, st));
    } else {
        // x split into float pairs, y = A x in float-pair arithmetic
        K(CGS_K_OTHER, launch_split_pair(nv, x, V.p2, st));
        K(CGS_K_OTHER, launch_fill_d(nv, reinterpret_cast<double*>(V.q2), 0.0, st));
        K(CGS_K_APPLY_A64, launch_apply_outer(E.P, V, st));
        K(CGS_K_OTHER, launch_pair_to_double(nv, V.q2, y, st));
    }
    return finish(st, false);
}

cgs_status cgs_mesh_step_status(cgs_mesh* m, void* stream) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CGS_CUDA(cudaSetDevice(m->ctx->device));
    SolveScalars h{};
    CGS_CUDA(cudaMemcpyAsync(&h, m->step_S, sizeof(SolveScalars), cudaMemcpyDeviceToHost, st));
    CGS_CUDA(cudaStreamSynchronize(st));
    CGS_CUDA(cudaMemsetAsync(m->step_S, 0, sizeof(SolveScalars), st));
    CGS_CUDA(cudaStreamSynchronize(st));
    if (h.timeouts > 0 || h.status == CGS_ERR_TIMEOUT)
        return fail(CGS_ERR_TIMEOUT, "a bounded device wait of a single-step call expired (" +
                                         std::to_string(h.timeouts) + " waits)");
    return CGS_OK;
}

cgs_status cgs_mesh_set_wait_limits(cgs_mesh* m, int tile_wait, int barrier_wait) {
    if (!m || tile_wait < 0 || barrier_wait < 0) return fail(CGS_ERR_INVALID_ARG, "bad mesh or limit");
    CGS_CUDA(cudaSetDevice(m->ctx->device));
    CGS_CUDA(cudaDeviceSynchronize());
    m->E.P.wait_limit = tile_wait;
    m->E.P.bar_limit = barrier_wait;
    if (m->E.gexec) {   // the captured loop holds the old limits
        cudaGraphExecDestroy(m->E.gexec);
        m->E.gexec = nullptr;
    }
    return CGS_OK;
}

cgs_status cgs_apply_local(cgs_mesh* m, const double* r, double* l, int weighted, void* stream) {
    if (!m || !r || !l) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = m->E;
    const Vecs V = step_vecs(m, st);
    if (m->fp64()) {
        K(CGS_K_OTHER, launch_precond_prep<double>(E.P, V, r, st));
        K(CGS_K_LOCAL, launch_local(E.P, V, E.prec, V.s, V.z, weighted != 0, st));
        K(CGS_K_OTHER, launch_copy_d(E.P, static_cast<const double*>(V.z), l, true, st));
    } else {
        K(CGS_K_OTHER, launch_precond_prep<float>(E.P, V, r, st));
        K(CGS_K_LOCAL, launch_local(E.P, V, E.prec, V.s, V.z, weighted != 0, st));
        K(CGS_K_OTHER, launch_convert_f2d(E.P, static_cast<const float*>(V.z), l, true, st));
    }
    return finish(st, false);
}

cgs_status cgs_restrict(cgs_mesh* m, const double* s, double* rr, void* stream) {
    if (!m || !s || (!rr && m->d.nr)) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m->d.nr == 0) return CGS_OK;
    Engine& E = m->E;
    const Vecs V = step_vecs(m, st);
    K(CGS_K_OTHER, launch_fill_d(m->d.nr, rr, 0.0, st));
    K(CGS_K_RESTRICT, launch_restrict(E.P, V, m->fp64(), s, true, rr, false, st));
    return finish(st, false);
}

cgs_status cgs_coarse_solve(cgs_mesh* m, const double* rr, double* ur, void* stream) {
    if (!m || ((!rr || !ur) && m->d.nr)) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = m->E;
    const Vecs V = step_vecs(m, st);
    if (E.P.any_xxt) K(CGS_K_OTHER, launch_fill_d(m->d.nr, V.rt, 0.0, st));   // t = X^T r_r accumulates
    if (m->fp64()) {
        if (E.P.any_xxt) K(CGS_K_COARSE, launch_xxt_pass1(E.P, V, false, rr, st));
        K(CGS_K_COARSE, launch_coarse(E.P, V, rr, ur, nullptr, st));
    } else {
        // the mixed forms keep A_r^{-1} (or X) as float pairs: r_r -> pairs first
        float2* rr2 = reinterpret_cast<float2*>(V.rr);
        K(CGS_K_OTHER, launch_split_pair(m->d.nr, rr, rr2, st));
        if (E.P.any_xxt) K(CGS_K_COARSE, launch_xxt_pass1(E.P, V, true, V.rr, st));
        K(CGS_K_COARSE, launch_coarse_pair(E.P, V, rr2, ur, nullptr, st));
    }
    return finish(st, false);
}

cgs_status cgs_interp(cgs_mesh* m, const double* ur, double* z, void* stream) {
    if (!m || !z || (!ur && m->d.nr)) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = m->E;
    const Vecs V = step_vecs(m, st);
    if (m->fp64()) {
        K(CGS_K_OTHER, launch_fill_d(m->d.nv, static_cast<double*>(V.z), 0.0, st));
        K(CGS_K_INTERP, launch_interp_add(E.P, V, true, ur, nullptr, V.z, false, nullptr, st));
        K(CGS_K_OTHER, launch_copy_d(E.P, static_cast<const double*>(V.z), z, true, st));
    } else {
        K(CGS_K_OTHER, launch_fill_f(m->d.nv, static_cast<float*>(V.z), 0.0f, st));
        K(CGS_K_INTERP, launch_interp_add(E.P, V, false, ur, nullptr, V.z, false, nullptr, st));
        K(CGS_K_OTHER, launch_convert_f2d(E.P, static_cast<const float*>(V.z), z, true, st));
    }
    return finish(st, false);
}

cgs_status cgs_apply_preconditioner(cgs_mesh* m, const double* r, double* z, void* stream) {
    if (!m || !r || !z) return fail(CGS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = m->E;
    const Vecs V = step_vecs(m, st);
    if (m->fp64()) {
        K(CGS_K_OTHER, launch_precond_prep<double>(E.P, V, r, st));
        precond_body(E, V, st);
        K(CGS_K_OTHER, launch_copy_d(E.P, static_cast<const double*>(V.z), z, true, st));
    } else {
        K(CGS_K_OTHER, launch_precond_prep<float>(E.P, V, r, st));
        precond_body(E, V, st);
        K(CGS_K_OTHER, launch_convert_f2d(E.P, static_cast<const float*>(V.z), z, true, st));
    }
    return finish(st, false);
}

// ---- solves ------------------------------------------------------------------

cgs_status cgs_mesh_set_projection(cgs_mesh* m, int l) {
    if (!m || l < 0 || l > CGS_PROJECTION_MAX) return fail(CGS_ERR_INVALID_ARG, "bad mesh or projection size");
    CGS_CUDA(cudaSetDevice(m->ctx->device));
    CGS_CUDA(cudaDeviceSynchronize());
    m->proj.release();
    if (l == 0) return CGS_OK;
    auto& pj = m->proj;
    const size_t nv = (size_t)m->d.nv;
    cudaError_t e = cudaSuccess;
    auto get = [&](double** p, size_t n) {
        if (e == cudaSuccess) e = cudaMalloc(p, n * sizeof(double));
    };
    get(&pj.X, (size_t)l * nv);
    get(&pj.AX, (size_t)l * nv);
    get(&pj.ubar, nv);
    get(&pj.bp, nv);
    get(&pj.coef, (size_t)l + 1);
    get(&pj.partial, (size_t)proj_partial_entries(l));
    if (e == cudaSuccess) e = cudaMallocHost(&pj.host, sizeof(double) * (l + 1));
    if (e != cudaSuccess) {
        pj.release();
        return e == cudaErrorMemoryAllocation ? fail(CGS_ERR_OOM, "projection vectors") : cuda_fail(e, "projection");
    }
    pj.l = l;
    return CGS_OK;
}

cgs_status cgs_mesh_projection_size(const cgs_mesh* m, int* k) {
    if (!m || !k) return fail(CGS_ERR_INVALID_ARG, "null argument");
    *k = m->proj.k;
    return CGS_OK;
}

namespace {
// coef[0..k] of the last launch_proj_dots, read on the host (synchronises)
cgs_status read_coef(cgs_mesh* m, int k1, cudaStream_t st) {
    CGS_CUDA(cudaMemcpyAsync(m->proj.host, m->proj.coef, sizeof(double) * k1, cudaMemcpyDeviceToHost, st));
    CGS_CUDA(cudaStreamSynchronize(st));
    return CGS_OK;
}

// One solve with the projected start (Sec. 5), then the basis update.
cgs_status projected_solve(cgs_mesh* m, const double* b, double* x, double rtol, int maxit, int& iters,
                           double& relres, cudaStream_t st) {
    Engine& E = m->E;
    auto& pj = m->proj;
    const int64_t nv = m->d.nv;
    const uint8_t* dir = m->d.dir;
    // c_j = x~_j . b and ||b||^2 (free entries); u_bar = sum c_j x~_j;
    // b' = b - sum c_j A x~_j
    K(CGS_K_OTHER, launch_proj_dots(pj.X, pj.k, nv, b, dir, pj.partial, pj.coef, st));
    E.launches++;   // two kernels
    if (cgs_status s = read_coef(m, pj.k + 1, st)) return s;
    const double nb2 = pj.host[pj.k];
    K(CGS_K_OTHER, launch_proj_combine(nv, nullptr, dir, 1.0, pj.coef, pj.k, pj.X, pj.ubar, st));
    K(CGS_K_OTHER, launch_proj_combine(nv, b, dir, -1.0, pj.coef, pj.k, pj.AX, pj.bp, st));
    K(CGS_K_OTHER, launch_proj_dots(nullptr, 0, nv, pj.bp, dir, pj.partial, pj.coef, st));
    E.launches++;
    if (cgs_status s = read_coef(m, 1, st)) return s;
    const double nbp2 = pj.host[0];
    iters = 0;
    relres = 0.0;
    cgs_status slot = CGS_OK;
    if (nb2 > 0.0 && nbp2 > rtol * rtol * nb2) {
        // the correction solve, its stopping test relative to ||b||
        E.V.b = pj.bp;
        cgs_status s = engine_solve(E, rtol * std::sqrt(nb2 / nbp2), maxit, st);
        E.V.b = nullptr;
        if (s != CGS_OK) return s;
        const SolveScalars& h = E.S_host[0];
        iters = h.iters;
        relres = slot_relres(h) * std::sqrt(nbp2 / nb2);   // ||b - A x|| / ||b||
        slot = slot_status(h);
        K(CGS_K_OTHER, launch_vec_add(nv, pj.ubar, E.V.x, x, st));
    } else {
        // the start meets the tolerance: x = u_bar, relres from b'
        K(CGS_K_OTHER, launch_copy_d(E.P, pj.ubar, x, false, st));
        relres = nb2 > 0.0 ? std::sqrt(nbp2 / nb2) : 0.0;
    }
    // append x, A-orthonormalised against the basis (a full basis restarts):
    // e_j = (A x~_j) . x (A symmetric), w = x - sum e_j x~_j, A w by one
    // product (so the kept A x~ matches x~ even when w is small), then
    // w / ||w||_A unless x adds no direction (||w||_A^2 below 1e-12 of
    // x's, sum e_j^2 + ||w||_A^2: its orthogonal part is solver error)
    if (pj.k >= pj.l) pj.k = 0;
    double* w = pj.X + (size_t)pj.k * nv;
    double* Aw = pj.AX + (size_t)pj.k * nv;
    K(CGS_K_OTHER, launch_proj_dots(pj.AX, pj.k, nv, x, dir, pj.partial, pj.coef, st));
    E.launches++;
    if (cgs_status s = read_coef(m, pj.k + 1, st)) return s;
    double esum = 0.0;
    for (int j = 0; j < pj.k; ++j) esum += pj.host[j] * pj.host[j];
    K(CGS_K_OTHER, launch_proj_combine(nv, x, dir, -1.0, pj.coef, pj.k, pj.X, w, st));
    K(CGS_K_OTHER, launch_fill_d(nv, Aw, 0.0, st));
    K(CGS_K_OTHER, launch_apply64(E.P, no_stop(E.V), w, Aw, 1.0, false, st));
    K(CGS_K_OTHER, launch_proj_dots(w, 1, nv, Aw, dir, pj.partial, pj.coef, st));
    E.launches++;
    if (cgs_status s = read_coef(m, 1, st)) return s;
    const double nrm2 = pj.host[0];          // w^T A w
    if (nrm2 > 1e-12 * (esum + nrm2) && std::isfinite(nrm2)) {
        const double s = 1.0 / std::sqrt(nrm2);
        K(CGS_K_OTHER, launch_vec_scale(nv, w, s, st));
        K(CGS_K_OTHER, launch_vec_scale(nv, Aw, s, st));
        pj.k++;
    }
    return slot;
}
}  // namespace

cgs_status cgs_solve(cgs_mesh* m, const double* b, double* x, int nrhs, double rtol, int maxit, int* iters,
                     double* relres, void* stream) {
    if (!m || !b || !x || !iters || !relres || nrhs < 0 || !(rtol >= 0.0))
        return fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = m->E;
    cgs_status first_bad = CGS_OK;
    for (int k = 0; k < nrhs; ++k) {
        const double* bk = b + (size_t)k * m->d.nv;
        double* xk = x + (size_t)k * m->d.nv;
        iters[k] = 0;
        relres[k] = 0.0;
        if (m->proj.l > 0) {
            const cgs_status ss = projected_solve(m, bk, xk, rtol, maxit, iters[k], relres[k], st);
            if (ss == CGS_ERR_CUDA || ss == CGS_ERR_OOM) return ss;
            if (ss != CGS_OK && first_bad == CGS_OK) first_bad = ss;
            continue;
        }
        E.V.b = bk;
        cgs_status s = engine_solve(E, rtol, maxit, st);
        E.V.b = nullptr;
        if (s != CGS_OK) return s;
        K(CGS_K_OTHER, launch_copy_d(E.P, E.V.x, xk, false, st));
        const SolveScalars& h = E.S_host[0];
        iters[k] = h.iters;
        relres[k] = slot_relres(h);
        const cgs_status ss = slot_status(h);
        if (ss != CGS_OK && first_bad == CGS_OK) first_bad = ss;
    }
    cgs_status fs = finish(st, true);
    if (fs != CGS_OK) return fs;
    return first_bad;
}

cgs_status cgs_solve_host(cgs_mesh* m, const double* b_host, double* x_host, int nrhs, double rtol, int maxit,
                          int* iters, double* relres, void* stream) {
    if (!m || !b_host || !x_host || nrhs < 0) return fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)nrhs * m->d.nv;
    if (n > m->h_cap) {
        if (m->hb) {
            cudaFree(m->hb);
            cudaFree(m->hx);
            m->hb = m->hx = nullptr;
            m->h_cap = 0;
        }
        CGS_CUDA(cudaMalloc(&m->hb, n * sizeof(double)));
        CGS_CUDA(cudaMalloc(&m->hx, n * sizeof(double)));
        m->h_cap = n;
    }
    CGS_CUDA(cudaMemcpyAsync(m->hb, b_host, n * sizeof(double), cudaMemcpyHostToDevice, st));
    cgs_status s = cgs_solve(m, m->hb, m->hx, nrhs, rtol, maxit, iters, relres, stream);
    if (s == CGS_ERR_CUDA || s == CGS_ERR_OOM) return s;
    CGS_CUDA(cudaMemcpyAsync(x_host, m->hx, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CGS_CUDA(cudaStreamSynchronize(st));
    return s;
}

// ---- batches -------------------------------------------------------------------

cgs_status cgs_batch_create(cgs_ctx* ctx, cgs_mesh* const* meshes, int nmesh, int nrhs, cgs_batch** out) {
    if (!out) return fail(CGS_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (!ctx || !meshes || nmesh <= 0 || nrhs <= 0) return fail(CGS_ERR_INVALID_ARG, "bad argument");
    for (int i = 0; i < nmesh; ++i) {
        if (!meshes[i] || meshes[i]->ctx != ctx) return fail(CGS_ERR_INVALID_ARG, "mesh of another context");
        if (meshes[i]->prm.prec != meshes[0]->prm.prec || meshes[i]->E.form != meshes[0]->E.form)
            return fail(CGS_ERR_INVALID_ARG, "meshes of one batch share precision and form");
    }
    CGS_CUDA(cudaSetDevice(ctx->device));
    cgs_batch* B = new (std::nothrow) cgs_batch;
    if (!B) return fail(CGS_ERR_INVALID_ARG, "host allocation failed");
    B->ctx = ctx;
    B->meshes.assign(meshes, meshes + nmesh);
    B->nrhs = nrhs;
    auto cleanup = [&](cgs_status s) {
        B->E.release();
        B->mem.release();
        if (B->bptr_h) cudaFreeHost(B->bptr_h);
        if (B->xptr_h) cudaFreeHost(B->xptr_h);
        delete B;
        return s;
    };
    Engine& E = B->E;
    E.f64 = meshes[0]->fp64();
    E.prec = meshes[0]->prm.prec;
    E.form = meshes[0]->E.form;
    const int nslots = nmesh * nrhs;
    std::vector<DevMesh> descs(nmesh);
    std::vector<MeshSizes> sizes(nmesh);
    int64_t total_v = 0, total_r = 0, total_sub = 0, total_pack = 0;
    for (int i = 0; i < nmesh; ++i) {
        const cgs_mesh* m = meshes[i];
        descs[i] = m->d;
        sizes[i] = m->sizes;
        E.P.max_m = std::max(E.P.max_m, m->d.max_m);
        E.P.any_nr = E.P.any_nr || m->d.nr > 0;
        E.P.lane_big = E.P.lane_big || m->d.max_pack_m > 32;
        E.P.ell = (i == 0 || E.P.ell) && m->d.nslice > 0 && m->d.ell_val;
        E.P.ell_pair = (i == 0 || E.P.ell_pair) && m->d.nslice > 0 && m->d.ell_pair;
        B->max_nv = std::max(B->max_nv, m->d.nv);
        total_v += (int64_t)nrhs * m->d.nv;
        total_r += (int64_t)nrhs * m->d.nr;
        total_sub += (int64_t)nrhs * m->d.n_sub;
        total_pack += (int64_t)nrhs * m->d.n_pack;
    }
    // the slots of one mesh are interleaved item by item so that blocks
    // reading the same tile run together (the repeats hit L2)
    E.build = [sizes, nrhs](const Schedule& sch, std::vector<Work> (&tabs)[kWorkKinds]) {
        int64_t voff = 0, roff = 0, poff = 0;
        for (size_t i = 0; i < sizes.size(); ++i) {
            std::vector<Work> one[kWorkKinds];
            append_mesh_work(one, (int)i, 0, 0, 0, 0, sizes[i], sch);
            Schedule smallest;
            smallest.vert_chunk = 256;
            smallest.sub_chunk = 8;
            smallest.box_chunk = 256;
            const int64_t ps = mesh_partial_slots(sizes[i], smallest);
            for (int k = 0; k < kWorkKinds; ++k)
                for (const Work& w0 : one[k])
                    for (int r = 0; r < nrhs; ++r) {
                        Work w = w0;
                        w.slot = (int32_t)i * nrhs + r;
                        w.voff = voff + (int64_t)r * sizes[i].nv;
                        w.roff = (int32_t)(roff + (int64_t)r * sizes[i].nr);
                        w.poff = (int32_t)(poff + (int64_t)r * ps);
                        tabs[k].push_back(w);
                    }
            voff += (int64_t)nrhs * sizes[i].nv;
            roff += (int64_t)nrhs * sizes[i].nr;
            poff += (int64_t)nrhs * ps;
        }
    };
    int64_t total_p = 0;
    {
        Schedule smallest;
        smallest.vert_chunk = 256;
        smallest.sub_chunk = 8;
        smallest.box_chunk = 256;
        for (int i = 0; i < nmesh; ++i) total_p += (int64_t)nrhs * mesh_partial_slots(sizes[i], smallest);
    }
    if (total_p >= INT32_MAX || total_r >= INT32_MAX) return cleanup(fail(CGS_ERR_INVALID_ARG, "batch too large"));
    {
        const DevMesh* dm = nullptr;
        cudaError_t e = B->mem.upload(&dm, descs);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "mesh descriptors"));
        E.P.meshes = dm;
        E.P.nslots = nslots;
        if ((e = alloc_pools(B->mem, E, total_v, total_r, total_p, nslots)) != cudaSuccess)
            return cleanup(cuda_fail(e, "pools"));
        if ((e = set_schedule(E, default_schedule(total_v, total_sub, total_pack, total_pack * 32))) != cudaSuccess)
            return cleanup(cuda_fail(e, "work tables"));
        if ((e = B->mem.alloc(&B->bptr_d, nslots)) != cudaSuccess) return cleanup(cuda_fail(e, "pointers"));
        if ((e = B->mem.alloc(&B->xptr_d, nslots)) != cudaSuccess) return cleanup(cuda_fail(e, "pointers"));
        if ((e = cudaMallocHost(&B->bptr_h, sizeof(double*) * nslots)) != cudaSuccess)
            return cleanup(cuda_fail(e, "pinned pointers"));
        if ((e = cudaMallocHost(&B->xptr_h, sizeof(double*) * nslots)) != cudaSuccess)
            return cleanup(cuda_fail(e, "pinned pointers"));
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup(cuda_fail(e, "batch setup"));
    }
    E.V.bptr = B->bptr_d;
    E.V.xptr = B->xptr_d;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->in_use += B->mem.bytes;
        ctx->live_meshes++;
    }
    *out = B;
    return CGS_OK;
}

cgs_status cgs_batch_free(cgs_batch* B) {
    if (!B) return fail(CGS_ERR_INVALID_ARG, "null batch");
    cudaSetDevice(B->ctx->device);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> lk(B->ctx->mu);
        B->ctx->in_use -= B->mem.bytes;
        B->ctx->live_meshes--;
    }
    B->E.release();
    B->mem.release();
    if (B->bptr_h) cudaFreeHost(B->bptr_h);
    if (B->xptr_h) cudaFreeHost(B->xptr_h);
    delete B;
    return CGS_OK;
}

cgs_status cgs_batch_solve(cgs_batch* B, const double* const* b, double* const* x, double rtol, int maxit,
                           int* iters, double* relres, int* status, void* stream) {
    if (!B || !b || !x || !iters || !relres || !(rtol >= 0.0)) return fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = B->E;
    const int nslots = E.P.nslots;
    // the staging buffers are free: the previous call on this batch synchronised
    for (int s = 0; s < nslots; ++s) {
        if (!b[s] || !x[s]) return fail(CGS_ERR_INVALID_ARG, "null right-hand side or solution");
        B->bptr_h[s] = b[s];
        B->xptr_h[s] = x[s];
    }
    CGS_CUDA(cudaMemcpyAsync(B->bptr_d, B->bptr_h, sizeof(double*) * nslots, cudaMemcpyHostToDevice, st));
    CGS_CUDA(cudaMemcpyAsync(B->xptr_d, B->xptr_h, sizeof(double*) * nslots, cudaMemcpyHostToDevice, st));
    cgs_status s = engine_solve(E, rtol, maxit, st);
    if (s != CGS_OK) return s;
    cgs_status first_bad = CGS_OK;
    for (int k = 0; k < nslots; ++k) {
        const SolveScalars& h = E.S_host[k];
        iters[k] = h.iters;
        relres[k] = slot_relres(h);
        const cgs_status ss = slot_status(h);
        if (status) status[k] = ss;
        if (ss != CGS_OK && first_bad == CGS_OK) first_bad = ss;
    }
    return first_bad;
}

int64_t cgs_batch_launches(const cgs_batch* B) { return B ? B->E.launches : 0; }

cgs_status cgs_mesh_get_schedule(const cgs_mesh* m, cgs_schedule* out) {
    if (!m || !out) return fail(CGS_ERR_INVALID_ARG, "null argument");
    const Schedule& s = m->E.sch;
    *out = cgs_schedule{s.vert_chunk, s.sub_chunk, s.pack_chunk, s.box_chunk, s.tile_tma, s.persistent,
                        m->E.P.pdl ? 1 : 0, s.row_packs, s.interp_cells};
    return CGS_OK;
}

cgs_status cgs_mesh_set_schedule(cgs_mesh* m, const cgs_schedule* c) {
    if (!m || !c) return fail(CGS_ERR_INVALID_ARG, "null argument");
    auto in = [](int v, int lo, int hi, int step) { return v >= lo && v <= hi && v % step == 0; };
    if (!in(c->vert_chunk, 256, 8192, 256) || !in(c->sub_chunk, 8, 512, 8) || !in(c->pack_chunk, 8, 256, 8) ||
        !in(c->box_chunk, 256, 4096, 256) || (c->tile_tma != 0 && c->tile_tma != 1) || c->persistent < -1 ||
        c->persistent > 1 || (c->pdl != 0 && c->pdl != 1) || (c->row_packs != 0 && c->row_packs != 1) ||
        (c->interp_cells != 0 && c->interp_cells != 1))
        return fail(CGS_ERR_INVALID_ARG, "schedule out of range");
    CGS_CUDA(cudaSetDevice(m->ctx->device));
    Schedule sch = m->E.sch;
    sch.vert_chunk = c->vert_chunk;
    sch.sub_chunk = c->sub_chunk;
    sch.pack_chunk = c->pack_chunk;
    sch.box_chunk = c->box_chunk;
    sch.tile_tma = c->tile_tma;
    sch.persistent = c->persistent;
    sch.pdl = c->pdl;
    sch.row_packs = c->row_packs;
    sch.interp_cells = c->interp_cells;
    CGS_CUDA(set_schedule(m->E, sch));
    return CGS_OK;
}

cgs_status cgs_mesh_tune(cgs_mesh* m, void* stream) {
    if (!m) return fail(CGS_ERR_INVALID_ARG, "null mesh");
    return tune_engine(m->E, static_cast<cudaStream_t>(stream));
}

cgs_status cgs_batch_tune(cgs_batch* B, void* stream) {
    if (!B) return fail(CGS_ERR_INVALID_ARG, "null batch");
    return tune_engine(B->E, static_cast<cudaStream_t>(stream));
}

cgs_status cgs_solve_batched(cgs_mesh* const* meshes, int nmesh, const double* const* b, double* const* x,
                             int nrhs, double rtol, int maxit, int* iters, double* relres, void* stream) {
    if (!meshes || nmesh <= 0 || !meshes[0]) return fail(CGS_ERR_INVALID_ARG, "bad argument");
    cgs_batch* B = nullptr;
    cgs_status s = cgs_batch_create(meshes[0]->ctx, meshes, nmesh, nrhs, &B);
    if (s != CGS_OK) return s;
    s = cgs_batch_solve(B, b, x, rtol, maxit, iters, relres, nullptr, stream);
    const std::string keep = g_err;
    cgs_batch_free(B);
    g_err = keep;
    return s;
}

}  // extern "C"

// ---- serving: continuous batching over a pool of solve slots -------------------

namespace {

// First-fit allocator over [0, cap) in units of `align` entries, with
// coalescing of neighbouring free ranges.  Host-side bookkeeping only; the
// entries themselves are one device allocation per vector.
class Arena {
public:
    void init(int64_t cap, int64_t align) {
        align_ = align;
        cap_ = cap / align * align;
        free_.clear();
        if (cap_ > 0) free_[0] = cap_;
        used_ = 0;
    }
    int64_t round(int64_t n) const { return (std::max<int64_t>(n, 1) + align_ - 1) / align_ * align_; }
    int64_t capacity() const { return cap_; }
    int64_t used() const { return used_; }
    // offset of n entries, or -1 when no free range is large enough
    int64_t alloc(int64_t n) {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const int64_t off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest > 0) free_[off + n] = rest;
            used_ += n;
            return off;
        }
        return -1;
    }
    void release(int64_t off, int64_t n) {
        n = round(n);
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }

private:
    std::map<int64_t, int64_t> free_;
    int64_t cap_ = 0, align_ = 1, used_ = 0;
};

}  // namespace

struct cgs_server {
    cgs_ctx* ctx = nullptr;
    int max_slots = 0;
    double rtol = 1e-8;
    int maxit = 1000;
    DevAllocs mem;
    Engine E;
    Schedule sch;
    // arenas of vertex entries, reduced entries and partial-sum entries
    Arena av, ar, ap;
    size_t bytes_per_v = 0, bytes_per_r = 0, bytes_per_p = sizeof(double);
    // registry of mesh descriptors on the device (index -> mesh)
    DevMesh* reg_d = nullptr;
    DevMesh* reg_stage = nullptr;   // pinned staging for descriptor uploads
    int reg_cap = 0;
    std::vector<cgs_mesh*> reg;
    std::vector<int> reg_users;
    struct Req {
        uint64_t ticket;
        cgs_mesh* mesh;
        const double* b;
        double* x;
    };
    std::deque<Req> queue;
    struct SlotState {
        bool busy = false;
        Req req{};
        int reg = -1;
        int64_t voff = 0, roff = 0, poff = 0, np = 0;
    };
    std::vector<SlotState> slots;
    struct Res {
        int done, iters, status;
        double relres;
    };
    std::unordered_map<uint64_t, Res> results;
    std::deque<uint64_t> completed;   // finished tickets not yet drained
    uint64_t next_ticket = 1;
    // work tables of the current slots, of the slots admitted this step and
    // of the slots finished this step (capacity-grown device buffers)
    struct Table {
        Work* d[kWorkKinds] = {};
        size_t cap[kWorkKinds] = {};
        Work* h[kWorkKinds] = {};     // pinned staging
        size_t hcap[kWorkKinds] = {};
    } t_main, t_admit, t_fin;
    Plan P_main, P_admit, P_fin;
    bool dirty = true;
    const double** bptr_h = nullptr;
    double** xptr_h = nullptr;
    const double** bptr_d = nullptr;
    double** xptr_d = nullptr;
};

namespace {

void free_table(cgs_server::Table& t) {
    for (int k = 0; k < kWorkKinds; ++k) {
        if (t.d[k]) cudaFree(t.d[k]);
        if (t.h[k]) cudaFreeHost(t.h[k]);
        t.d[k] = nullptr;
        t.h[k] = nullptr;
        t.cap[k] = t.hcap[k] = 0;
    }
}

// Work tables for the listed slots, uploaded into a capacity-grown table.
cudaError_t server_tables(cgs_server* sv, const std::vector<int>& ids, cgs_server::Table& t, Plan& P,
                          cudaStream_t st) {
    std::vector<Work> tabs[kWorkKinds];
    P = Plan();
    P.meshes = sv->reg_d;
    P.nslots = sv->max_slots;
    P.wait_limit = sv->E.P.wait_limit;
    P.bar_limit = sv->E.P.bar_limit;
    P.tile_tma = sv->sch.tile_tma != 0;
    P.pack_chunk = sv->sch.pack_chunk;
    P.pdl = sv->sch.pdl != 0;
    P.interp_cells = sv->sch.interp_cells != 0;
    P.ell = !ids.empty();
    P.ell_pair = !ids.empty();
    for (int k : ids) {
        const cgs_server::SlotState& ss = sv->slots[k];
        const cgs_mesh* m = ss.req.mesh;
        append_mesh_work(tabs, ss.reg, k, ss.voff, ss.roff, ss.poff, m->sizes, sv->sch);
        P.max_m = std::max(P.max_m, m->d.max_m);
        P.any_nr = P.any_nr || m->d.nr > 0;
        P.lane_big = P.lane_big || m->d.max_pack_m > 32;
        P.ell = P.ell && m->d.nslice > 0 && m->d.ell_val;
        P.ell_pair = P.ell_pair && m->d.nslice > 0 && m->d.ell_pair;
    }
    for (int kind = 0; kind < kWorkKinds; ++kind) {
        const size_t n = tabs[kind].size();
        if (n > t.cap[kind]) {
            if (t.d[kind]) cudaFree(t.d[kind]);
            if (t.h[kind]) cudaFreeHost(t.h[kind]);
            const size_t c = std::max<size_t>(n, 2 * t.cap[kind]);
            cudaError_t e = cudaMalloc(&t.d[kind], c * sizeof(Work));
            if (e != cudaSuccess) return e;
            if ((e = cudaMallocHost(&t.h[kind], c * sizeof(Work))) != cudaSuccess) return e;
            t.cap[kind] = t.hcap[kind] = c;
        }
        if (n) {
            std::memcpy(t.h[kind], tabs[kind].data(), n * sizeof(Work));
            cudaError_t e = cudaMemcpyAsync(t.d[kind], t.h[kind], n * sizeof(Work), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
        }
        P.work[kind] = t.d[kind];
        P.nwork[kind] = (unsigned int)n;
    }
    P.any_xxt = P.nwork[kWorkXSeg] > 0;
    P.hyb_restrict = hyb_restrict_ok(P, tabs);
    return cudaSuccess;
}

int server_register(cgs_server* sv, cgs_mesh* m, cudaStream_t st) {
    for (int i = 0; i < sv->reg_cap; ++i)
        if (sv->reg[i] == m) {
            sv->reg_users[i]++;
            return i;
        }
    for (int i = 0; i < sv->reg_cap; ++i)
        if (!sv->reg[i] || sv->reg_users[i] == 0) {
            sv->reg[i] = m;
            sv->reg_users[i] = 1;
            sv->reg_stage[i] = m->d;
            cudaMemcpyAsync(sv->reg_d + i, sv->reg_stage + i, sizeof(DevMesh), cudaMemcpyHostToDevice, st);
            return i;
        }
    return -1;
}

}  // namespace

extern "C" {

cgs_status cgs_server_create(cgs_ctx* ctx, int max_slots, int64_t pool_nv, int64_t pool_nr, cgs_precision prec,
                             cgs_form form, double rtol, int maxit, cgs_server** out) {
    if (!out) return fail(CGS_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (!ctx || max_slots <= 0 || pool_nv <= 0 || pool_nr < 0 || !(rtol >= 0.0) || pool_nv > (int64_t(1) << 40) ||
        pool_nr > (int64_t(1) << 30))
        return fail(CGS_ERR_INVALID_ARG, "bad argument");
    CGS_CUDA(cudaSetDevice(ctx->device));
    cgs_server* sv = new (std::nothrow) cgs_server;
    if (!sv) return fail(CGS_ERR_INVALID_ARG, "host allocation failed");
    sv->ctx = ctx;
    sv->max_slots = max_slots;
    // vertex entries in 32-entry units (256-byte aligned double vectors)
    sv->av.init((pool_nv + 31) / 32 * 32, 32);
    sv->ar.init((pool_nr + 7) / 8 * 8 + 8 * max_slots, 8);
    sv->ap.init(2 * ((pool_nv + 127) / 128) + 64 * (int64_t)max_slots, 8);
    sv->bytes_per_v = 4 * sizeof(double) + (prec == CGS_FP64 ? 3 * sizeof(double) : sizeof(float2) + 2 * sizeof(float));
    sv->bytes_per_r = 3 * sizeof(double) + (prec == CGS_FP64 ? 0 : sizeof(float));
    sv->rtol = rtol;
    sv->maxit = maxit;
    sv->slots.resize(max_slots);
    sv->reg_cap = 4 * max_slots + 16;
    sv->reg.assign(sv->reg_cap, nullptr);
    sv->reg_users.assign(sv->reg_cap, 0);
    Engine& E = sv->E;
    E.f64 = prec == CGS_FP64;
    E.prec = prec;
    E.form = form;
    auto cleanup = [&](cgs_status s) {
        E.release();
        sv->mem.release();
        if (sv->reg_stage) cudaFreeHost(sv->reg_stage);
        if (sv->bptr_h) cudaFreeHost(sv->bptr_h);
        if (sv->xptr_h) cudaFreeHost(sv->xptr_h);
        delete sv;
        return s;
    };
    cudaError_t e;
    if ((e = sv->mem.alloc(&sv->reg_d, sv->reg_cap)) != cudaSuccess) return cleanup(cuda_fail(e, "registry"));
    if ((e = cudaMallocHost(&sv->reg_stage, sizeof(DevMesh) * sv->reg_cap)) != cudaSuccess)
        return cleanup(cuda_fail(e, "registry staging"));
    if ((e = alloc_pools(sv->mem, E, sv->av.capacity(), sv->ar.capacity(), sv->ap.capacity(), max_slots)) !=
        cudaSuccess)
        return cleanup(cuda_fail(e, "vector arena"));
    if ((e = sv->mem.alloc(&sv->bptr_d, max_slots)) != cudaSuccess) return cleanup(cuda_fail(e, "pointers"));
    if ((e = sv->mem.alloc(&sv->xptr_d, max_slots)) != cudaSuccess) return cleanup(cuda_fail(e, "pointers"));
    if ((e = cudaMallocHost(&sv->bptr_h, sizeof(double*) * max_slots)) != cudaSuccess)
        return cleanup(cuda_fail(e, "pointers"));
    if ((e = cudaMallocHost(&sv->xptr_h, sizeof(double*) * max_slots)) != cudaSuccess)
        return cleanup(cuda_fail(e, "pointers"));
    for (int k = 0; k < max_slots; ++k) {
        sv->bptr_h[k] = nullptr;
        sv->xptr_h[k] = nullptr;
    }
    // chunks sized for the whole arena as one problem: many slots at once
    sv->sch = default_schedule(pool_nv, pool_nv / 8, pool_nv / 256, pool_nv / 8);
    E.V.bptr = sv->bptr_d;
    E.V.xptr = sv->xptr_d;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->budget && ctx->in_use + sv->mem.bytes > ctx->budget)
            return cleanup(fail(CGS_ERR_ADMISSION, "vector arena exceeds the context's HBM budget"));
        ctx->in_use += sv->mem.bytes;
        ctx->live_meshes++;
    }
    *out = sv;
    return CGS_OK;
}

cgs_status cgs_server_free(cgs_server* sv) {
    if (!sv) return fail(CGS_ERR_INVALID_ARG, "null server");
    cudaSetDevice(sv->ctx->device);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> lk(sv->ctx->mu);
        sv->ctx->in_use -= sv->mem.bytes;
        sv->ctx->live_meshes--;
    }
    free_table(sv->t_main);
    free_table(sv->t_admit);
    free_table(sv->t_fin);
    sv->E.release();
    sv->mem.release();
    if (sv->reg_stage) cudaFreeHost(sv->reg_stage);
    if (sv->bptr_h) cudaFreeHost(sv->bptr_h);
    if (sv->xptr_h) cudaFreeHost(sv->xptr_h);
    delete sv;
    return CGS_OK;
}

cgs_status cgs_submit(cgs_server* sv, cgs_mesh* mesh, const double* b, double* x, uint64_t* ticket) {
    if (!sv || !mesh || !b || !x || !ticket) return fail(CGS_ERR_INVALID_ARG, "null argument");
    if (mesh->ctx != sv->ctx) return fail(CGS_ERR_INVALID_ARG, "mesh of another context");
    if (mesh->prm.prec != sv->E.prec || mesh->E.form != sv->E.form)
        return fail(CGS_ERR_INVALID_ARG, "mesh precision or form differs from the server's");
    if (sv->av.round(mesh->d.nv) > sv->av.capacity() || sv->ar.round(mesh->d.nr) > sv->ar.capacity() ||
        sv->ap.round(mesh_partial_slots(mesh->sizes, sv->sch)) > sv->ap.capacity())
        return fail(CGS_ERR_ADMISSION, "request larger than the server's vector arena");
    *ticket = sv->next_ticket++;
    sv->queue.push_back(cgs_server::Req{*ticket, mesh, b, x});
    sv->results[*ticket] = cgs_server::Res{0, 0, CGS_OK, 0.0};
    return CGS_OK;
}

cgs_status cgs_server_step(cgs_server* sv, int iterations, void* stream, int* active, int* queued,
                           int* finished) {
    if (!sv || iterations < 0) return fail(CGS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Engine& E = sv->E;
    // 1. admit queued requests, in arrival order, while a slot is free and
    //    the arena holds the request's vectors
    std::vector<int> fresh;
    int k = 0;
    while (!sv->queue.empty()) {
        while (k < sv->max_slots && sv->slots[k].busy) ++k;
        if (k == sv->max_slots) break;
        const cgs_server::Req& rq = sv->queue.front();
        const int64_t np = mesh_partial_slots(rq.mesh->sizes, sv->sch);
        const int64_t vo = sv->av.alloc(rq.mesh->d.nv);
        if (vo < 0) break;
        const int64_t ro = sv->ar.alloc(rq.mesh->d.nr);
        if (ro < 0) {
            sv->av.release(vo, rq.mesh->d.nv);
            break;
        }
        const int64_t po = sv->ap.alloc(np);
        if (po < 0) {
            sv->av.release(vo, rq.mesh->d.nv);
            sv->ar.release(ro, rq.mesh->d.nr);
            break;
        }
        const int ri = server_register(sv, rq.mesh, st);
        if (ri < 0) {
            sv->av.release(vo, rq.mesh->d.nv);
            sv->ar.release(ro, rq.mesh->d.nr);
            sv->ap.release(po, np);
            break;
        }
        cgs_server::SlotState& ss = sv->slots[k];
        ss.busy = true;
        ss.req = rq;
        ss.reg = ri;
        ss.voff = vo;
        ss.roff = ro;
        ss.poff = po;
        ss.np = np;
        sv->queue.pop_front();
        sv->bptr_h[k] = ss.req.b;
        sv->xptr_h[k] = ss.req.x;
        fresh.push_back(k);
    }
    std::vector<int> busy;
    for (int k = 0; k < sv->max_slots; ++k)
        if (sv->slots[k].busy) busy.push_back(k);
    if (!fresh.empty()) {
        CGS_CUDA(cudaMemcpyAsync(sv->bptr_d, sv->bptr_h, sizeof(double*) * sv->max_slots, cudaMemcpyHostToDevice, st));
        CGS_CUDA(cudaMemcpyAsync(sv->xptr_d, sv->xptr_h, sizeof(double*) * sv->max_slots, cudaMemcpyHostToDevice, st));
        CGS_CUDA(server_tables(sv, fresh, sv->t_admit, sv->P_admit, st));
        sv->dirty = true;
    }
    if (sv->dirty) {
        CGS_CUDA(server_tables(sv, busy, sv->t_main, sv->P_main, st));
        sv->dirty = false;
    }
    // 2. start the new slots: r = b, z = M r, p = z
    if (!fresh.empty()) {
        E.P = sv->P_admit;
        pcg_start(E, E.P, sv->rtol, sv->maxit, st);
    }
    // 3. iterate every running slot (slots that stop skip their blocks)
    if (!busy.empty()) {
        E.P = sv->P_main;
        if (use_persistent(E, sv->sch))
            CGS_CUDA(persistent_launch(E, iterations, st));
        else
            for (int i = 0; i < iterations; ++i) pcg_iteration(E, st);
    }
    CGS_CUDA(cudaMemcpyAsync(E.S_host, E.V.S, sizeof(SolveScalars) * sv->max_slots, cudaMemcpyDeviceToHost, st));
    CGS_CUDA(cudaStreamSynchronize(st));
    // 4. retire finished slots: true residual, solution out
    std::vector<int> done;
    for (int k : busy)
        if (E.S_host[k].done) done.push_back(k);
    if (!done.empty()) {
        CGS_CUDA(server_tables(sv, done, sv->t_fin, sv->P_fin, st));
        E.P = sv->P_fin;
        const Vecs Vn = no_stop(E.V);
        if (!E.f64) K(CGS_K_OTHER, launch_finalize_x_pair(E.P, E.V, st));
        for (int k : done)
            CGS_CUDA(cudaMemsetAsync(E.V.y + sv->slots[k].voff, 0, sizeof(double) * sv->slots[k].req.mesh->d.nv, st));
        K(CGS_K_OTHER, launch_apply64(E.P, Vn, E.V.x, E.V.y, 1.0, false, st));
        K(CGS_K_OTHER, launch_resid_norm(E.P, E.V, st));
        CGS_CUDA(cudaMemcpyAsync(E.S_host, E.V.S, sizeof(SolveScalars) * sv->max_slots, cudaMemcpyDeviceToHost, st));
        CGS_CUDA(cudaStreamSynchronize(st));
        for (int k : done) {
            cgs_server::SlotState& ss = sv->slots[k];
            const SolveScalars& h = E.S_host[k];
            sv->results[ss.req.ticket] = cgs_server::Res{1, h.iters, (int)slot_status(h), slot_relres(h)};
            sv->completed.push_back(ss.req.ticket);
            sv->reg_users[ss.reg]--;
            sv->av.release(ss.voff, ss.req.mesh->d.nv);
            sv->ar.release(ss.roff, ss.req.mesh->d.nr);
            sv->ap.release(ss.poff, ss.np);
            ss.busy = false;
            ss.reg = -1;
        }
        sv->dirty = true;
    }
    cgs_status fs = finish(st, false);
    if (fs != CGS_OK) return fs;
    if (active) *active = (int)(busy.size() - done.size());
    if (queued) *queued = (int)sv->queue.size();
    if (finished) *finished = (int)done.size();
    return CGS_OK;
}

cgs_status cgs_poll(cgs_server* sv, uint64_t ticket, int* done, int* iters, double* relres, int* status) {
    if (!sv || !done) return fail(CGS_ERR_INVALID_ARG, "null argument");
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return fail(CGS_ERR_INVALID_ARG, "unknown ticket");
    const cgs_server::Res& r = it->second;
    *done = r.done;
    if (iters) *iters = r.iters;
    if (relres) *relres = r.relres;
    if (status) *status = r.status;
    if (r.done) sv->results.erase(it);
    return CGS_OK;
}

int cgs_server_drain(cgs_server* sv, uint64_t* tickets, int* iters, double* relres, int* status, int cap) {
    if (!sv || cap < 0 || (cap > 0 && !tickets)) {
        fail(CGS_ERR_INVALID_ARG, "bad argument");
        return -1;
    }
    int n = 0;
    while (n < cap && !sv->completed.empty()) {
        const uint64_t t = sv->completed.front();
        sv->completed.pop_front();
        auto it = sv->results.find(t);
        if (it == sv->results.end()) continue;   // already taken by cgs_poll
        tickets[n] = t;
        if (iters) iters[n] = it->second.iters;
        if (relres) relres[n] = it->second.relres;
        if (status) status[n] = it->second.status;
        sv->results.erase(it);
        ++n;
    }
    return n;
}

cgs_status cgs_server_footprint(const cgs_server* sv, const cgs_mesh* mesh, size_t* bytes) {
    if (!sv || !mesh || !bytes) return fail(CGS_ERR_INVALID_ARG, "null argument");
    *bytes = (size_t)sv->av.round(mesh->d.nv) * sv->bytes_per_v + (size_t)sv->ar.round(mesh->d.nr) * sv->bytes_per_r +
             (size_t)sv->ap.round(mesh_partial_slots(mesh->sizes, sv->sch)) * sv->bytes_per_p;
    return CGS_OK;
}

cgs_status cgs_server_stats(const cgs_server* sv, size_t* arena_bytes, size_t* bytes_in_use, int* active,
                            int* queued) {
    if (!sv) return fail(CGS_ERR_INVALID_ARG, "null server");
    if (arena_bytes)
        *arena_bytes = (size_t)sv->av.capacity() * sv->bytes_per_v + (size_t)sv->ar.capacity() * sv->bytes_per_r +
                       (size_t)sv->ap.capacity() * sv->bytes_per_p;
    if (bytes_in_use)
        *bytes_in_use = (size_t)sv->av.used() * sv->bytes_per_v + (size_t)sv->ar.used() * sv->bytes_per_r +
                        (size_t)sv->ap.used() * sv->bytes_per_p;
    if (active) {
        int n = 0;
        for (const auto& ss : sv->slots) n += ss.busy ? 1 : 0;
        *active = n;
    }
    if (queued) *queued = (int)sv->queue.size();
    return CGS_OK;
}

int64_t cgs_server_launches(const cgs_server* sv) { return sv ? sv->E.launches : 0; }

}  // extern "C"
