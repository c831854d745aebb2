// cgs_apply_preconditioner_noalloc: z = M r with every working vector in a
// static device array, so the call never allocates device memory.
//
// Who needs it: callers that cannot allocate at call time, such as serving
// loops that forbid allocation after warm-up, or hosts whose device memory
// belongs to another runtime's pool (an allocation of ours would bypass that
// pool's accounting or fail).
//
// The array below is a host-side stand-in when named in host code: only its
// device address, looked up once per device by cudaGetSymbolAddress with that
// device current, may be handed to kernels.  The first call on each device
// does that lookup (make it before any stream capture).  Every call shares
// the array, which keeps the last call's contents; this call clears what must
// start at zero.  Calls that overlap on the GPU race on the array.
#include <mutex>
#include <string>

#include "internal.h"
#include "kernels.h"

namespace {

static __device__ __align__(256) unsigned char g_precond_scratch[CGS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of g_precond_scratch on `device` (looked up on first use).
cudaError_t scratch_on(int device, void** out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[device]) {
        int cur = 0;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_precond_scratch);
        if (cur != device) cudaSetDevice(cur);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = ptr;
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace

using namespace cgs;

extern "C" cgs_status cgs_apply_preconditioner_noalloc(cgs_mesh* mesh, const double* r, double* z, void* stream) {
    if (!mesh || !r || !z) {
        set_last_error("null argument");
        return CGS_ERR_INVALID_ARG;
    }
    const DevMesh& d = mesh_dev(mesh);
    if (d.nv > CGS_NOALLOC_MAX_NV || d.nr > CGS_NOALLOC_MAX_NR) {
        set_last_error("mesh too large for cgs_apply_preconditioner_noalloc: nv " + std::to_string(d.nv) +
                       " (limit " + std::to_string(CGS_NOALLOC_MAX_NV) + "), n_r " + std::to_string(d.nr) +
                       " (limit " + std::to_string(CGS_NOALLOC_MAX_NR) + ")");
        return CGS_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    cudaError_t e = scratch_on(mesh_device(mesh), &base);
    if (e != cudaSuccess) {
        set_last_error(std::string("no-allocation scratch lookup: ") + cudaGetErrorString(e));
        return CGS_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* p = static_cast<unsigned char*>(base);
    // the mesh's own work tables (one slot at offset 0) with every working
    // vector in the static array
    const Plan& P = mesh_plan(mesh);
    Vecs V;
    // an expired element-tile wait is recorded in the mesh's step status
    // word (set up with the mesh, so nothing is allocated here)
    V.S = mesh_step_status_word(mesh, st);
    V.step = 1;
    V.z = p;                                           // nv entries of 8 bytes
    V.s = p + (size_t)8 * CGS_NOALLOC_MAX_NV;          // nv entries of 8 bytes
    V.rr = reinterpret_cast<double*>(p + (size_t)16 * CGS_NOALLOC_MAX_NV);
    V.ur = V.rr + CGS_NOALLOC_MAX_NR;
    V.rt = V.ur + CGS_NOALLOC_MAX_NR;                  // zeroed with r_r by the prep kernel
    const cgs_precision prec = mesh_prec(mesh);
    const bool f64 = prec == CGS_FP64;
    // z = 0, s = r in the bulk precision, r_r = 0
    if (f64)
        launch_precond_prep<double>(P, V, r, st);
    else
        launch_precond_prep<float>(P, V, r, st);
    const cgs_form form = mesh_form(mesh);
    const bool weighted = form == CGS_HYBRID;
    // additive mixed form: the local solves and the restriction of s share
    // one launch when every subdomain is in packs (as in the regular call)
    const bool restricted = form == CGS_ADDITIVE && !f64 && d.nr &&
                            launch_local_restrict(P, V, prec, static_cast<const float*>(V.s),
                                                  static_cast<float*>(V.z), V.rr, st);
    if (!restricted) launch_local(P, V, prec, V.s, V.z, weighted ? 1 : form == CGS_RAS ? 2 : 0, st);
    // hybrid: r_r = J~^T r - (A J~)^T l straight from r and l (as the regular
    // call does when the mesh has the entries), else s = r - A l first
    const bool hyb_direct = weighted && d.nr && P.hyb_restrict;
    if (hyb_direct) launch_restrict_hybrid(P, V, f64, V.s, V.z, V.rr, st);
    if (weighted && !hyb_direct) {
        if (f64)
            launch_apply64(P, V, static_cast<const double*>(V.z), static_cast<double*>(V.s), -1.0, false, st);
        else
            launch_apply28f_tiled(P, V, static_cast<const float*>(V.z), static_cast<float*>(V.s), -1.0f, st);
    }
    if (d.nr && f64) {
        if (!hyb_direct) launch_restrict(P, V, true, V.s, true, V.rr, false, st);
        launch_xxt_pass1(P, V, false, V.rr, st);   // XX^T meshes only
        launch_coarse(P, V, V.rr, V.ur, nullptr, st);
        launch_interp_add(P, V, true, V.ur, nullptr, V.z, false, nullptr, st);
    } else if (d.nr) {
        // r_r as float pairs, the pair product writes u_r rounded to float
        float* ur32 = reinterpret_cast<float*>(V.ur);
        if (!restricted && !hyb_direct) launch_restrict(P, V, false, V.s, false, V.rr, true, st);
        launch_xxt_pass1(P, V, true, V.rr, st);    // XX^T meshes only
        launch_coarse_pair(P, V, reinterpret_cast<const float2*>(V.rr), nullptr, ur32, st);
        launch_interp_add(P, V, false, nullptr, ur32, V.z, false, nullptr, st);
    }
    if (f64)
        launch_copy_d(P, static_cast<const double*>(V.z), z, true, st);
    else
        launch_convert_f2d(P, static_cast<const float*>(V.z), z, true, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("kernel launch: ") + cudaGetErrorString(e));
        return CGS_ERR_CUDA;
    }
    return CGS_OK;
}
