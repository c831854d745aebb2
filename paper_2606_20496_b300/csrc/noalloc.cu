// cgs_apply_preconditioner_noalloc: z = M r with every working vector in a
// static device array, so the call never allocates device memory.
//
// Who needs it: callers that cannot allocate at call time, such as work being
// captured into a CUDA graph, serving loops that forbid allocation after
// warm-up, or hosts whose device memory belongs to another runtime's pool.
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
    void* zb = p;                                        // nv entries of 8 bytes
    void* sb = p + (size_t)8 * CGS_NOALLOC_MAX_NV;       // nv entries of 8 bytes
    double* rr = reinterpret_cast<double*>(p + (size_t)16 * CGS_NOALLOC_MAX_NV);
    double* ur = rr + CGS_NOALLOC_MAX_NR;
    const bool f64 = mesh_prec(mesh) == CGS_FP64;
    const int64_t nv = d.nv;
    // z = 0, s = r in the bulk precision, r_r = 0
    if (f64) {
        launch_fill_d(nv, static_cast<double*>(zb), 0.0, st);
        launch_copy_d(nv, r, static_cast<double*>(sb), nullptr, st);
    } else {
        launch_fill_f(nv, static_cast<float*>(zb), 0.0f, st);
        launch_convert_d2f(nv, r, static_cast<float*>(sb), nullptr, st);
    }
    if (d.nr) launch_fill_d(d.nr, rr, 0.0, st);
    if (mesh_form(mesh) == CGS_HYBRID) {
        launch_local(d, mesh_prec(mesh), sb, zb, true, nullptr, st);
        if (f64)
            launch_apply64(d, static_cast<const double*>(zb), static_cast<double*>(sb), -1.0, nullptr, nullptr,
                           false, st);
        else
            launch_apply28f_tiled(d, static_cast<const float*>(zb), static_cast<float*>(sb), -1.0f, nullptr, st);
        if (d.nr) {
            launch_restrict(d, f64, sb, f64, rr, nullptr, st);
            launch_coarse(d, rr, ur, nullptr, nullptr, st);
            launch_interp_add(d, f64, ur, nullptr, zb, nullptr, st);
        }
    } else {
        launch_local(d, mesh_prec(mesh), sb, zb, false, nullptr, st);
        if (d.nr) {
            launch_restrict(d, f64, sb, f64, rr, nullptr, st);
            launch_coarse(d, rr, ur, nullptr, nullptr, st);
            launch_interp_add(d, f64, ur, nullptr, zb, nullptr, st);
        }
    }
    if (f64)
        launch_copy_d(nv, static_cast<const double*>(zb), z, mesh_dir(mesh), st);
    else
        launch_convert_f2d(nv, static_cast<const float*>(zb), z, mesh_dir(mesh), st);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("kernel launch: ") + cudaGetErrorString(e));
        return CGS_ERR_CUDA;
    }
    return CGS_OK;
}
