// noalloc.cu -- a time step that allocates no device memory (lbm_step_noalloc in include/lbm.h).
//
// Who needs it: callers that must not call cudaMalloc at the time they step the solver, e.g. code
// that records its work into a CUDA graph (allocation during stream capture is not allowed), an
// application whose device memory is owned by another allocator (a framework's caching pool) and
// is already fully reserved, or a loop with a fixed memory budget where an allocation that can fail
// or stall is not acceptable.  lbm_step itself may allocate (it grows the force history), so these
// callers step the lattice through this entry point instead: the populations and the force live in
// buffers the caller owns, and the only other memory the step kernel needs -- its per-tile force
// partials and the ticket of its last-tile reduction -- lives in one file-scope device array below,
// loaded with the library and held by every GPU that uses it until the process exits.
//
// The kernel is the library's step kernel itself; only the scratch pointers differ.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"
#include "runtime.h"
#include "step_kernel.cuh"

namespace {

// Scratch: LBM_NOALLOC_MAX_SLOTS per-tile force partials (16 B each), then the ticket counter and
// the non-finite flag.  Shared by every call in the process on a given device.
constexpr size_t kPartialBytes = (size_t)LBM_NOALLOC_MAX_SLOTS * sizeof(double2);
constexpr size_t kScratchBytes = kPartialBytes + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};  // null until a lookup on that device has succeeded

// Device address of the scratch array on `device` (looked up with that device current; the name
// g_noalloc_scratch in host code is only a host-side stand-in, never a device address).  Only a
// successful lookup is kept: a failed one (say, inside a stream capture) is retried by the next call.
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[device]) {
        void* p = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (rc != cudaSuccess) {
            cudaGetLastError();  // the failure is reported through the return code, not left pending
            *out = nullptr;
            return rc;
        }
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace

using namespace lbm;

extern "C" int lbm_step_noalloc(const lbm_sim* sim, long n, const void* g_in, void* g_out, double* force_out,
                                void* stream) {
    clear_error();
    if (!sim) return set_error(LBM_EINVAL, "null simulation");
    if (!g_in || !g_out || !force_out) return set_error(LBM_EINVAL, "null device buffer");
    if (g_in == g_out) return set_error(LBM_EINVAL, "g_in and g_out must be different buffers");
    if (n < 0) return set_error(LBM_EINVAL, "negative step index");
    const SimView v = sim_view(sim);
    if (v.nslots > LBM_NOALLOC_MAX_SLOTS)
        return set_error(LBM_ERANGE,
                         "lbm_step_noalloc: the geometry has %d tiles with body links, more than the %d its static "
                         "scratch holds; use lbm_step, or a larger tile (lbm_set_tile)",
                         v.nslots, LBM_NOALLOC_MAX_SLOTS);
    if (v.device < 0 || v.device >= kMaxDevices) return set_error(LBM_EINVAL, "device %d out of range", v.device);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return set_error(LBM_ECUDA, "cudaGetDevice failed");
    if (cur != v.device && cudaSetDevice(v.device) != cudaSuccess)
        return set_error(LBM_ECUDA, "cudaSetDevice(%d) failed", v.device);
    void* base = nullptr;
    const cudaError_t arc = scratch_address(v.device, &base);
    if (arc != cudaSuccess || !base)
        return set_error(LBM_ECUDA, "cudaGetSymbolAddress of the step scratch: %s", cudaGetErrorString(arc));
    StepLaunchFn fn = find_step_launcher(v.Q, v.storage, v.collision, v.inst.wall_ds);
    if (!fn) return set_error(LBM_EINVAL, "no kernel for this simulation");

    unsigned char* b = static_cast<unsigned char*>(base);
    InstDev P = v.inst;
    P.src = g_in;
    P.dst = g_out;
    P.partials = reinterpret_cast<double2*>(b);
    P.ticket = reinterpret_cast<unsigned int*>(b + kPartialBytes);
    P.err = reinterpret_cast<int*>(b + kPartialBytes + 128);
    P.force_out = reinterpret_cast<double2*>(force_out);
    P.dv = drive_value(v.drive, v.u0, v.omega, n);
    P.dv_f = (float)P.dv;
    P.stream_off = 0;  // caller buffers hold plain scaled deviations: no offsets
    for (int m = 0; m < 4; ++m) P.He[m] = P.Ho[m] = 0.f;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the ticket must start at zero (a completed call leaves it at zero; this also covers a call
    // that never completed); the partials are always written before they are read
    cudaError_t e = cudaMemsetAsync(b + kPartialBytes, 0, 256, st);
    if (e == cudaSuccess) e = fn(P, dim3(v.bx, v.by), st);
    if (e == cudaSuccess && v.nslots == 0) e = cudaMemsetAsync(force_out, 0, 2 * sizeof(double), st);
    if (cur != v.device) cudaSetDevice(cur);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, "lbm_step_noalloc: %s", cudaGetErrorString(e));
    return LBM_OK;
}
