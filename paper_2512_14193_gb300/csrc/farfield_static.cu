// bm_far_field_static: the far field of bm_far_field without any device allocation.
//
// Who needs it: callers that must not allocate device memory while they run.  bm_far_field
// allocates a small device buffer for the observation angles on every call (charged to the
// handle's HBM budget) and frees it afterwards: it fails outright once resident factorisations
// have used the budget up, and each allocation may have to grow the device's memory pool, which a
// caller that holds a fixed device-memory footprint (a serving loop sized to the GPU) cannot
// allow.  This entry point launches the same far-field kernel on the same data, but reads the
// angles from a fixed device array compiled into the library.
//
// Scratch: g_ff_angles below, BM_FAR_FIELD_STATIC_MAX_ANGLES doubles (8192 x 8 bytes = 64 KB);
// the linker gives each device its own copy.  A call copies its M angles into the first M
// entries before the kernel reads them, and the kernel reads nothing else, so no part of the
// array has to start at zero and the call clears none of it.
//
// Set-up: the first call on a device, with that device current, looks up the device address of
// the array (cudaGetSymbolAddress) and keeps it for later calls on that device, together with the
// unique ID of the CUDA context it belongs to (a context created after a reset gets a new ID, even
// where the driver reuses the old context's handle).  The lookup can load the library's device code onto the device, so
// make this first call before any stream capture starts on the device.  If the device's context
// has been replaced since (cudaDeviceReset, then new work), the address is looked up again: an
// address from the old context would no longer belong to the array.
//
// Overlapping calls race: the array is shared by every handle and host thread that uses the
// device, so two calls running at the same time can overwrite each other's angles before the
// kernel reads them.  Each call waits for its stream to finish before it returns, so calls made
// one after another, from any handle, are safe.
#include "common.cuh"
#include "kernels.cuh"

#include <cmath>
#include <mutex>

static __device__ __align__(256) double g_ff_angles[BM_FAR_FIELD_STATIC_MAX_ANGLES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
double* g_angles_ptr[MAX_DEVICES] = {};
unsigned long long g_angles_ctx[MAX_DEVICES] = {};  // ID of the context each address was looked up in

// Device address of g_ff_angles on `dev` (the current device), looked up once per device and
// context.
bm_status angles_scratch(int dev, double** out) {
    if (dev < 0 || dev >= MAX_DEVICES) {
        bm_set_error("bm_far_field_static: device index " + std::to_string(dev) + " out of range");
        return BM_EINVAL;
    }
    const unsigned long long ctx = cuda_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_angles_ptr[dev] == nullptr || ctx == 0 || ctx != g_angles_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ff_angles);
        if (e != cudaSuccess || p == nullptr) {
            bm_set_error(std::string("bm_far_field_static: cudaGetSymbolAddress failed: ") +
                         cudaGetErrorString(e));
            return BM_ECUDA;
        }
        g_angles_ptr[dev] = static_cast<double*>(p);
        g_angles_ctx[dev] = ctx;
    }
    *out = g_angles_ptr[dev];
    return BM_OK;
}

}  // namespace

extern "C" bm_status bm_far_field_static(bm_ctx* c, const bm_c64* X, int ldx, int nrhs, const double* angles, int M,
                                         bm_c64* Uinf, int ldu) {
    if (c == nullptr || X == nullptr || angles == nullptr || Uinf == nullptr || nrhs < 1 || M < 1) return BM_EINVAL;
    if (M > BM_FAR_FIELD_STATIC_MAX_ANGLES) {
        bm_set_error("bm_far_field_static: M = " + std::to_string(M) + " angles exceeds the fixed device array of " +
                     std::to_string(BM_FAR_FIELD_STATIC_MAX_ANGLES) + " (use bm_far_field, or split the angles)");
        return BM_EINVAL;
    }
    if (!c->assembled) return BM_ESTATE;
    if (ldx < c->nsys || ldu < M) return BM_EINVAL;
    for (int i = 0; i < M; ++i)
        if (!std::isfinite(angles[i])) {
            bm_set_error("bm_far_field_static: angle " + std::to_string(i) + " is not finite");
            return BM_ENONFINITE;
        }
    BM_CUDA_TRY(cudaSetDevice(c->device));
    double* d_ang = nullptr;
    BM_TRY(angles_scratch(c->device, &d_ang));
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemcpyAsync(d_ang, angles, (size_t)M * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        e = launch_far_field(s, c, reinterpret_cast<const double2*>(X), ldx, nrhs, d_ang, M,
                             reinterpret_cast<double2*>(Uinf), ldu);
        c->launches += 1;
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        bm_set_error(std::string("bm_far_field_static: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return BM_ECUDA;
    }
    return BM_OK;
}
