// qs_norm_noalloc: the norm reduction for callers that cannot allocate.
//
// qs_norm needs a qs_state, and creating or wrapping one allocates device
// scratch (the per-block partial sums) and a pinned host buffer.  Some
// callers cannot do that: a process whose device memory has been reserved up
// front by another allocator (a framework's caching allocator, say), an
// application that fixes its device-memory budget at start-up, or code that
// must stay off the driver's allocation path because cudaMalloc/cudaFree can
// synchronise the device.  This entry point takes the amplitudes as a raw
// device pointer and keeps its scratch in a fixed array in the library's
// device image instead, so it allocates nothing at all.
#include <mutex>

#include "qs_internal.h"

namespace qsgb {

// Partial sums (one per reduction block) followed by the result slot.
constexpr int kNoAllocMaxPartials = 4096;
static __device__ __align__(256) double g_norm_scratch[kNoAllocMaxPartials + 8];

// Device address of g_norm_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress (with that device current).  Outside stream capture
// every call looks it up again, so the address stays right after a device
// reset reloads the library's module; a call made during a capture uses
// the address found by the last call on that device outside any capture.
constexpr int kNoAllocMaxDevices = 64;
static double* g_norm_scratch_dev[kNoAllocMaxDevices] = {nullptr};
static std::mutex g_norm_scratch_mu;

static qs_status norm_scratch_address(int dev, cudaStream_t st, double** out) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    QS_CUDA(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lock(g_norm_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(norm scratch)");
        g_norm_scratch_dev[dev] = static_cast<double*>(p);
    } else if (!g_norm_scratch_dev[dev]) {
        return fail(QS_ERR_STATE, "first qs_norm_noalloc call on device %d made during stream capture", dev);
    }
    *out = g_norm_scratch_dev[dev];
    return QS_OK;
}

}  // namespace qsgb

using namespace qsgb;

extern "C" qs_status qs_norm_noalloc(const void* device_amplitudes, int n, qs_dtype dt, void* stream,
                                     double* out) {
    if (!device_amplitudes || !out) return fail(QS_ERR_ARG, "null argument");
    if (((uintptr_t)device_amplitudes) & 15) return fail(QS_ERR_ARG, "amplitudes not 16-byte aligned");
    if (n < 1 || n > kMaxQubits) return fail(QS_ERR_ARG, "n=%d outside 1..%d", n, kMaxQubits);
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_ERR_ARG, "bad dtype");
    int dev = -1;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(QS_ERR_UNSUPPORTED, "device %d beyond the %d devices this entry point tracks", dev,
                    kNoAllocMaxDevices);
    const int nb = reduce_blocks();
    if (nb > kNoAllocMaxPartials)
        return fail(QS_ERR_UNSUPPORTED,
                    "this GPU needs %d partial sums, more than the %d the fixed scratch array holds", nb,
                    kNoAllocMaxPartials);
    cudaStream_t s = (cudaStream_t)stream;
    double* scratch = nullptr;
    qs_status st = norm_scratch_address(dev, s, &scratch);
    if (st != QS_OK) return st;
    // every partial the sum reads is written by the same call, and the
    // result slot is overwritten, so nothing needs clearing first
    QS_CUDA(launch_norm(device_amplitudes, n, dt, scratch, scratch + kNoAllocMaxPartials, s));
    QS_CUDA(cudaMemcpyAsync(out, scratch + kNoAllocMaxPartials, sizeof(double), cudaMemcpyDeviceToHost, s));
    QS_CUDA(cudaStreamSynchronize(s));
    return QS_OK;
}
