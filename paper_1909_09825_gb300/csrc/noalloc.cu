// fgt1d_execute_noalloc: the transform for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where
// they run the transform: code inside an allocator-free region of a larger runtime, a
// real-time loop with a fixed memory budget, or a host thread that must not
// synchronise with the device allocator.  This entry point takes only the inputs and
// the output; its scratch is a fixed array in the library's own device memory,
// reserved on every GPU that loads the library and held until the process exits.
//
// Limits and contract:
//  - the scratch holds kNoAllocBytes (16 MiB), enough for any plan (FP64 or FP32,
//    any n_e) with M + N <= 65,536 points; more points return FGT1D_ETOOLARGE;
//  - the first call on a device with work to do looks up the array's device address
//    (once per device, with that device current; a failed lookup is retried by the next
//    call); make that first call before any stream capture;
//  - every call shares the one array and its contents persist between calls; the
//    transform clears the parts that must start at zero itself;
//  - calls whose GPU work can overlap (on different streams, or from several threads
//    without ordering) race on the array and give wrong results: order them;
//  - device-side conditions (a NaN/Inf coordinate, an expired wait) are recorded in the
//    array's header and are not reported back by this entry point.
#include <cuda_runtime.h>

#include <mutex>

#include "fgt1d_internal.h"
#include "kernels.h"

namespace fgt1d {
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;
constexpr int64_t kNoAllocMaxPoints = 65536;  // M + N; the largest plan (n_e = 8, FP64) needs 10.3 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array per device, set once a lookup has succeeded.  A
// failed lookup (e.g. made while the stream was capturing) is not remembered: the next
// call tries again.
std::mutex g_lock;
void* g_scratch[kMaxDevices];

int scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> hold(g_lock);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();  // reset the runtime's last-error state for the caller's next call
            return FGT1D_ECUDA;
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return FGT1D_OK;
}

}  // namespace
}  // namespace fgt1d

extern "C" int fgt1d_execute_noalloc(fgt1d_plan plan, const double* x, int64_t M, const double* y,
                                     const double* alpha, int64_t N, double* u, fgt1d_stream stream) {
    using namespace fgt1d;
    if (!plan || M < 0 || N < 0 || M + N >= (int64_t(1) << 31)) return FGT1D_EINVAL;
    // the same pointer rules as fgt1d_execute, checked before anything reaches the GPU
    if (M > 0 && (!x || !u)) return FGT1D_EINVAL;
    if (N > 0 && M > 0 && (!y || !alpha)) return FGT1D_EINVAL;
    if (M + N > kNoAllocMaxPoints || transform_workspace_bytes(*plan, M, N) > kNoAllocBytes) return FGT1D_ETOOLARGE;
    if (M == 0 || N == 0)  // nothing to sort: no scratch needed
        return run_transform_in(*plan, x, M, y, alpha, N, u, nullptr, 0, static_cast<cudaStream_t>(stream));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FGT1D_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return FGT1D_EUNSUPPORTED;
    void* scratch = nullptr;
    const int r = scratch_address(dev, &scratch);
    if (r) return r;
    return run_transform_in(*plan, x, M, y, alpha, N, u, scratch, kNoAllocBytes, static_cast<cudaStream_t>(stream));
}
