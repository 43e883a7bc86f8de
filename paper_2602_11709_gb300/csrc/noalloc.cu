// Allocation-free entry point: xrd_pattern_batch_noalloc.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need a pattern: code that runs while a framework's memory pool
// owns the whole device, plug-ins whose host application forbids raw device
// allocations, and latency-critical loops where an allocation's implicit
// device synchronisation would stall other streams. For them this entry point
// runs the same pattern pipeline as xrd_pattern_batch, but its scratch space
// is a fixed file-scope device array instead of a caller-provided workspace.
//
// The array is XRD_NOALLOC_SCRATCH_BYTES (64 MiB) per device. CUDA reserves it
// on a device the first time this entry point runs there and keeps it until
// the process exits. All calls share it and it keeps the previous call's
// contents; the pipeline clears what must start at zero (its status flags) on
// every call. Calls that overlap on the GPU (two streams, or two host threads)
// race on the array and must be serialised by the caller.
#include <mutex>

#include "xrd_launch.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[XRD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(int device, void** ptr)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = p;
    }
    *ptr = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int xrd_pattern_batch_noalloc(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts,
                                         const xrd_pattern* out, void* stream)
{
    if (!h) return XRD_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return XRD_ECUDA;
    const int bound = xrd::handle_device(h);
    if (bound < 0 || bound >= kMaxDevices) return XRD_EINVAL;
    if (device != bound && cudaSetDevice(bound) != cudaSuccess) return XRD_ECUDA;
    void* scratch = nullptr;
    const cudaError_t e = scratch_address(bound, &scratch);
    int rc;
    if (e != cudaSuccess) {
        rc = xrd::set_error(h, XRD_ECUDA, "xrd_pattern_batch_noalloc: cudaGetSymbolAddress failed");
    } else {
        rc = xrd_pattern_batch(h, batch, opts, out, scratch, (size_t)XRD_NOALLOC_SCRATCH_BYTES, stream);
        if (rc == XRD_ECAPACITY)
            rc = xrd::set_error(h, XRD_ECAPACITY,
                               "xrd_pattern_batch_noalloc: the batch's per-structure and per-atom arrays do not fit "
                               "the fixed 64 MiB scratch; split the batch or use xrd_pattern_batch");
    }
    if (device != bound) cudaSetDevice(device);
    return rc;
}
