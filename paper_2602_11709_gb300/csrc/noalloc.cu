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
// The array is XRD_NOALLOC_SCRATCH_BYTES (64 MiB) per device and stays
// reserved until the process exits. When it is reserved depends on CUDA's
// module loading: with lazy loading (the default) on a device the first time
// this entry point runs there; with eager loading (CUDA_MODULE_LOADING=EAGER)
// on every device where the library's module is loaded, whether or not this
// entry point is ever called there. All calls share the array and it keeps the
// previous call's contents; the pipeline clears what must start at zero (its
// status flags) on every call. Calls that overlap on the GPU (two streams, or
// two host threads) race on the array and must be serialised by the caller.
//
// Host code cannot use the array's name as a device address. Set-up, once per
// device and context, with that device current: cudaGetSymbolAddress gives the
// address, which is cached together with the unique ID of the context it
// belongs to. A context that is destroyed and recreated (cudaDeviceReset, or
// the primary context released and retained again) has a new ID, so the
// address is looked up again instead of reusing one from the old context.
#include <cuda.h>  // CUcontext and CUresult types; the driver entry points come from the runtime

#include <mutex>

#include "xrd_launch.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[XRD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;

struct ScratchSlot {
    bool valid = false;
    unsigned long long ctx_id = 0;  // unique ID of the context the address belongs to
    void* ptr = nullptr;
};
ScratchSlot g_slot[kMaxDevices];
std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique ID of the calling thread's current context; false when it cannot be
// read (no current context yet, or a driver without the entry points).
// Caller holds g_scratch_mu.
bool current_context_id(unsigned long long* id)
{
    static bool looked_up = false;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
    }
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current context of `device`
// (which is current): the cached one while the context is the same, else a
// fresh cudaGetSymbolAddress. Without a readable context ID nothing is cached.
cudaError_t scratch_address(int device, void** ptr)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot& slot = g_slot[device];
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    if (have_id && slot.valid && slot.ctx_id == id) {
        *ptr = slot.ptr;
        return cudaSuccess;
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        slot.valid = false;
        return e;
    }
    if (!have_id) have_id = current_context_id(&id);  // the lookup may have created the context
    slot.valid = have_id;
    slot.ctx_id = id;
    slot.ptr = p;
    *ptr = p;
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
