// Allocation-free entry point (nn_neighbors_both_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs inside an application
// which owns all device memory through its own pool and forbids plug-ins from
// allocating, or a real-time loop that must never take the driver's
// allocation path.  For them the library keeps one fixed scratch array in
// device memory, declared below, and builds both neighbor CSRs into the
// caller's output buffers without allocating anything.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds NN_NOALLOC_SCRATCH_BYTES of it until the process exits.  In
// host code its name is only a host-side stand-in, not a device address, so
// the first call on each device looks up the real address with
// cudaGetSymbolAddress (with that device current) and keeps it, with the
// identity of the device's context; that first call should therefore come
// before any stream capture.  A later call in another context of the device
// (after cudaDeviceReset, which reloads the module) looks the address up
// again instead of using a stale one.  All calls share the
// one array and it keeps the last call's contents (the build clears the parts
// that must start at zero), so calls whose work overlaps on the GPU -- two
// streams, or a second call before the first has finished on another stream
// -- race and must be serialised by the caller.
#include <cuda.h>

#include <mutex>

#include "nn_internal.h"

namespace {

__device__ __align__(256) unsigned char g_nn_scratch[NN_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;

struct DeviceScratch {
    bool ready = false;
    void* ptr = nullptr;
    unsigned long long ctx = 0;  // unique id of the context the address belongs to (0: unknown)
    int sms = 0;
    size_t smem_optin = 0, smem_per_sm = 0;
};

DeviceScratch g_dev[MAX_DEVICES];
std::mutex g_mu;

// The unique id of the calling thread's current context, by the driver's
// cuCtxGetCurrent / cuCtxGetId (resolved once through the runtime); 0 when
// there is none or the driver does not say.  Called with g_mu held.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        resolved = true;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void**>(&get_current), 12000,
                                             cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void**>(&get_id), 12000,
                                             cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Once per device (and again after its context changed), with the device
// current: the array's device address and the limits the build plan needs.
nn_status setup(int dev, DeviceScratch* out) {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch& d = g_dev[dev];
    if (d.ready && d.ctx != 0 && current_context_id() != d.ctx) d.ready = false;  // a new context: look up again
    if (!d.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_nn_scratch) != cudaSuccess || ptr == nullptr) return NN_ERR_CUDA;
        const unsigned long long ctx = current_context_id();  // the lookup has made the context current
        int sms = 0, optin = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
            return NN_ERR_CUDA;
        if (nn::set_emit_smem_all((size_t)optin) != cudaSuccess ||
            nn::set_bucket_smem_all((size_t)optin) != cudaSuccess)
            return NN_ERR_CUDA;
        d.ptr = ptr;
        d.ctx = ctx;
        d.sms = sms;
        d.smem_optin = (size_t)optin;
        d.smem_per_sm = (size_t)per_sm;
        d.ready = true;
    }
    *out = d;
    return NN_OK;
}

}  // namespace

extern "C" nn_status nn_neighbors_both_noalloc(const nn_mesh* mesh, nn_csr* nodes, nn_csr* elems,
                                               int32_t* d_status, nn_stream_t stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NN_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return NN_ERR_ARG;
    DeviceScratch d;
    nn_status st = setup(dev, &d);
    if (st != NN_OK) return st;
    return nn::build_with_limits(d.sms, d.smem_optin, d.smem_per_sm, mesh, NN_WANT_BOTH, nodes, elems, d.ptr,
                                 NN_NOALLOC_SCRATCH_BYTES, d_status, reinterpret_cast<cudaStream_t>(stream),
                                 nullptr);
}
