// Diagnostic entry point for the bounded device-side waits.
//
// The single-pass scans of a build (bucket offsets, node-row placement,
// element-adjacency offsets) wait for their predecessor tiles in the
// decoupled lookback of nn_device.cuh.  That wait gives up after
// WAIT_LIMIT_NS without progress, writes NN_ERR_TIMEOUT to the call's status
// word, publishes its own tile so that later tiles do not wait as well, and
// returns.  In a correct build every predecessor publishes and the limit is
// never reached.  nn_diag_wait_timeout runs the same wait for a tile whose
// predecessor never publishes, so that a test can check that the wait ends,
// that the status is reported, and that the context stays usable afterwards.
#include "nn_device.cuh"

namespace nn {
namespace {

// One warp resolves tile 1 of a three-word state: word 0 (tile 0) stays
// zero (not ready) for the whole run, word 1 receives tile 1's inclusive
// prefix when the wait ends, word 2 the time the wait took in ns.
__global__ void __launch_bounds__(32) k_wait_probe(uint64_t* state, int32_t* status) {
    const uint64_t t0 = global_ns();
    lb_resolve(state, 1, 1, status);
    if (threadIdx.x == 0) state[2] = global_ns() - t0;
}

}  // namespace
}  // namespace nn

extern "C" nn_status nn_diag_wait_timeout(uint64_t* d_state, int32_t* d_status, nn_stream_t stream) {
    if (!d_state || !d_status || (reinterpret_cast<uintptr_t>(d_state) & 7) ||
        (reinterpret_cast<uintptr_t>(d_status) & 3))
        return NN_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_state, 0, 3 * sizeof(uint64_t), s) != cudaSuccess ||
        cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess)
        return NN_ERR_CUDA;
    nn::k_wait_probe<<<1, 32, 0, s>>>(d_state, d_status);
    return cudaGetLastError() == cudaSuccess ? NN_OK : NN_ERR_CUDA;
}
