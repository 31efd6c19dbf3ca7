// One-call batched build (nn_batch_submit): the batch entry point for callers
// that do not replay CUDA graphs.
//
// The three-step batch calls (nn_batch_query / nn_batch_prepare /
// nn_batch_launch) keep the batch description in pinned staging memory that
// the caller owns, so that one captured launch replays for every batch.
// nn_batch_submit composes the same three steps for one batch: its capacity
// is the meshes' own totals, and its staging is host memory that the call
// allocates and hands to the stream, which frees it (cudaLaunchHostFunc) once
// the batch has run.  The staging must outlive the host-to-device copy of the
// tables: on systems where the GPU reads pageable host memory directly, that
// copy may still be reading when the call returns.
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "nn_internal.h"

namespace {

nn_status caps_of(const nn_mesh* meshes, int n, int want, nn_batch_caps* c) {
    if (n < 1 || !meshes || want < 1 || want > 3) return NN_ERR_ARG;
    *c = nn_batch_caps{};
    c->max_meshes = n;
    c->want = want;
    for (int m = 0; m < n; ++m) {
        const nn_mesh& M = meshes[m];
        if (M.n_elems < 0 || M.n_nodes < 0 || M.n_conn < 0) return NN_ERR_ARG;
        c->max_elems += M.n_elems;
        c->max_nodes += M.n_nodes;
        c->max_conn += M.n_conn;
        // sums beyond the limits are refused by the batch plan; stop before they overflow
        if (c->max_elems >= (1ll << 31) || c->max_conn >= (1ll << 31) || c->max_nodes >= (1ll << 40))
            return NN_ERR_ARG;
    }
    return NN_OK;
}

void CUDART_CB free_staging(void* p) { delete static_cast<std::vector<uint64_t>*>(p); }

}  // namespace

extern "C" nn_status nn_batch_submit_query(nn_handle* h, const nn_mesh* meshes, int n_meshes, int want,
                                           size_t* ws_bytes) {
    nn_batch_caps c;
    nn_status st = caps_of(meshes, n_meshes, want, &c);
    if (st != NN_OK) return st;
    return nn_batch_query(h, &c, ws_bytes, nullptr);
}

extern "C" nn_status nn_batch_submit(nn_handle* h, const nn_mesh* meshes, nn_csr* node_out, nn_csr* elem_out,
                                     int n_meshes, void* ws, size_t ws_bytes, int32_t* d_status,
                                     nn_stream_t stream) {
    if (!h || n_meshes < 0) return NN_ERR_ARG;
    if (n_meshes == 0) return NN_OK;
    const int want = (node_out ? NN_WANT_NODES : 0) | (elem_out ? NN_WANT_ELEMS : 0);
    nn_batch_caps c;
    nn_status st = caps_of(meshes, n_meshes, want, &c);
    if (st != NN_OK) return st;
    if (nn::handle_offline(h)) return NN_ERR_ARG;
    // the staging is freed by a host function on the stream: captured in a
    // graph, every replay would free it again, so a capturing stream is refused
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cap) != cudaSuccess) return NN_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return NN_ERR_ARG;
    size_t staging_bytes = 0;
    if ((st = nn_batch_query(h, &c, nullptr, &staging_bytes)) != NN_OK) return st;
    std::vector<uint64_t>* staging = nullptr;
    try {
        staging = new std::vector<uint64_t>((staging_bytes + 7) / 8);
    } catch (...) {  // host memory exhausted
        return NN_ERR_BUDGET;
    }
    st = nn_batch_prepare(h, &c, meshes, node_out, elem_out, d_status, n_meshes, staging->data(), staging_bytes);
    if (st != NN_OK) {
        delete staging;
        return st;
    }
    st = nn_batch_launch(h, &c, staging->data(), ws, ws_bytes, stream);
    if (st == NN_ERR_ARG || st == NN_ERR_WORKSPACE) {  // refused before anything was enqueued
        delete staging;
        return st;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaLaunchHostFunc(s, free_staging, staging) != cudaSuccess) {
        // the copy may be pending: wait for the stream before freeing
        cudaStreamSynchronize(s);
        delete staging;
        return st != NN_OK ? st : NN_ERR_CUDA;
    }
    return st;
}
