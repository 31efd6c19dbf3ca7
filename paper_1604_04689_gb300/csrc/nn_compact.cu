// Node-CSR placement: the bucket pass leaves every bucket's distinct-
// neighbour rows in a scratch area at a position bounded in advance (K times
// the bucket's first record: a record adds at most K neighbours), with each
// node's offset inside its bucket and the bucket's total.  Two short kernels
// then place them: an exclusive scan of the bucket totals (single pass,
// decoupled lookback over tiles of buckets), and a copy of every bucket's rows
// to its offset in the mesh's col, with the row pointers.  No bucket ever waits
// for another while it builds its rows.
#include "nn_device.cuh"

namespace nn {

namespace {

constexpr int SCAN_THREADS = 128;
constexpr int COPY_THREADS = 256;

__global__ void __launch_bounds__(SCAN_THREADS) k_node_scan(CompactParams p) {
    __shared__ uint64_t sh_scan[33];
    __shared__ uint32_t sh_tile;
    __shared__ uint64_t sh_base;
    const int64_t B = p.batch.hdr ? p.batch.hdr->n_buckets : p.n_buckets;
    if (threadIdx.x == 0) sh_tile = atomicAdd(p.ticket, 1u);
    __syncthreads();
    const uint32_t tile = sh_tile;
    const int64_t b = (int64_t)tile * SCAN_THREADS + threadIdx.x;
    if ((int64_t)tile * SCAN_THREADS >= B) return;  // whole CTA: no buckets left
    const uint64_t x = b < B ? p.ubk[b] : 0;
    uint64_t agg;
    const uint64_t ex = block_excl_scan(x, &agg, sh_scan);
    if (threadIdx.x < 32) {
        const uint64_t base = warp_lookback(p.lb_state, tile, agg, p.status);
        if (threadIdx.x == 0) sh_base = base;
    }
    __syncthreads();
    if (b < B) p.nstart[b] = sh_base + ex;
    if (b == B - 1) p.nstart[B] = sh_base + ex + x;
}

__global__ void __launch_bounds__(COPY_THREADS) k_node_copy(CompactParams p) {
    const bool batched = p.batch.hdr != nullptr;
    const int64_t B = batched ? p.batch.hdr->n_buckets : p.n_buckets;
    const int sb = batched ? p.batch.hdr->fmt.sb : p.sb;
    const int K = batched ? 3 : p.k;
    const int n_meshes = batched ? p.batch.hdr->n_meshes : 1;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        int64_t first = 0, N = p.n_nodes;
        int64_t* rp = p.rp_n;
        int32_t* col = p.col_n;
        int64_t cap = p.cap_n;
        int32_t* status = p.status;
        bool last = b == B - 1;
        if (batched) {
            int lo = 0, hi = n_meshes;  // largest m with bucket_off[m] <= b
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (p.batch.bucket_off[mid] <= b) lo = mid;
                else hi = mid;
            }
            const BatchMesh& M = p.batch.meshes[lo];
            first = p.batch.bucket_off[lo];
            last = b == p.batch.bucket_off[lo + 1] - 1;
            N = M.n_nodes;
            rp = M.rp_n;
            col = M.col_n;
            cap = M.cap_n;
            status = M.status;
        }
        const uint64_t gn = p.nstart[b] - p.nstart[first] + (p.base ? (uint64_t)p.base[1] : 0ull);
        const uint32_t ub = p.ubk[b];
        const int64_t v0 = (b - first) << sb;
        const int nb = (int)(N - v0 < ((int64_t)1 << sb) ? N - v0 : ((int64_t)1 << sb));
        const uint32_t* loc = p.nloc + ((size_t)b << sb);
        for (int l = threadIdx.x; l < nb; l += COPY_THREADS)
            if (NN_IN(((size_t)b << sb) + l, p.nloc_words, status)) rp[v0 + l] = (int64_t)(gn + loc[l]);
        if (last && threadIdx.x == 0) rp[N] = (int64_t)(gn + ub);
        if (gn + ub > (uint64_t)cap) {
            if (threadIdx.x == 0) set_status(status, NN_ERR_CAPACITY);
            continue;
        }
        const uint32_t* src = p.ntmp + (size_t)K * p.bstart[b];
        int32_t* dst = col + gn;
        if (!NN_IN((size_t)K * p.bstart[b] + (ub ? ub - 1 : 0), p.ntmp_words + (ub ? 0 : 1), status)) continue;
        for (uint32_t i = threadIdx.x; i < ub; i += COPY_THREADS) dst[i] = (int32_t)__ldg(src + i);
    }
}

// Chunked builds run one node range after another into the same CSRs; after
// a chunk, the running bases move past its element and node entries.
__global__ void k_chunk_advance(int64_t* base, const uint32_t* estart, const uint64_t* nstart, int64_t B) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (estart) base[0] += (int64_t)estart[B];
        if (nstart) base[1] += (int64_t)nstart[B];
    }
}

}  // namespace

cudaError_t launch_chunk_advance(int64_t* base, const uint32_t* estart, const uint64_t* nstart, int64_t B,
                                 cudaStream_t s) {
    k_chunk_advance<<<1, 32, 0, s>>>(base, estart, nstart, B);
    return cudaGetLastError();
}

cudaError_t launch_node_compact(const CompactParams& p, int copy_grid, cudaStream_t s) {
    const int64_t B = p.n_buckets_cap;
    const unsigned tiles = (unsigned)((B + SCAN_THREADS - 1) / SCAN_THREADS);
    if (tiles == 0) return cudaSuccess;
    k_node_scan<<<tiles, SCAN_THREADS, 0, s>>>(p);
    k_node_copy<<<copy_grid, COPY_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace nn
