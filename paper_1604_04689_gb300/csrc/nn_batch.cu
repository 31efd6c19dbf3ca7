// Batched element walk: many meshes of any types in one launch sequence.
//
// The batch tables (header, one BatchMesh per mesh, element and bucket
// offsets) are in device memory, so the grids below do not depend on the
// batch: persistent grid-stride loops read the totals from the header, and a
// captured launch sequence can be replayed for every batch that fits the
// workspace.  Each mesh owns a contiguous range of buckets; bucket counts are
// gathered with global reductions (a batch can have far more buckets than a
// shared-memory histogram holds), then the same offsets scan, record format
// and bucket pass as the single-mesh build turn them into per-mesh CSRs.
#include "nn_device.cuh"

namespace nn {

namespace {

constexpr int BATCH_THREADS = 256;
constexpr int CHUNK = 8;  // elements per lane per warp chunk

// Load element e of mesh M (any type); returns its type, sets *ok.
__device__ __forceinline__ int load_elem_any(const BatchMesh& M, int64_t e, int32_t* nd, bool* ok) {
    int t = M.type;
    int npe;
    if (t == NN_MIXED) {
        t = __ldg(M.elem_type + e);
        const int64_t a = __ldg(M.elem_ptr + e), b = __ldg(M.elem_ptr + e + 1);
        if (t > NN_HEX || a < 0 || b > M.n_conn || b - a != npe_of(t)) {
            set_status(M.status, NN_ERR_ELEM_PTR);
            *ok = false;
            return NN_HEX;
        }
        npe = (int)(b - a);
#pragma unroll
        for (int q = 0; q < 8; ++q) nd[q] = q < npe ? __ldg(M.conn + a + q) : 0;
    } else if (t == NN_TRI) {
        npe = 3;
        nd[0] = __ldg(M.conn + 3 * e);
        nd[1] = __ldg(M.conn + 3 * e + 1);
        nd[2] = __ldg(M.conn + 3 * e + 2);
    } else if (t == NN_HEX) {
        npe = 8;
        const int4* c4 = reinterpret_cast<const int4*>(M.conn) + 2 * e;
        int4 x = __ldg(c4), y = __ldg(c4 + 1);
        nd[0] = x.x; nd[1] = x.y; nd[2] = x.z; nd[3] = x.w;
        nd[4] = y.x; nd[5] = y.y; nd[6] = y.z; nd[7] = y.w;
    } else {
        npe = 4;
        int4 x = __ldg(reinterpret_cast<const int4*>(M.conn) + e);
        nd[0] = x.x; nd[1] = x.y; nd[2] = x.z; nd[3] = x.w;
    }
    bool v = true;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (q < npe) v = v && nd[q] >= 0 && (int64_t)nd[q] < M.n_nodes;
    if (!v) set_status(M.status, NN_ERR_NODE_RANGE);
    *ok = v;
    return t;
}

// Walk all elements of the batch, warp chunk by warp chunk (lanes interleaved
// for coalesced loads), calling f(mesh index, mesh, local element id, type,
// nodes) for every valid element.
template <class F>
__device__ __forceinline__ void walk_batch(const BatchTables& bt, F&& f) {
    const int64_t total = bt.hdr->n_elems;
    const int n_meshes = bt.hdr->n_meshes;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_chunks = (total + 32 * CHUNK - 1) / (32 * CHUNK);
    for (int64_t c = warp; c < n_chunks; c += n_warps) {
        const int64_t e0 = c * 32 * CHUNK;
        int lo = 0, hi = n_meshes;  // largest m with elem_off[m] <= e0
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (bt.elem_off[mid] <= e0) lo = mid;
            else hi = mid;
        }
        int m = lo;
        for (int i = 0; i < CHUNK; ++i) {
            const int64_t e = e0 + (int64_t)i * 32 + lane;
            if (e >= total) break;
            while (e >= bt.elem_off[m + 1]) ++m;
            const BatchMesh& M = bt.meshes[m];
            int32_t nd[8];
            bool ok;
            const int64_t le = e - bt.elem_off[m];
            const int t = load_elem_any(M, le, nd, &ok);
            if (ok) f(m, M, le, t, nd);
        }
    }
}

__global__ void __launch_bounds__(BATCH_THREADS) k_batch_init(BatchTables bt, uint32_t* bcount, uint32_t* nfc,
                                                              uint64_t* lb_off, uint32_t* ctrl, uint64_t* lb_ns) {
    const int64_t B = bt.hdr->n_buckets;
    const int64_t tiles = (B + OFFSETS_THREADS - 1) / OFFSETS_THREADS;
    const int n = bt.hdr->n_meshes;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0; i < B; i += st) {
        bcount[i] = 0;
        nfc[i] = 0;
    }
    for (int64_t i = i0; i < tiles + 1; i += st) lb_off[i] = 0;
    if (lb_ns)
        for (int64_t i = i0; i < (B + 127) / 128 + 1; i += st) lb_ns[i] = 0;
    for (int64_t i = i0; i < 16; i += st) ctrl[i] = 0;
    for (int64_t i = i0; i < n; i += st) {
        const BatchMesh& M = bt.meshes[i];
        *M.status = 0;
        if (M.n_nodes == 0) {  // no bucket will write the single row pointer
            if (M.rp_n) M.rp_n[0] = 0;
            if (M.rp_e) M.rp_e[0] = 0;
        }
    }
}

// Records per bucket, and (rare) records of a node already seen in its
// element, which add no element entry.
__global__ void __launch_bounds__(BATCH_THREADS) k_hist_b(BatchTables bt, uint32_t* bcount, uint32_t* nfc) {
    const int sb = bt.hdr->fmt.sb;
    walk_batch(bt, [&](int m, const BatchMesh& M, int64_t, int t, const int32_t* nd) {
        const int npe = npe_of(t);
        uint32_t* cnt = bcount + bt.bucket_off[m];
        uint32_t* rep = nfc + bt.bucket_off[m];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i >= npe) break;
            atomicAdd(&cnt[(uint32_t)nd[i] >> sb], 1u);
            int nf = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) nf |= (q < i) && (nd[q] == nd[i]);
            if (nf) atomicAdd(&rep[(uint32_t)nd[i] >> sb], 1u);
        }
    });
}

__global__ void __launch_bounds__(BATCH_THREADS) k_part_b(BatchTables bt, uint32_t* gcur, uint8_t* rec) {
    const RecFmt f = bt.hdr->fmt;
    const uint64_t cap = (uint64_t)bt.hdr->n_records;
    const uint32_t vmask = (1u << f.sb) - 1;
    walk_batch(bt, [&](int m, const BatchMesh& M, int64_t le, int t, const int32_t* nd) {
        const int npe = npe_of(t), K = k_of(t);
        uint32_t* cur = gcur + bt.bucket_off[m];
        uint32_t pos[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) pos[i] = i < npe ? atomicAdd(&cur[(uint32_t)nd[i] >> f.sb], 1u) : 0xFFFFFFFFu;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (pos[i] >= cap) continue;
            const int32_t v = nd[i];
            int nf = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) nf |= (q < i) && (nd[q] == v);
            Rec r{(uint64_t)((uint32_t)v & vmask), 0};
            if (f.want & NN_WANT_ELEMS) {
                rec_put(r, (uint64_t)nf, f.off_nf);
                rec_put(r, (uint64_t)le, f.off_e);
            }
            if (f.want & NN_WANT_NODES) {
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    if (s >= K) break;
                    const int32_t y = nbr_node(t, nd, i, s);
                    rec_put(r, y == v ? 0ull : (uint64_t)(uint32_t)(y + 1), f.off_n + s * f.nb);
                }
            }
            reinterpret_cast<ulonglong2*>(rec)[pos[i]] = make_ulonglong2(r.lo, r.hi);
        }
    });
}

}  // namespace

cudaError_t launch_batch_emit(const BatchTables& bt, uint32_t* bcount, uint32_t* nfc, uint32_t* gcur, uint8_t* rec,
                              uint64_t* lb_off, uint32_t* ctrl, int grid, int stage, cudaStream_t s,
                              uint64_t* lb_ns) {
    if (stage == 0) k_batch_init<<<grid, BATCH_THREADS, 0, s>>>(bt, bcount, nfc, lb_off, ctrl, lb_ns);
    else if (stage == 1) k_hist_b<<<grid, BATCH_THREADS, 0, s>>>(bt, bcount, nfc);
    else k_part_b<<<grid, BATCH_THREADS, 0, s>>>(bt, gcur, rec);
    return cudaGetLastError();
}

int batch_threads() { return BATCH_THREADS; }

}  // namespace nn
