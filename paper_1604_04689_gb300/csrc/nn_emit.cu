// Element walk kernels: bucket histogram, bucket offsets, partition.
//
// The paper's GPU recipe (Sec. 2.2.1) has one thread per triangle emit its
// integer pairs and then sorts them by key.  Here the pairs of one node never
// leave a packed per-incidence record (node, element, the node's edge
// neighbours in that element), and records are partitioned by node range
// ("bucket") instead of sorted: a histogram pass over the connectivity (each
// CTA owns a fixed slice of elements and counts into shared memory), a scan
// of the bucket totals, and a partition pass that appends every record to
// its bucket through one cursor per bucket, so the random global traffic is
// one L2 atomic and one vector store per incidence, and the partially filled
// sectors at the buckets' write heads (one per bucket) stay resident in L2.
#include <algorithm>

#include "nn_bulk.cuh"

namespace nn {

namespace {

// A checked node id relative to the build's first node (vr), and whether it
// lies in the build's node range.  RANGED = false is a whole-mesh build:
// every checked id is in range and vr = v, with no arithmetic at all.
template <bool RANGED>
__device__ __forceinline__ bool node_in(const EmitParams& p, int32_t v, uint32_t& vr) {
    if constexpr (RANGED) {
        const uint64_t r = (uint64_t)((int64_t)v - p.node_lo);  // a node before the range wraps above every span
        vr = (uint32_t)r;
        return r < (uint64_t)p.node_span;
    } else {
        vr = (uint32_t)v;
        return true;
    }
}

__host__ __device__ inline bool ranged(const EmitParams& p) { return p.node_lo != 0 || p.node_span != p.n_nodes; }

// The npe (<= 8) nodes of a mixed mesh's element at conn[a ..]: 16-byte loads
// when the element starts on a 16-byte boundary (hex and tet elements of a
// mesh whose earlier elements all have 4 or 8 nodes), else one load per node.
// Entries from npe on are 0.
__device__ __forceinline__ void load_mixed_nodes(const int32_t* conn, int64_t a, int npe, int32_t* nd) {
    const int32_t* src = conn + a;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (npe == 4 || npe == 8)) {
        const int4 x = __ldg(reinterpret_cast<const int4*>(src));
        nd[0] = x.x; nd[1] = x.y; nd[2] = x.z; nd[3] = x.w;
        if (npe == 8) {
            const int4 y = __ldg(reinterpret_cast<const int4*>(src) + 1);
            nd[4] = y.x; nd[5] = y.y; nd[6] = y.z; nd[7] = y.w;
        } else {
            nd[4] = nd[5] = nd[6] = nd[7] = 0;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) nd[q] = q < npe ? __ldg(src + q) : 0;
    }
}

// Per-incidence callback signature: (v, nf, e, x0, x1, x2) with x_s = -1 for none.
template <int TYPE, class F>
__device__ __forceinline__ void visit_elem(const int32_t* nd, int64_t e, int64_t n_nodes, int32_t* status,
                                           int t_rt, F&& f) {
    constexpr int NPE = TYPE == NN_MIXED ? 8 : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::NPE;
    const int npe = TYPE == NN_MIXED ? npe_of(t_rt) : NPE;
    const int t = TYPE == NN_MIXED ? t_rt : TYPE;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < NPE; ++i)
        if (i < npe && (nd[i] < 0 || (int64_t)nd[i] >= n_nodes)) ok = false;
    if (!ok) {
        set_status(status, NN_ERR_NODE_RANGE);
        return;
    }
    const int K = TYPE == NN_MIXED ? k_of(t) : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::K;
#pragma unroll
    for (int i = 0; i < NPE; ++i) {
        if (i >= npe) break;
        const int32_t v = nd[i];
        int nf = 0;
#pragma unroll
        for (int j = 0; j < i; ++j) nf |= (nd[j] == v);
        int32_t x[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            int32_t y = -1;
            if (s < K) {
                y = TYPE == NN_MIXED ? nbr_node(t, nd, i, s) : nd[ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::nbr(i, s)];
                if (y == v) y = -1;
            }
            x[s] = y;
        }
        f(v, nf, e, x[0], x[1], x[2]);
    }
}

// Walk this CTA's slice of work units and call f for every valid incidence.
template <int TYPE, class F>
__device__ __forceinline__ void walk_cta(const EmitParams& p, F&& f) {
    constexpr int UNIT = TYPE == NN_TRI ? 4 : 1;
    const int64_t n_units = (p.n_elems + UNIT - 1) / UNIT;
    const int64_t u0 = n_units * blockIdx.x / gridDim.x, u1 = n_units * (blockIdx.x + 1) / gridDim.x;
    for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        if constexpr (TYPE == NN_TRI) {
            const int64_t e0 = u * 4;
            int32_t nd[12];
            if (e0 + 4 <= p.n_elems) {
                const int4* c4 = reinterpret_cast<const int4*>(p.conn + e0 * 3);
                int4 a = __ldg(c4), b = __ldg(c4 + 1), c = __ldg(c4 + 2);
                nd[0] = a.x; nd[1] = a.y; nd[2] = a.z; nd[3] = a.w;
                nd[4] = b.x; nd[5] = b.y; nd[6] = b.z; nd[7] = b.w;
                nd[8] = c.x; nd[9] = c.y; nd[10] = c.z; nd[11] = c.w;
            } else {
                for (int q = 0; q < 12; ++q) nd[q] = (e0 * 3 + q < p.n_conn) ? __ldg(p.conn + e0 * 3 + q) : 0;
            }
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if (e0 + w < p.n_elems) visit_elem<NN_TRI>(nd + 3 * w, e0 + w, p.n_nodes, p.status, NN_TRI, f);
        } else if constexpr (TYPE == NN_QUAD || TYPE == NN_TET) {
            int4 a = __ldg(reinterpret_cast<const int4*>(p.conn) + u);
            int32_t nd[4] = {a.x, a.y, a.z, a.w};
            visit_elem<TYPE>(nd, u, p.n_nodes, p.status, TYPE, f);
        } else if constexpr (TYPE == NN_HEX) {
            const int4* c4 = reinterpret_cast<const int4*>(p.conn) + 2 * u;
            int4 a = __ldg(c4), b = __ldg(c4 + 1);
            int32_t nd[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            visit_elem<NN_HEX>(nd, u, p.n_nodes, p.status, NN_HEX, f);
        } else {  // mixed
            const int t = __ldg(p.elem_type + u);
            const int64_t a = __ldg(p.elem_ptr + u), b = __ldg(p.elem_ptr + u + 1);
            if (t > NN_HEX || a < 0 || b > p.n_conn || b - a != npe_of(t)) {
                set_status(p.status, NN_ERR_ELEM_PTR);
                continue;
            }
            int32_t nd[8];
            load_mixed_nodes(p.conn, a, (int)(b - a), nd);
            visit_elem<NN_MIXED>(nd, u, p.n_nodes, p.status, t, f);
        }
    }
}

// Counts per bucket of this CTA's element slice, in shared memory.  When the
// buckets outnumber the shared counters (hist_chunk), the slice is walked once
// per chunk of buckets.
//
// With twice as many buckets as 32-bit counters fit (p.hist_chunk < B <=
// 2 p.hist_chunk) the slice is first counted in one walk with two 16-bit
// counters per word.  A count that would pass 65535 carries into its
// neighbour; the thread whose add would do so sees the old value, flags the
// CTA, and the CTA counts its slice again with 32-bit counters.
template <int TYPE, bool RANGED>
__global__ void __launch_bounds__(EMIT_THREADS) k_hist(EmitParams p) {
    extern __shared__ uint32_t sh_hist[];  // (no static shared memory: the dynamic part may take the whole limit)
    const int64_t B = p.n_buckets;
    const int sb = p.fmt.sb;
    uint32_t* row = p.hist + (int64_t)blockIdx.x * B;
    if (B > p.hist_chunk && B <= 2 * p.hist_chunk) {
        const int64_t words = (B + 1) / 2;
        for (int64_t w = threadIdx.x; w < words; w += blockDim.x) sh_hist[w] = 0;
        __syncthreads();
        bool wrapped = false;
        walk_cta<TYPE>(p, [&](int32_t v, int nf, int64_t, int32_t, int32_t, int32_t) {
            uint32_t vr;
            if (!node_in<RANGED>(p, v, vr)) return;  // another chunk's node
            const uint32_t b = vr >> sb, sh = (b & 1u) * 16u;
            const uint32_t old = atomicAdd(&sh_hist[b >> 1], 1u << sh);
            wrapped |= ((old >> sh) & 0xFFFFu) == 0xFFFFu;
            if (nf && p.nfc && NN_IN(b, B, p.status)) atomicAdd(&p.nfc[b], 1u);  // rare: degenerate elements only
        });
        if (!__syncthreads_or(wrapped)) {
            for (int64_t b = threadIdx.x; b < B; b += blockDim.x)
                if (NN_IN((int64_t)blockIdx.x * B + b, p.hist_words, p.status))
                    row[b] = (sh_hist[b >> 1] >> ((b & 1) * 16)) & 0xFFFFu;
            return;
        }
        __syncthreads();  // a count wrapped: count again below (the repeated-node counts are complete)
    }
    const bool nf_done = B > p.hist_chunk && B <= 2 * p.hist_chunk;
    for (int64_t c0 = 0; c0 < B; c0 += p.hist_chunk) {
        const int64_t nc = min(B - c0, p.hist_chunk);
        for (int64_t b = threadIdx.x; b < nc; b += blockDim.x) sh_hist[b] = 0;
        __syncthreads();
        walk_cta<TYPE>(p, [&](int32_t v, int nf, int64_t, int32_t, int32_t, int32_t) {
            uint32_t vr;
            if (!node_in<RANGED>(p, v, vr)) return;  // another chunk's node
            const int64_t b = (int64_t)(vr >> sb) - c0;
            if (b >= 0 && b < nc) atomicAdd(&sh_hist[b], 1u);
            if (nf && c0 == 0 && !nf_done && p.nfc && NN_IN(vr >> sb, B, p.status))
                atomicAdd(&p.nfc[vr >> sb], 1u);  // rare: degenerate elements only
        });
        __syncthreads();
        for (int64_t b = threadIdx.x; b < nc; b += blockDim.x)
            if (NN_IN((int64_t)blockIdx.x * B + c0 + b, p.hist_words, p.status)) row[c0 + b] = sh_hist[b];
        __syncthreads();
    }
}

// Incidences per node slab (2^shift consecutive nodes), for planning a
// chunked build: one shared counter per slab, added to counts at the end.
template <int TYPE>
__global__ void __launch_bounds__(EMIT_THREADS) k_slab_count(EmitParams p, int shift, int n_slabs, uint32_t* counts) {
    __shared__ uint32_t sh_cnt[NN_CHUNK_SLABS_MAX];
    for (int i = threadIdx.x; i < n_slabs; i += blockDim.x) sh_cnt[i] = 0;
    __syncthreads();
    walk_cta<TYPE>(p, [&](int32_t v, int, int64_t, int32_t, int32_t, int32_t) {
        const int s = v >> shift;  // v is a checked node id, so s < n_slabs
        if (s < n_slabs) atomicAdd(&sh_cnt[s], 1u);
    });
    __syncthreads();
    for (int i = threadIdx.x; i < n_slabs; i += blockDim.x)
        if (sh_cnt[i]) atomicAdd(&counts[i], sh_cnt[i]);
}

// Load one work unit (4 triangles or one element); returns the runtime type
// (the element's own type for mixed meshes) and sets ok[w] for each valid
// element of the unit.  Invalid elements raise the status and are skipped.
template <int TYPE>
__device__ __forceinline__ int load_unit(const EmitParams& p, int64_t u, int32_t* nd, bool* ok) {
    if constexpr (TYPE == NN_TRI) {
        const int64_t e0 = u * 4;
        if (e0 + 4 <= p.n_elems) {
            const int4* c4 = reinterpret_cast<const int4*>(p.conn + e0 * 3);
            int4 a = __ldg(c4), b = __ldg(c4 + 1), c = __ldg(c4 + 2);
            nd[0] = a.x; nd[1] = a.y; nd[2] = a.z; nd[3] = a.w;
            nd[4] = b.x; nd[5] = b.y; nd[6] = b.z; nd[7] = b.w;
            nd[8] = c.x; nd[9] = c.y; nd[10] = c.z; nd[11] = c.w;
        } else {
#pragma unroll
            for (int q = 0; q < 12; ++q) nd[q] = (e0 * 3 + q < p.n_conn) ? __ldg(p.conn + e0 * 3 + q) : 0;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            bool v = e0 + w < p.n_elems;
#pragma unroll
            for (int i = 0; i < 3; ++i) v = v && nd[3 * w + i] >= 0 && (int64_t)nd[3 * w + i] < p.n_nodes;
            if (!v && e0 + w < p.n_elems) set_status(p.status, NN_ERR_NODE_RANGE);
            ok[w] = v;
        }
        return NN_TRI;
    } else if constexpr (TYPE == NN_MIXED) {
        const int t = __ldg(p.elem_type + u);
        const int64_t a = __ldg(p.elem_ptr + u), b = __ldg(p.elem_ptr + u + 1);
        if (t > NN_HEX || a < 0 || b > p.n_conn || b - a != npe_of(t)) {
            set_status(p.status, NN_ERR_ELEM_PTR);
            ok[0] = false;
            return NN_HEX;
        }
        const int npe = (int)(b - a);
        load_mixed_nodes(p.conn, a, npe, nd);
        bool v = true;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < npe) v = v && nd[q] >= 0 && (int64_t)nd[q] < p.n_nodes;
        if (!v) set_status(p.status, NN_ERR_NODE_RANGE);
        ok[0] = v;
        return t;
    } else {
        constexpr int NPE = ElemT<TYPE>::NPE;
        const int4* c4 = reinterpret_cast<const int4*>(p.conn) + (NPE / 4) * u;
        int4 a = __ldg(c4);
        nd[0] = a.x; nd[1] = a.y; nd[2] = a.z; nd[3] = a.w;
        if constexpr (NPE == 8) {
            int4 b = __ldg(c4 + 1);
            nd[4] = b.x; nd[5] = b.y; nd[6] = b.z; nd[7] = b.w;
        }
        bool v = true;
#pragma unroll
        for (int i = 0; i < NPE; ++i) v = v && nd[i] >= 0 && (int64_t)nd[i] < p.n_nodes;
        if (!v) set_status(p.status, NN_ERR_NODE_RANGE);
        ok[0] = v;
        return TYPE;
    }
}

// Partition pass.  A thread takes UPT consecutive work units and issues all
// their cursor atomics before writing any record, so it keeps 8-16 L2
// atomics in flight (the pass is bound by atomic latency, not bandwidth).
template <int TYPE>
struct PartShape {
    static constexpr int UNIT = TYPE == NN_TRI ? 4 : 1;
    static constexpr int NPE = TYPE == NN_MIXED ? 8 : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::NPE;
    static constexpr int UPT = (TYPE == NN_TRI) ? 1 : (NPE == 8 ? 2 : 3);  // units per thread per round
};

template <int TYPE, int RB, bool RANGED>
__global__ void __launch_bounds__(PART_THREADS, 2) k_part(EmitParams p) {
    using S = PartShape<TYPE>;
    constexpr int UNIT = S::UNIT, NPE = S::NPE, UPT = S::UPT, NI = NPE * UNIT;
    const RecFmt f = p.fmt;
    const uint32_t vmask = (1u << f.sb) - 1;
    const int64_t n_units = (p.n_elems + UNIT - 1) / UNIT;
    const int64_t u0 = n_units * blockIdx.x / gridDim.x, u1 = n_units * (blockIdx.x + 1) / gridDim.x;
    for (int64_t ub = u0 + (int64_t)threadIdx.x * UPT; ub < u1; ub += (int64_t)blockDim.x * UPT) {
        int32_t nd[UPT][NI];
        bool ok[UPT][UNIT];
        int t[UPT];
        uint32_t pos[UPT][NI];
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
#pragma unroll
            for (int w = 0; w < UNIT; ++w) ok[k][w] = false;
            t[k] = TYPE == NN_MIXED ? NN_HEX : TYPE;
            if (ub + k < u1) t[k] = load_unit<TYPE>(p, ub + k, nd[k], ok[k]);
        }
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
            const int npe = TYPE == NN_MIXED ? npe_of(t[k]) : NPE;
#pragma unroll
            for (int j = 0; j < NI; ++j) {
                const int w = j / NPE, i = j % NPE;
                pos[k][j] = 0xFFFFFFFFu;
                uint32_t vr;
                if (ok[k][w] && i < npe && node_in<RANGED>(p, nd[k][j], vr) && NN_IN(vr >> f.sb, p.n_buckets, p.status))
                    pos[k][j] = atomicAdd(&p.gcur[vr >> f.sb], 1u);
            }
        }
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
            const int tk = t[k];
#pragma unroll
            for (int j = 0; j < NI; ++j) {
                const int w = j / NPE, i = j % NPE;
                if (pos[k][j] >= p.rec_cap) continue;  // not an incidence, or overlapping invalid mixed elements
                const int32_t* e_nd = nd[k] + w * NPE;
                const int32_t v = e_nd[i];
                int nf = 0;
#pragma unroll
                for (int q = 0; q < NPE; ++q) nf |= (q < i) && (e_nd[q] == v);
                const int K = TYPE == NN_MIXED ? k_of(tk) : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::K;
                uint32_t vr;
                node_in<RANGED>(p, v, vr);
                Rec r{(uint64_t)(vr & vmask), 0};
                if (f.want & NN_WANT_ELEMS) {
                    rec_put(r, (uint64_t)nf, f.off_nf);
                    rec_put(r, (uint64_t)((ub + k) * UNIT + w), f.off_e);
                }
                if (f.want & NN_WANT_NODES) {
#pragma unroll
                    for (int s = 0; s < 3; ++s) {
                        if (s >= K) break;
                        const int32_t y = TYPE == NN_MIXED
                                              ? nbr_node(tk, e_nd, i, s)
                                              : e_nd[ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::nbr(i, s)];
                        rec_put(r, y == v ? 0ull : (uint64_t)(uint32_t)(y + 1), f.off_n + s * f.nb);
                    }
                }
                if constexpr (RB == 8) {
                    reinterpret_cast<uint64_t*>(p.rec)[pos[k][j]] = r.lo;
                } else {
                    reinterpret_cast<ulonglong2*>(p.rec)[pos[k][j]] = make_ulonglong2(r.lo, r.hi);
                }
            }
        }
    }
}

// ------------------------------------------------ tile-sorted partition
// A CTA builds the records of a tile of work units, ranks them by radix digit
// in shared memory, reserves one global range per digit present in the tile
// (one atomic per digit, not per record) and writes each digit's run
// contiguously, so global stores are coalesced runs instead of one scattered
// 16-byte store per record.

// Exclusive scan of hist[0..n) (any n) into dof, a contiguous chunk per thread;
// returns the total.  Ends with a barrier: any thread may read any dof entry.
__device__ __forceinline__ uint32_t tile_scan_n(const uint32_t* hist, uint32_t* dof, int n, uint64_t* sh) {
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    uint64_t x = 0;
    for (int i = lo; i < hi; ++i) x += hist[i];
    uint64_t total;
    uint64_t run = block_excl_scan(x, &total, sh);
    for (int i = lo; i < hi; ++i) {
        dof[i] = (uint32_t)run;
        run += hist[i];
    }
    __syncthreads();
    return (uint32_t)total;
}

// Exclusive scan of hist[0..n) (n <= blockDim.x) into dof; returns the total.
// Ends with a barrier: every thread may read any dof entry afterwards.
__device__ __forceinline__ uint32_t tile_scan(const uint32_t* hist, uint32_t* dof, int n, uint64_t* sh) {
    const uint64_t x = threadIdx.x < n ? hist[threadIdx.x] : 0;
    uint64_t total;
    const uint64_t ex = block_excl_scan(x, &total, sh);
    if (threadIdx.x < n) dof[threadIdx.x] = (uint32_t)ex;
    __syncthreads();
    return (uint32_t)total;
}

template <int TYPE>
struct SortShape {
    static constexpr int UNIT = TYPE == NN_TRI ? 4 : 1;
    static constexpr int NPE = TYPE == NN_MIXED ? 8 : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::NPE;
    static constexpr int UPT = (TYPE == NN_TET || TYPE == NN_QUAD) ? 2 : 1;
    static constexpr int NI = NPE * UNIT;
    static constexpr int RPT = NI * UPT;
    static constexpr int TILE = SORT_THREADS * RPT;
};

template <int TYPE>
__host__ __device__ constexpr size_t coarse_smem() {
    return (size_t)SortShape<TYPE>::TILE * 17 + 3 * 256 * 4;
}
// Records per thread of a fine-pass tile: 4, or 8 when a coarse region has
// at least 512 buckets (then a 1024-record tile has about two records per
// bucket, and its one cursor atomic per bucket present would come close to
// one per two records; with 256 buckets the larger tile measured slower).
constexpr int FINE_RPT_WIDE_DIGITS = 512;
__host__ __device__ constexpr int fine_rpt(int nd) { return nd >= FINE_RPT_WIDE_DIGITS ? 8 : 4; }
constexpr int FINE_DIGITS = 4096;  // buckets per coarse region: at most 256 x 4096 buckets in all
// shared memory of the fine pass for nd digits per coarse region and rb-byte
// records: two tile stages (bulk-copy targets, 16 bytes of slack for an odd
// 8-byte first record), the tile in digit order with its digits, three
// per-digit tables and the first work item of every coarse region
__host__ __device__ constexpr size_t fine_stage_bytes(int tile, int rb) { return (size_t)tile * rb + 16; }
__host__ __device__ constexpr size_t fine_smem(int nd, int rb) {
    return 2 * fine_stage_bytes(SORT_THREADS * fine_rpt(nd), rb) + (size_t)SORT_THREADS * fine_rpt(nd) * 18 +
           3 * (size_t)nd * 4 + 257 * 4;
}
constexpr size_t FINE_SMEM = fine_smem(FINE_DIGITS, 16);

// vr: the node's id relative to the build's first node
template <int TYPE>
__device__ __forceinline__ Rec make_rec(const RecFmt& f, const int32_t* e_nd, int i, int t, int64_t e, uint32_t vr) {
    constexpr int NPE = SortShape<TYPE>::NPE;
    const int32_t v = e_nd[i];
    int nf = 0;
#pragma unroll
    for (int q = 0; q < NPE; ++q) nf |= (q < i) && (e_nd[q] == v);
    const int K = TYPE == NN_MIXED ? k_of(t) : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::K;
    Rec r{(uint64_t)(vr & ((1u << f.sb) - 1)), 0};
    if (f.want & NN_WANT_ELEMS) {
        rec_put(r, (uint64_t)nf, f.off_nf);
        rec_put(r, (uint64_t)e, f.off_e);
    }
    if (f.want & NN_WANT_NODES) {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (s >= K) break;
            const int32_t y = TYPE == NN_MIXED ? nbr_node(t, e_nd, i, s)
                                               : e_nd[ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::nbr(i, s)];
            rec_put(r, y == v ? 0ull : (uint64_t)(uint32_t)(y + 1), f.off_n + s * f.nb);
        }
    }
    if (f.cshift > 0) rec_put(r, (uint64_t)((vr >> f.sb) & ((1u << f.cshift) - 1)), f.off_fb);
    return r;
}

template <int RB>
__device__ __forceinline__ void store_rec(uint8_t* base, uint64_t pos, const ulonglong2& r) {
    if constexpr (RB == 8) reinterpret_cast<uint64_t*>(base)[pos] = r.x;
    else reinterpret_cast<ulonglong2*>(base)[pos] = r;
}
template <int RB>
__device__ __forceinline__ ulonglong2 load_rec2(const uint8_t* base, uint64_t pos) {
    if constexpr (RB == 8) return make_ulonglong2(__ldg(reinterpret_cast<const unsigned long long*>(base) + pos), 0);
    else return __ldg(reinterpret_cast<const ulonglong2*>(base) + pos);
}

// First (or only) pass: records from the connectivity, radix digit = coarse
// region (two levels) or bucket (one level, at most 256 buckets).
template <int TYPE, int RB, bool RANGED>
__global__ void __launch_bounds__(SORT_THREADS) k_part_coarse(EmitParams p) {
    using S = SortShape<TYPE>;
    constexpr int UNIT = S::UNIT, NPE = S::NPE, UPT = S::UPT, NI = S::NI, TILE = S::TILE;
    extern __shared__ __align__(16) uint8_t sm[];
    ulonglong2* out = reinterpret_cast<ulonglong2*>(sm);
    uint8_t* odig = reinterpret_cast<uint8_t*>(out + TILE);
    uint32_t* hist = reinterpret_cast<uint32_t*>(odig + TILE);
    uint32_t* dof = hist + 256;
    uint32_t* gbase = dof + 256;
    __shared__ uint64_t sh_scan[34];
    const RecFmt f = p.fmt;
    const bool two = f.cshift > 0;
    const int dshift = f.sb + (two ? f.cshift : 0);
    uint32_t* cursor = two ? p.gcur_coarse : p.gcur;
    uint8_t* dst = two ? p.rec_tmp : p.rec;
    const int64_t n_units = (p.n_elems + UNIT - 1) / UNIT;
    const int64_t u0 = n_units * blockIdx.x / gridDim.x, u1 = n_units * (blockIdx.x + 1) / gridDim.x;
    for (int64_t tu = u0; tu < u1; tu += (int64_t)SORT_THREADS * UPT) {
        hist[threadIdx.x] = 0;
        __syncthreads();
        int32_t nd[UPT][NI];
        bool ok[UPT][UNIT];
        int t[UPT];
        uint16_t rk[UPT][NI];
        uint8_t dg[UPT][NI];
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
            const int64_t u = tu + (int64_t)threadIdx.x * UPT + k;
#pragma unroll
            for (int w = 0; w < UNIT; ++w) ok[k][w] = false;
            t[k] = TYPE == NN_MIXED ? NN_HEX : TYPE;
            if (u < u1) t[k] = load_unit<TYPE>(p, u, nd[k], ok[k]);
            const int npe = TYPE == NN_MIXED ? npe_of(t[k]) : NPE;
#pragma unroll
            for (int j = 0; j < NI; ++j) {
                const int w = j / NPE, i = j % NPE;
                dg[k][j] = 0;
                rk[k][j] = 0xFFFF;
                uint32_t vr;
                if (ok[k][w] && i < npe && node_in<RANGED>(p, nd[k][j], vr)) {
                    const uint32_t d = vr >> dshift;
                    dg[k][j] = (uint8_t)d;
                    rk[k][j] = (uint16_t)atomicAdd(&hist[d], 1u);
                }
            }
        }
        __syncthreads();
        const uint32_t n_tile = tile_scan(hist, dof, 256, sh_scan);
        if (hist[threadIdx.x]) gbase[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], hist[threadIdx.x]);
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
            const int64_t u = tu + (int64_t)threadIdx.x * UPT + k;
#pragma unroll
            for (int j = 0; j < NI; ++j) {
                if (rk[k][j] == 0xFFFF) continue;
                const int w = j / NPE, i = j % NPE;
                uint32_t vr;
                node_in<RANGED>(p, nd[k][j], vr);
                const Rec r = make_rec<TYPE>(f, nd[k] + w * NPE, i, t[k], u * UNIT + w, vr);
                const uint32_t q = dof[dg[k][j]] + rk[k][j];
                out[q] = make_ulonglong2(r.lo, r.hi);
                odig[q] = dg[k][j];
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < n_tile; q += SORT_THREADS) {
            const uint32_t d = odig[q];
            const uint64_t pos = (uint64_t)gbase[d] + (q - dof[d]);
            if (pos < p.rec_cap) store_rec<RB>(dst, pos, out[q]);
        }
        __syncthreads();
    }
}

// Second pass: one coarse region per work item group; radix digit = bucket
// inside the region (stored in the record by the first pass).  A CTA's work
// items are tiles of FINE_TILE records; each tile is brought into shared
// memory by a bulk asynchronous copy issued while the CTA still sorts and
// writes the tile before it (two stages, one mbarrier each, bounded waits),
// so the tile loads overlap the in-tile sort instead of stalling it.
template <int RB, int FINE_RPT>
__global__ void __launch_bounds__(SORT_THREADS) k_part_fine(EmitParams p, const uint32_t* bstart) {
    constexpr int FINE_TILE = SORT_THREADS * FINE_RPT;
    extern __shared__ __align__(16) uint8_t sm[];
    constexpr uint32_t SB = (uint32_t)fine_stage_bytes(FINE_TILE, RB);
    uint8_t* const stage = sm;  // [2][SB]
    ulonglong2* out = reinterpret_cast<ulonglong2*>(sm + 2 * SB);
    uint16_t* odig = reinterpret_cast<uint16_t*>(out + FINE_TILE);
    const RecFmt f = p.fmt;
    const int cs = f.cshift;
    const int nd_ = 1 << cs;  // digits (buckets) per coarse region, <= FINE_DIGITS
    uint32_t* hist = reinterpret_cast<uint32_t*>(odig + FINE_TILE);
    uint32_t* dof = hist + nd_;
    uint32_t* gbase = dof + nd_;
    uint32_t* tpre = gbase + nd_;  // [257] first tile of each coarse region
    __shared__ uint64_t sh_scan[34];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t sh_tile[2][4];  // per stage: region, first record, end, offset of record 0 in the stage
    __shared__ int32_t sh_lost;
    const int64_t B = p.n_buckets;
    const int R1 = (int)((B + (1ll << cs) - 1) >> cs);
    const int d0 = threadIdx.x;
    uint32_t my_tiles = 0;
    if (d0 < R1) {
        const uint32_t a = bstart[(int64_t)d0 << cs];
        const int64_t e_ = ((int64_t)d0 + 1) << cs;
        const uint32_t b = bstart[e_ < B ? e_ : B];
        my_tiles = (b - a + FINE_TILE - 1) / FINE_TILE;
    }
    {
        uint64_t total;
        const uint64_t ex = block_excl_scan(my_tiles, &total, sh_scan);
        if (d0 < R1) tpre[d0] = (uint32_t)ex;
        if (d0 == 0) tpre[R1] = (uint32_t)total;
    }
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0]);
        mbar_init(&mbar[1]);
        sh_lost = 0;
    }
    __syncthreads();
    const uint32_t W = tpre[R1];
    // One thread: locate work item wi and start the copy of its records
    // into stage st (stage st is free: its previous tile passed a barrier).
    auto issue = [&](int st, uint32_t wi) {
        int lo = 0, hi = R1;  // largest d with tpre[d] <= wi
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tpre[mid] <= wi) lo = mid;
            else hi = mid;
        }
        const int d = lo;
        const int64_t fb0 = (int64_t)d << cs;
        const int64_t fe = fb0 + (1ll << cs);
        const uint32_t ra = bstart[fb0], rb_ = bstart[fe < B ? fe : B];
        const uint32_t r0 = ra + (wi - tpre[d]) * FINE_TILE;
        const uint32_t r1 = min(r0 + (uint32_t)FINE_TILE, rb_);
        const uint32_t roff = RB == 8 ? (r0 & 1u) * 8u : 0u;
        sh_tile[st][0] = (uint32_t)d;
        sh_tile[st][1] = r0;
        sh_tile[st][2] = r1;
        sh_tile[st][3] = roff;
        if (r1 > r0) {
            // the coarse-sorted records are padded to 256 bytes, so the rounded-up tail stays inside them
            const uint32_t bytes = ((r1 - r0) * RB + roff + 15u) & ~15u;
            fence_async_smem();
            mbar_expect(&mbar[st], bytes);
            bulk_load(stage + st * SB, p.rec_tmp + (uint64_t)r0 * RB - roff, bytes, &mbar[st]);
        }
    };
    if (threadIdx.x == 0 && blockIdx.x < W) issue(0, blockIdx.x);
    uint32_t par[2] = {0u, 0u};  // parity of each stage's next copy
    int it = 0;
    for (uint32_t wi = blockIdx.x; wi < W; wi += gridDim.x, ++it) {
        const int st = it & 1;
        // the next tile of this CTA, into the other stage
        if (threadIdx.x == 0 && wi + gridDim.x < W) issue(st ^ 1, wi + gridDim.x);
        for (int i = threadIdx.x; i < nd_; i += SORT_THREADS) hist[i] = 0;
        // thread 0 issued this stage's copy and waits for it; the others wait
        // at the barrier, after which the stage's records and bounds are seen
        if (threadIdx.x == 0 && sh_tile[st][2] > sh_tile[st][1]) {
            if (!mbar_wait(&mbar[st], par[st])) sh_lost = 1;
            par[st] ^= 1u;
        }
        __syncthreads();
        if (sh_lost) {  // a copy that never completed (bounded wait): report and stop
            if (threadIdx.x == 0) set_status(p.status, NN_ERR_TIMEOUT);
            return;
        }
        const int d = (int)sh_tile[st][0];
        const int64_t fb0 = (int64_t)d << cs;
        const uint32_t n = sh_tile[st][2] - sh_tile[st][1];
        const uint8_t* const src = stage + st * SB + sh_tile[st][3];
        // a thread keeps its records' digits and ranks, and the records
        // themselves in registers when it holds four (else they are read
        // from the stage again when placed)
        auto rec_at = [&](uint32_t r) {
            if constexpr (RB == 8) return make_ulonglong2(reinterpret_cast<const unsigned long long*>(src)[r], 0);
            else return reinterpret_cast<const ulonglong2*>(src)[r];
        };
        constexpr int XR = FINE_RPT <= 4 ? FINE_RPT : 1;
        ulonglong2 x[XR];
        uint16_t rk[FINE_RPT];
        uint16_t dg[FINE_RPT];
#pragma unroll
        for (int k = 0; k < FINE_RPT; ++k) {
            const uint32_t r = threadIdx.x + k * SORT_THREADS;
            rk[k] = 0xFFFF;
            dg[k] = 0;
            if (r < n) {
                const ulonglong2 xr = rec_at(r);
                if constexpr (FINE_RPT <= 4) x[k] = xr;
                const Rec rr{xr.x, xr.y};
                dg[k] = (uint16_t)rec_get(rr, f.off_fb, cs);
            }
        }
#pragma unroll
        for (int k = 0; k < FINE_RPT; ++k)
            if (threadIdx.x + k * SORT_THREADS < n) rk[k] = (uint16_t)atomicAdd(&hist[dg[k]], 1u);
        __syncthreads();
        const uint32_t n_tile = tile_scan_n(hist, dof, nd_, sh_scan);
        for (int i = threadIdx.x; i < nd_; i += SORT_THREADS)
            if (hist[i] && NN_IN(fb0 + i, B, p.status)) gbase[i] = atomicAdd(&p.gcur[fb0 + i], hist[i]);
#pragma unroll
        for (int k = 0; k < FINE_RPT; ++k) {
            if (rk[k] == 0xFFFF) continue;
            const uint32_t q = dof[dg[k]] + rk[k];
            if constexpr (FINE_RPT <= 4) out[q] = x[k];
            else out[q] = rec_at(threadIdx.x + k * SORT_THREADS);
            odig[q] = dg[k];
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < n_tile; q += SORT_THREADS) {
            const uint32_t dd = odig[q];
            const uint64_t pos = (uint64_t)gbase[dd] + (q - dof[dd]);
            if (pos < p.rec_cap) store_rec<RB>(p.rec, pos, out[q]);
        }
        __syncthreads();
    }
}

// Per bucket b: total records = sum over CTAs of hist[c][b]; bucket starts by
// a lookback scan over tiles of buckets; each bucket's write cursor starts at
// its start.
__global__ void __launch_bounds__(OFFSETS_THREADS) k_offsets(OffsetsParams p) {
    __shared__ uint64_t sh_scan[33];
    __shared__ uint32_t sh_tile;
    __shared__ uint64_t sh_base;
    if (threadIdx.x == 0) sh_tile = atomicAdd(p.ticket, 1u);
    __syncthreads();
    const uint32_t tile = sh_tile;
    const int64_t B = p.hdr ? p.hdr->n_buckets : p.n_buckets;
    const int64_t b = (int64_t)tile * blockDim.x + threadIdx.x;
    uint64_t tot = 0, nf = 0;
    if (b < B) {
        for (int c = 0; c < p.n_cta; ++c) tot += p.hist[(int64_t)c * B + b];
        if (p.nfc) nf = p.nfc[b];
    }
    // records (low 31 bits) and repeated-node records (next 31) in one scan;
    // both totals stay below 2^31
    uint64_t agg;
    const uint64_t ex2 = block_excl_scan(tot | (nf << 31), &agg, sh_scan);
    const uint64_t ex = ex2 & 0x7fffffffull, ex_nf = ex2 >> 31;
    if (threadIdx.x < 32) {
        const uint64_t base = warp_lookback(p.lb_state, tile, agg, p.status);
        if (threadIdx.x == 0) sh_base = base;
    }
    __syncthreads();
    if (b < B) {
        const uint64_t base = sh_base & 0x7fffffffull, base_nf = sh_base >> 31;
        const uint64_t run = base + ex;
        p.bstart[b] = (uint32_t)min(run, p.rec_cap);
        if (p.estart) {
            const uint64_t erun = run - (base_nf + ex_nf);
            p.estart[b] = (uint32_t)min(erun, p.rec_cap);
            if (b == B - 1) p.estart[B] = (uint32_t)min(erun + tot - nf, p.rec_cap);
        }
        p.gcur[b] = (uint32_t)min(run, p.rec_cap);
        if (p.cshift > 0 && (b & ((1ll << p.cshift) - 1)) == 0) p.gcur_coarse[b >> p.cshift] = (uint32_t)min(run, p.rec_cap);
        if (b == B - 1) {
            p.bstart[B] = (uint32_t)min(run + tot, p.rec_cap);
            // more records than the record array holds: the record count the
            // workspace was planned for was wrong (a chunk planned from stale
            // counts); the partition stops at the array's end
            if (run + tot > p.rec_cap) set_status(p.status, NN_ERR_WORKSPACE);
        }
    }
}

template <int TYPE>
cudaError_t hist_t(const EmitParams& p, size_t smem, cudaStream_t s) {
    if (ranged(p)) k_hist<TYPE, true><<<p.n_cta, EMIT_THREADS, smem, s>>>(p);
    else k_hist<TYPE, false><<<p.n_cta, EMIT_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}
template <int TYPE, bool RANGED>
void part_r(const EmitParams& p, cudaStream_t s) {
    if (p.fmt.rb == 8) k_part<TYPE, 8, RANGED><<<p.n_cta_part, PART_THREADS, 0, s>>>(p);
    else k_part<TYPE, 16, RANGED><<<p.n_cta_part, PART_THREADS, 0, s>>>(p);
}
template <int TYPE>
cudaError_t part_t(const EmitParams& p, cudaStream_t s) {
    if (ranged(p)) part_r<TYPE, true>(p, s);
    else part_r<TYPE, false>(p, s);
    return cudaGetLastError();
}

template <int TYPE>
cudaError_t set_sorted_smem() {
    const int b = (int)coarse_smem<TYPE>();
    cudaError_t e = cudaFuncSetAttribute(k_part_coarse<TYPE, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_coarse<TYPE, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_coarse<TYPE, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_coarse<TYPE, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

template <int TYPE>
cudaError_t set_emit_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_hist<TYPE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_hist<TYPE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

}  // namespace

cudaError_t launch_hist(const EmitParams& p, size_t smem, cudaStream_t s) {
    switch (p.type) {
        case NN_TRI: return hist_t<NN_TRI>(p, smem, s);
        case NN_QUAD: return hist_t<NN_QUAD>(p, smem, s);
        case NN_TET: return hist_t<NN_TET>(p, smem, s);
        case NN_HEX: return hist_t<NN_HEX>(p, smem, s);
        default: return hist_t<NN_MIXED>(p, smem, s);
    }
}

cudaError_t launch_part(const EmitParams& p, cudaStream_t s) {
    switch (p.type) {
        case NN_TRI: return part_t<NN_TRI>(p, s);
        case NN_QUAD: return part_t<NN_QUAD>(p, s);
        case NN_TET: return part_t<NN_TET>(p, s);
        case NN_HEX: return part_t<NN_HEX>(p, s);
        default: return part_t<NN_MIXED>(p, s);
    }
}

template <int TYPE, bool RANGED>
void coarse_r(const EmitParams& p, cudaStream_t s) {
    const size_t smem = coarse_smem<TYPE>();
    if (p.fmt.rb == 8) k_part_coarse<TYPE, 8, RANGED><<<p.n_cta_part, SORT_THREADS, smem, s>>>(p);
    else k_part_coarse<TYPE, 16, RANGED><<<p.n_cta_part, SORT_THREADS, smem, s>>>(p);
}

template <int TYPE>
cudaError_t part_coarse_t(const EmitParams& p, cudaStream_t s) {
    if (ranged(p)) coarse_r<TYPE, true>(p, s);
    else coarse_r<TYPE, false>(p, s);
    return cudaGetLastError();
}

cudaError_t launch_part_coarse(const EmitParams& p, cudaStream_t s) {
    switch (p.type) {
        case NN_TRI: return part_coarse_t<NN_TRI>(p, s);
        case NN_QUAD: return part_coarse_t<NN_QUAD>(p, s);
        case NN_TET: return part_coarse_t<NN_TET>(p, s);
        case NN_HEX: return part_coarse_t<NN_HEX>(p, s);
        default: return part_coarse_t<NN_MIXED>(p, s);
    }
}

// One CTA per resident slot (the SMs times the CTAs its shared memory
// allows per SM): each CTA works through its tiles with the copies in flight.
template <int RB, int RPT>
cudaError_t fine_t(const EmitParams& p, const uint32_t* bstart, int sms, cudaStream_t s) {
    const size_t fs = fine_smem(1 << p.fmt.cshift, RB);
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_part_fine<RB, RPT>, SORT_THREADS, fs);
    if (e != cudaSuccess) return e;
    k_part_fine<RB, RPT><<<std::max(1, sms * std::max(occ, 1)), SORT_THREADS, fs, s>>>(p, bstart);
    return cudaGetLastError();
}

cudaError_t launch_part_fine(const EmitParams& p, const uint32_t* bstart, int sms, cudaStream_t s) {
    if (p.fmt.cshift <= 0) return cudaSuccess;
    const bool wide = fine_rpt(1 << p.fmt.cshift) == 8;
    if (p.fmt.rb == 8) return wide ? fine_t<8, 8>(p, bstart, sms, s) : fine_t<8, 4>(p, bstart, sms, s);
    return wide ? fine_t<16, 8>(p, bstart, sms, s) : fine_t<16, 4>(p, bstart, sms, s);
}

cudaError_t launch_part_sorted(const EmitParams& p, const uint32_t* bstart, int sms, cudaStream_t s) {
    cudaError_t e = launch_part_coarse(p, s);
    if (e != cudaSuccess) return e;
    return launch_part_fine(p, bstart, sms, s);
}

template <int TYPE>
cudaError_t slab_count_t(const EmitParams& p, int shift, int n_slabs, uint32_t* counts, cudaStream_t s) {
    k_slab_count<TYPE><<<p.n_cta, EMIT_THREADS, 0, s>>>(p, shift, n_slabs, counts);
    return cudaGetLastError();
}

cudaError_t launch_slab_count(const EmitParams& p, int shift, int n_slabs, uint32_t* counts, cudaStream_t s) {
    if (n_slabs < 1 || n_slabs > NN_CHUNK_SLABS_MAX) return cudaErrorInvalidValue;
    switch (p.type) {
        case NN_TRI: return slab_count_t<NN_TRI>(p, shift, n_slabs, counts, s);
        case NN_QUAD: return slab_count_t<NN_QUAD>(p, shift, n_slabs, counts, s);
        case NN_TET: return slab_count_t<NN_TET>(p, shift, n_slabs, counts, s);
        case NN_HEX: return slab_count_t<NN_HEX>(p, shift, n_slabs, counts, s);
        default: return slab_count_t<NN_MIXED>(p, shift, n_slabs, counts, s);
    }
}

cudaError_t launch_offsets(const OffsetsParams& p, cudaStream_t s) {
    const int64_t tiles = (p.n_buckets + OFFSETS_THREADS - 1) / OFFSETS_THREADS;
    if (tiles == 0) return cudaSuccess;
    k_offsets<<<(unsigned)tiles, OFFSETS_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t set_emit_smem_all(size_t bytes) {
    cudaError_t e = set_sorted_smem<NN_TRI>();
    if (e == cudaSuccess) e = set_sorted_smem<NN_QUAD>();
    if (e == cudaSuccess) e = set_sorted_smem<NN_TET>();
    if (e == cudaSuccess) e = set_sorted_smem<NN_HEX>();
    if (e == cudaSuccess) e = set_sorted_smem<NN_MIXED>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_fine<8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FINE_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_fine<8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FINE_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_fine<16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FINE_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_fine<16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FINE_SMEM);
    if (e == cudaSuccess) e = set_emit_smem<NN_TRI>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_QUAD>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_TET>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_HEX>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_MIXED>(bytes);
    return e;
}

}  // namespace nn
