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
#include "nn_device.cuh"

namespace nn {

namespace {

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
                int li = TYPE == NN_MIXED ? nbr_of(t, i, s) : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::nbr(i, s);
                y = nd[li];
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
#pragma unroll
            for (int q = 0; q < 8; ++q) nd[q] = q < b - a ? __ldg(p.conn + a + q) : 0;
            visit_elem<NN_MIXED>(nd, u, p.n_nodes, p.status, t, f);
        }
    }
}

template <int TYPE>
__global__ void __launch_bounds__(EMIT_THREADS) k_hist(EmitParams p) {
    extern __shared__ uint32_t sh_hist[];
    const int64_t B = p.n_buckets;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) sh_hist[b] = 0;
    __syncthreads();
    const int sb = p.fmt.sb;
    walk_cta<TYPE>(p, [&](int32_t v, int, int64_t, int32_t, int32_t, int32_t) {
        atomicAdd(&sh_hist[v >> sb], 1u);
    });
    __syncthreads();
    uint32_t* row = p.hist + (int64_t)blockIdx.x * B;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) row[b] = sh_hist[b];
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
        bool v = true;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            nd[q] = q < npe ? __ldg(p.conn + a + q) : 0;
            if (q < npe) v = v && nd[q] >= 0 && (int64_t)nd[q] < p.n_nodes;
        }
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

template <int TYPE, int RB>
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
                if (ok[k][w] && i < npe) pos[k][j] = atomicAdd(&p.gcur[(uint32_t)nd[k][j] >> f.sb], 1u);
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
                Rec r{(uint64_t)((uint32_t)v & vmask), 0};
                if (f.want & NN_WANT_ELEMS) {
                    rec_put(r, (uint64_t)nf, f.off_nf);
                    rec_put(r, (uint64_t)((ub + k) * UNIT + w), f.off_e);
                }
                if (f.want & NN_WANT_NODES) {
#pragma unroll
                    for (int s = 0; s < 3; ++s) {
                        if (s >= K) break;
                        const int li = TYPE == NN_MIXED ? nbr_of(tk, i, s)
                                                        : ElemT<(TYPE == NN_MIXED ? NN_HEX : TYPE)>::nbr(i, s);
                        const int32_t y = e_nd[li];
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
    uint64_t tot = 0;
    if (b < B)
        for (int c = 0; c < p.n_cta; ++c) tot += p.hist[(int64_t)c * B + b];
    uint64_t agg;
    uint64_t ex = block_excl_scan(tot, &agg, sh_scan);
    if (threadIdx.x < 32) {
        const uint64_t base = warp_lookback(p.lb_state, tile, agg, p.status);
        if (threadIdx.x == 0) sh_base = base;
    }
    __syncthreads();
    if (b < B) {
        const uint64_t run = sh_base + ex;
        p.bstart[b] = (uint32_t)min(run, p.rec_cap);
        p.gcur[b] = (uint32_t)min(run, p.rec_cap);
        if (b == B - 1) p.bstart[B] = (uint32_t)min(run + tot, p.rec_cap);
    }
}

template <int TYPE>
cudaError_t hist_t(const EmitParams& p, size_t smem, cudaStream_t s) {
    k_hist<TYPE><<<p.n_cta, EMIT_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}
template <int TYPE>
cudaError_t part_t(const EmitParams& p, cudaStream_t s) {
    if (p.fmt.rb == 8) k_part<TYPE, 8><<<p.n_cta_part, PART_THREADS, 0, s>>>(p);
    else k_part<TYPE, 16><<<p.n_cta_part, PART_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

template <int TYPE>
cudaError_t set_emit_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_hist<TYPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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

cudaError_t launch_offsets(const OffsetsParams& p, cudaStream_t s) {
    const int64_t tiles = (p.n_buckets + OFFSETS_THREADS - 1) / OFFSETS_THREADS;
    if (tiles == 0) return cudaSuccess;
    k_offsets<<<(unsigned)tiles, OFFSETS_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t set_emit_smem_all(size_t bytes) {
    cudaError_t e = set_emit_smem<NN_TRI>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_QUAD>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_TET>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_HEX>(bytes);
    if (e == cudaSuccess) e = set_emit_smem<NN_MIXED>(bytes);
    return e;
}

}  // namespace nn
