// Element walk kernels: bucket histogram, bucket offsets, partition.
//
// The paper's GPU recipe (Sec. 2.2.1) has one thread per triangle emit its
// integer pairs and then sorts them by key.  Here the pairs of one node never
// leave a packed per-incidence record (node, element, the node's edge
// neighbours in that element), and records are partitioned by node range
// ("bucket") instead of sorted: a histogram pass and a partition pass over
// the connectivity, each CTA owning a fixed slice of elements and keeping its
// per-bucket counters in shared memory, so the only random global traffic is
// one vector store per incidence into a bucket's write head.
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
    const int64_t u0 = n_units * blockIdx.x / p.n_cta, u1 = n_units * (blockIdx.x + 1) / p.n_cta;
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

template <int TYPE, int RB>
__global__ void __launch_bounds__(EMIT_THREADS) k_part(EmitParams p) {
    extern __shared__ uint32_t sh_cur[];
    const int64_t B = p.n_buckets;
    const uint32_t* row = p.hist + (int64_t)blockIdx.x * B;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) sh_cur[b] = row[b];
    __syncthreads();
    const RecFmt f = p.fmt;
    const uint32_t vmask = (1u << f.sb) - 1;
    walk_cta<TYPE>(p, [&](int32_t v, int nf, int64_t e, int32_t x0, int32_t x1, int32_t x2) {
        const uint32_t pos = atomicAdd(&sh_cur[v >> f.sb], 1u);
        Rec r{(uint64_t)((uint32_t)v & vmask), 0};
        if (f.want & NN_WANT_ELEMS) {
            rec_put(r, (uint64_t)nf, f.off_nf);
            rec_put(r, (uint64_t)e, f.off_e);
        }
        if (f.want & NN_WANT_NODES) {
            rec_put(r, (uint64_t)(uint32_t)(x0 + 1), f.off_n);
            rec_put(r, (uint64_t)(uint32_t)(x1 + 1), f.off_n + f.nb);
            if (f.k > 2) rec_put(r, (uint64_t)(uint32_t)(x2 + 1), f.off_n + 2 * f.nb);
        }
        if (pos >= p.rec_cap) return;  // only with overlapping (invalid) mixed elements
        if constexpr (RB == 8) {
            reinterpret_cast<uint64_t*>(p.rec)[pos] = r.lo;
        } else {
            reinterpret_cast<ulonglong2*>(p.rec)[pos] = make_ulonglong2(r.lo, r.hi);
        }
    });
}

// Per bucket b: total records = sum over CTAs of hist[c][b]; bucket starts by
// a lookback scan over tiles of buckets; then each CTA's write offset inside
// the bucket (CTA order, so a bucket's records are grouped by element slice).
__global__ void __launch_bounds__(OFFSETS_THREADS) k_offsets(OffsetsParams p) {
    __shared__ uint64_t sh_scan[33];
    __shared__ uint32_t sh_tile;
    __shared__ uint64_t sh_base;
    if (threadIdx.x == 0) sh_tile = atomicAdd(p.ticket, 1u);
    __syncthreads();
    const uint32_t tile = sh_tile;
    const int64_t B = p.n_buckets;
    const int64_t b = (int64_t)tile * blockDim.x + threadIdx.x;
    uint64_t tot = 0;
    if (b < B)
        for (int c = 0; c < p.n_cta; ++c) tot += p.hist[(int64_t)c * B + b];
    uint64_t agg;
    uint64_t ex = block_excl_scan(tot, &agg, sh_scan);
    if (threadIdx.x == 0) sh_base = lookback(p.lb_state, tile, agg, p.status);
    __syncthreads();
    if (b < B) {
        uint64_t run = sh_base + ex;
        p.bstart[b] = (uint32_t)min(run, p.rec_cap);
        for (int c = 0; c < p.n_cta; ++c) {
            uint32_t t = p.hist[(int64_t)c * B + b];
            p.hist[(int64_t)c * B + b] = (uint32_t)min(run, p.rec_cap);
            run += t;
        }
        if (b == B - 1) p.bstart[B] = (uint32_t)min(run, p.rec_cap);
    }
}

template <int TYPE>
cudaError_t hist_t(const EmitParams& p, size_t smem, cudaStream_t s) {
    k_hist<TYPE><<<p.n_cta, EMIT_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}
template <int TYPE>
cudaError_t part_t(const EmitParams& p, size_t smem, cudaStream_t s) {
    if (p.fmt.rb == 8) k_part<TYPE, 8><<<p.n_cta, EMIT_THREADS, smem, s>>>(p);
    else k_part<TYPE, 16><<<p.n_cta, EMIT_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

template <int TYPE>
cudaError_t set_emit_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_hist<TYPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part<TYPE, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part<TYPE, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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

cudaError_t launch_part(const EmitParams& p, size_t smem, cudaStream_t s) {
    switch (p.type) {
        case NN_TRI: return part_t<NN_TRI>(p, smem, s);
        case NN_QUAD: return part_t<NN_QUAD>(p, smem, s);
        case NN_TET: return part_t<NN_TET>(p, smem, s);
        case NN_HEX: return part_t<NN_HEX>(p, smem, s);
        default: return part_t<NN_MIXED>(p, smem, s);
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
