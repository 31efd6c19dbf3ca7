// Bucket pass: builds the rows of one node range per CTA from its records.
//
// For the 2^sb nodes of a bucket the CTA counts, per node, the element
// entries and the neighbour candidates of its records; lays out one element
// list, one open-addressing hash table (one slot more than the node has
// candidates, so it never fills) and one list of distinct neighbours per node
// in shared memory; inserts the candidates (a repeated neighbour -- an edge
// shared by several elements -- hits its own slot and is dropped, a new one is
// appended to the node's list); sorts each row by ranking; and writes
// row_ptr and col of both CSRs at offsets found by a lookback scan over the
// buckets, which are processed in node order.  A bucket whose lists and
// tables do not fit shared memory keeps its tables in a global spill area
// and its element lists directly in the output.
//
// Rows are sets in ascending order: the paper's pipeline (Sec. 2.2.1) sorts
// pairs by key only and counts pairs per key, which lists an edge shared by
// two elements twice; one-ring neighbours are a set (Sec. 1), so repeated
// neighbours are dropped and each row is sorted.
#include "nn_device.cuh"

namespace nn {

namespace {

constexpr int BUCKET_THREADS = 512;  // default block size (256 is the other choice)
constexpr int LONG_ROW = 48;  // rows longer than this are sorted by the whole block
constexpr int UNROLL = 2;     // records loaded per thread before they are used
constexpr uint32_t RANK_MAX = 64;  // rows up to this length are sorted by ranking

template <int RB>
__device__ __forceinline__ Rec load_rec(const uint8_t* base, uint32_t r) {
    Rec x;
    if constexpr (RB == 8) {
        x.lo = __ldg(reinterpret_cast<const unsigned long long*>(base) + r);
        x.hi = 0;
    } else {
        ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2*>(base) + r);
        x.lo = w.x;
        x.hi = w.y;
    }
    return x;
}

// Insert x into the open-addressing table tab[0..T); true if x was new.  T is
// larger than the number of distinct values ever inserted (T = candidates + 1),
// so a free slot always exists; the probe count is still bounded and an
// overrun reports NN_ERR_WORKSPACE.  The start slot is the high word of
// hash(x) * T (a multiply-shift range reduction onto [0, T)).
__device__ __forceinline__ bool tab_insert(uint32_t* tab, uint32_t T, uint32_t x, int32_t* status) {
    uint32_t h = __umulhi(x * 0x9E3779B1u, T);
    for (uint32_t probes = 0; probes < T; ++probes) {
        uint32_t cur = *reinterpret_cast<volatile uint32_t*>(&tab[h]);
        if (cur == x) return false;
        if (cur == EMPTY) {
            uint32_t old = atomicCAS(&tab[h], EMPTY, x);
            if (old == EMPTY) return true;
            if (old == x) return false;
        }
        h = h + 1 == T ? 0 : h + 1;
    }
    set_status(status, NN_ERR_WORKSPACE);
    return false;
}

__device__ __forceinline__ uint32_t table_size(uint32_t c) { return c == 0 ? 0 : (c < 0xFFFFFFFEu ? c + 1 : c); }

struct BucketOut {
    int64_t n_nodes, first;
    bool last;
    int64_t* rp_n; int32_t* col_n; int64_t cap_n;
    int64_t* rp_e; int32_t* col_e; int64_t cap_e;
    int32_t* status;
};

template <int RB, int K, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_bucket(BucketParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ BucketOut sh_out;
    const bool batched = p.batch.hdr != nullptr;
    const RecFmt f = batched ? p.batch.hdr->fmt : p.fmt;
    const int64_t n_buckets = batched ? p.batch.hdr->n_buckets : p.n_buckets;
    const int n_meshes = batched ? p.batch.hdr->n_meshes : 1;
    const int NB = 1 << f.sb;
    const uint32_t vmask = (uint32_t)NB - 1;
    uint64_t* cnt = reinterpret_cast<uint64_t*>(smem);  // [NB] counts / scan scratch
    uint32_t* eoff = reinterpret_cast<uint32_t*>(cnt + NB);
    uint32_t* toff = eoff + NB;
    uint32_t* tsz = toff + NB;
    uint32_t* ucnt = tsz + NB;
    uint32_t* aux = ucnt + NB;                            // element cursor, then row offsets
    uint64_t* sh_scan = reinterpret_cast<uint64_t*>(aux + NB);  // 34 words
    uint64_t* misc = sh_scan + 34;                              // 8 words
    uint32_t* area = reinterpret_cast<uint32_t*>(misc + 8);
    const bool want_n = f.want & NN_WANT_NODES, want_e = f.want & NN_WANT_ELEMS;
    const int tid = threadIdx.x, BS = blockDim.x;

    if (tid == 0) misc[0] = atomicAdd(p.ticket, 1u);
    __syncthreads();
    int64_t b_next = (int64_t)misc[0];
    __syncthreads();
    for (;;) {
        const int64_t b = b_next;
        if (b >= n_buckets) break;
        // take the next bucket now and start pulling its records into L2
        if (tid == 0) {
            const uint32_t nx = atomicAdd(p.ticket, 1u);
            misc[5] = nx;
            if (nx < n_buckets) {
                uint64_t lo = (uint64_t)p.bstart[nx] * RB, hi = (uint64_t)p.bstart[nx + 1] * RB;
                lo &= ~15ull;
                hi = (hi + 15) & ~15ull;  // the record array is padded to 256 bytes
                for (uint64_t a = lo; a < hi; a += 32768) {
                    const uint32_t n = (uint32_t)(hi - a < 32768ull ? hi - a : 32768ull);
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p.rec + a), "r"(n) : "memory");
                }
            }
        }
        // the mesh this bucket belongs to (the only one unless batched); its
        // output pointers stay in shared memory until they are needed
        if (tid == 0) {
            BucketOut o{p.n_nodes, 0, b == n_buckets - 1, p.rp_n, p.col_n, p.cap_n, p.rp_e, p.col_e, p.cap_e, p.status};
            if (batched) {
                int lo = 0, hi = n_meshes;  // largest m with bucket_off[m] <= b
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (p.batch.bucket_off[mid] <= b) lo = mid;
                    else hi = mid;
                }
                const BatchMesh& M = p.batch.meshes[lo];
                o = BucketOut{M.n_nodes, p.batch.bucket_off[lo], b == p.batch.bucket_off[lo + 1] - 1, M.rp_n, M.col_n,
                              M.cap_n, M.rp_e, M.col_e, M.cap_e, M.status};
                if (*p.batch_err) set_status(o.status, *p.batch_err);
            }
            sh_out = o;
        }
        __syncthreads();
        const int64_t N = sh_out.n_nodes, first = sh_out.first;
        int32_t* const status = sh_out.status;
        const int64_t v0 = (b - first) << f.sb;
        const int nb = (int)(N - v0 < (int64_t)NB ? N - v0 : (int64_t)NB);
        const uint32_t r0 = p.bstart[b], r1 = p.bstart[b + 1];

        // counts per node: element entries (high word) and candidates (low word)
        for (int l = tid; l < NB; l += BS) cnt[l] = 0;
        __syncthreads();
        for (uint32_t r = r0 + tid; r < r1; r += UNROLL * BS) {
            Rec xs[UNROLL];
#pragma unroll
            for (int q = 0; q < UNROLL; ++q)
                if (r + q * BS < r1) xs[q] = load_rec<RB>(p.rec, r + q * BS);
#pragma unroll
            for (int q = 0; q < UNROLL; ++q) {
                if (r + q * BS >= r1) break;
                const Rec& x = xs[q];
                const uint32_t vloc = (uint32_t)x.lo & vmask;
                uint64_t inc = 0;
                if (want_e && !rec_get(x, f.off_nf, 1)) inc += 1ull << 32;
                if (want_n) {
#pragma unroll
                    for (int s = 0; s < K; ++s) inc += rec_get(x, f.off_n + s * f.nb, f.nb) != 0;
                }
                if (inc) atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[vloc]), (unsigned long long)inc);
            }
        }
        __syncthreads();
        // element offsets
        for (int l = tid; l < NB; l += BS) {
            const uint64_t c = cnt[l];
            tsz[l] = table_size((uint32_t)c);
            ucnt[l] = 0;
            aux[l] = 0;
            cnt[l] = c >> 32;
        }
        __syncthreads();
        const uint64_t Eb = smem_array_excl_scan(cnt, NB, sh_scan);
        for (int l = tid; l < NB; l += BS) {
            eoff[l] = (uint32_t)cnt[l];
            cnt[l] = tsz[l];
        }
        __syncthreads();
        const uint64_t Tb = smem_array_excl_scan(cnt, NB, sh_scan);
        for (int l = tid; l < NB; l += BS) toff[l] = (uint32_t)cnt[l];
        const bool fast_b = Eb + 2 * Tb <= p.area_words;  // element lists, tables, unique lists
        if (want_e && tid == 0) lb_publish(p.lb_e, b, Eb, first);
        if (tid < 32) {  // large buckets write element lists straight to the output: need the offset now
            const uint64_t ge = (want_e && !fast_b) ? lb_resolve(p.lb_e, b, Eb, status, first) : 0;
            if (tid == 0) misc[1] = ge;
        }
        if (tid == 0) {
            const bool fast = fast_b;  // else: tables in the spill area, rows gathered from them
            uint64_t spill_off = 0;
            bool tab_ok = true;
            if (!fast && want_n && Tb > 0) {
                spill_off = atomicAdd(p.spill_cursor, (unsigned long long)Tb);
                if (spill_off + Tb > p.spill_words || Tb >= 0xFFFFFFFFull) {
                    tab_ok = false;
                    set_status(status, NN_ERR_WORKSPACE);
                }
            }
            misc[2] = spill_off;
            misc[4] = (fast ? 1 : 0) | (tab_ok ? 2 : 0);
        }
        __syncthreads();
        uint64_t Ge = misc[1];
        const bool fast = misc[4] & 1, tab_ok = (misc[4] & 2) && want_n;
        bool e_ok = want_e && Ge + Eb <= (uint64_t)sh_out.cap_e;  // final for large buckets, rechecked below
        uint32_t* elist = fast ? area : reinterpret_cast<uint32_t*>(sh_out.col_e) + Ge;
        const bool e_write = want_e && (fast || e_ok);
        uint32_t* tab = fast ? area + Eb : p.spill + misc[2];
        uint32_t* ulist = fast ? area + Eb + Tb : nullptr;  // distinct neighbours of node l at ulist[toff[l]..]
        if (tab_ok)
            for (uint64_t i = tid; i < Tb; i += BS) tab[i] = EMPTY;
        __syncthreads();

        // second pass: element lists and neighbour tables
        for (uint32_t r = r0 + tid; r < r1; r += UNROLL * BS) {
          Rec xs[UNROLL];
#pragma unroll
          for (int q = 0; q < UNROLL; ++q)
              if (r + q * BS < r1) xs[q] = load_rec<RB>(p.rec, r + q * BS);
#pragma unroll
          for (int q = 0; q < UNROLL; ++q) {
            if (r + q * BS >= r1) break;
            const Rec& x = xs[q];
            const uint32_t vloc = (uint32_t)x.lo & vmask;
            if (e_write && !rec_get(x, f.off_nf, 1)) {
                const uint32_t q = atomicAdd(&aux[vloc], 1u);
                elist[eoff[vloc] + q] = rec_get(x, f.off_e, f.eb);
            }
            if (tab_ok) {
                const uint32_t T = tsz[vloc], o = toff[vloc];
                uint32_t* t = tab + o;
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    const uint32_t y = rec_get(x, f.off_n + s * f.nb, f.nb);
                    if (y && tab_insert(t, T, y - 1, status)) {
                        const uint32_t pos = atomicAdd(&ucnt[vloc], 1u);
                        if (ulist) ulist[o + pos] = y - 1;
                    }
                }
            }
          }
        }
        __syncthreads();
        for (int l = tid; l < NB; l += BS) cnt[l] = ucnt[l];
        __syncthreads();
        const uint64_t Ub = smem_array_excl_scan(cnt, NB, sh_scan);
        for (int l = tid; l < NB; l += BS) aux[l] = (uint32_t)cnt[l];
        if (want_n && tid == 0) lb_publish(p.lb_n, b, Ub, first);
        __syncthreads();  // row offsets (aux) are read across threads below
        uint64_t Gn = 0;
        bool n_ok = false;
        // output offsets of this bucket: resolved now for large buckets (they
        // write straight to the output), at the very end for the others, when
        // the predecessors have long published
        auto resolve = [&](bool elem_too) {
            if (tid < 32) {
                const uint64_t gn = want_n ? lb_resolve(p.lb_n, b, Ub, status, first) : 0;
                const uint64_t ge = (want_e && elem_too) ? lb_resolve(p.lb_e, b, Eb, status, first) : misc[1];
                if (tid == 0) {
                    misc[3] = gn;
                    misc[1] = ge;
                    if (want_n && gn + Ub > (uint64_t)sh_out.cap_n) set_status(status, NN_ERR_CAPACITY);
                    if (want_e && ge + Eb > (uint64_t)sh_out.cap_e) set_status(status, NN_ERR_CAPACITY);
                }
            }
            __syncthreads();
            Gn = misc[3];
            Ge = misc[1];
            n_ok = tab_ok && Gn + Ub <= (uint64_t)sh_out.cap_n;
            e_ok = want_e && Ge + Eb <= (uint64_t)sh_out.cap_e;
            for (int l = tid; l < nb; l += BS) {
                if (want_n) sh_out.rp_n[v0 + l] = (int64_t)(Gn + aux[l]);
                if (want_e) sh_out.rp_e[v0 + l] = (int64_t)(Ge + eoff[l]);
            }
            if (sh_out.last && tid == 0) {
                if (want_n) sh_out.rp_n[N] = (int64_t)(Gn + Ub);
                if (want_e) sh_out.rp_e[N] = (int64_t)(Ge + Eb);
            }
        };

        // rows: each node's distinct neighbours are in its unique list (fast
        // buckets); rank-sort every row, four threads per node
        uint32_t* stage = (fast && Eb + 2 * Tb + Ub <= p.area_words) ? area + Eb + 2 * Tb : nullptr;
        uint32_t* sorted = nullptr;
        if (fast) {
            if (Ub + Eb <= Tb) sorted = tab;  // the tables are dead after the second pass
            else if (Eb + 2 * Tb + Ub + Eb <= p.area_words) sorted = area + Eb + 2 * Tb;
        }
        if (sorted) {
            int has_long = 0;
            uint32_t* sorted_e = sorted + Ub;
            for (int idx = tid; idx < NB * 4; idx += BS) {
                const int l = idx >> 2, part = idx & 3;
                if (tab_ok) {
                    const uint32_t U = ucnt[l], a = toff[l], o = aux[l];
                    if (U > RANK_MAX) has_long = 1;
                    for (uint32_t j = part; j < U; j += 4) {
                        const uint32_t x = ulist[a + j];
                        uint32_t rank = j;
                        if (U <= RANK_MAX) {
                            rank = 0;
                            for (uint32_t i = 0; i < U; ++i) rank += ulist[a + i] < x;
                        }
                        sorted[o + rank] = x;
                    }
                }
                if (want_e) {
                    const uint32_t a = eoff[l], E = (l + 1 < NB ? eoff[l + 1] : (uint32_t)Eb) - a;
                    if (E > RANK_MAX) has_long = 1;
                    for (uint32_t j = part; j < E; j += 4) {
                        const uint32_t x = elist[a + j];
                        uint32_t rank = j;
                        if (E <= RANK_MAX) {
                            rank = 0;
                            for (uint32_t i = 0; i < E; ++i) rank += elist[a + i] < x;
                        }
                        sorted_e[a + rank] = x;
                    }
                }
            }
            has_long = __syncthreads_or(has_long);
            for (int l = 0; has_long && l < NB; ++l) {  // uniform loop: long rows, whole block
                if (tab_ok && ucnt[l] > RANK_MAX) block_bitonic_sort(sorted + aux[l], ucnt[l]);
                if (want_e) {
                    const uint32_t E = (l + 1 < NB ? eoff[l + 1] : (uint32_t)Eb) - eoff[l];
                    if (E > RANK_MAX) block_bitonic_sort(sorted_e + eoff[l], E);
                }
            }
            resolve(true);
            if (n_ok)
                for (uint64_t i = tid; i < Ub; i += BS) sh_out.col_n[Gn + i] = (int32_t)sorted[i];
            if (e_ok)
                for (uint64_t i = tid; i < Eb; i += BS) sh_out.col_e[Ge + i] = (int32_t)sorted_e[i];
            __syncthreads();
        } else {
            // large buckets: one thread per node, rows in global memory or staged
            resolve(fast);
            uint32_t* dst_n = stage ? stage : reinterpret_cast<uint32_t*>(sh_out.col_n) + Gn;
            int has_long = 0;
            if (n_ok) {
                for (int l = tid; l < NB; l += BS) {
                    const uint32_t U = ucnt[l];
                    if (U == 0) continue;
                    has_long |= U > LONG_ROW;
                    uint32_t* d = dst_n + aux[l];
                    const uint32_t* t = tab + toff[l];
                    const uint32_t T = tsz[l];
                    uint32_t j = 0;
                    for (uint32_t q = 0; q < T; ++q) {
                        const uint32_t y = t[q];
                        if (y != EMPTY) d[j++] = y;
                    }
                    if (U <= LONG_ROW) insertion_sort(d, (int)U);
                }
            }
            if (e_write) {
                for (int l = tid; l < NB; l += BS) {
                    const uint32_t E = (l + 1 < NB ? eoff[l + 1] : (uint32_t)Eb) - eoff[l];
                    has_long |= E > LONG_ROW;
                    if (E > 1 && E <= LONG_ROW) insertion_sort(elist + eoff[l], (int)E);
                }
            }
            has_long = __syncthreads_or(has_long);
            for (int l = 0; has_long && l < NB; ++l) {  // uniform loop: long rows, whole block
                if (n_ok && ucnt[l] > LONG_ROW) block_bitonic_sort(dst_n + aux[l], ucnt[l]);
                if (e_write) {
                    const uint32_t E = (l + 1 < NB ? eoff[l + 1] : (uint32_t)Eb) - eoff[l];
                    if (E > LONG_ROW) block_bitonic_sort(elist + eoff[l], E);
                }
            }
            __syncthreads();
            if (stage && n_ok)
                for (uint64_t i = tid; i < Ub; i += BS) sh_out.col_n[Gn + i] = (int32_t)stage[i];
            if (fast && e_ok)
                for (uint64_t i = tid; i < Eb; i += BS) sh_out.col_e[Ge + i] = (int32_t)elist[i];
            __syncthreads();
        }
        b_next = (int64_t)misc[5];
        __syncthreads();
    }
}

// Allow up to `bytes` of dynamic shared memory, less the kernel's own static
// shared memory (the sum may not exceed the per-block opt-in limit).
template <int RB, int K, int THREADS>
cudaError_t set_attr(size_t bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_bucket<RB, K, THREADS>);
    if (e != cudaSuccess) return e;
    const size_t dyn = bytes > a.sharedSizeBytes ? bytes - a.sharedSizeBytes : 0;
    return cudaFuncSetAttribute(k_bucket<RB, K, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

template <int THREADS>
void launch_t(const BucketParams& p, int grid, size_t smem, cudaStream_t s) {
    if (p.fmt.rb == 8) {
        if (p.fmt.k == 2) k_bucket<8, 2, THREADS><<<grid, THREADS, smem, s>>>(p);
        else k_bucket<8, 3, THREADS><<<grid, THREADS, smem, s>>>(p);
    } else {
        if (p.fmt.k == 2) k_bucket<16, 2, THREADS><<<grid, THREADS, smem, s>>>(p);
        else k_bucket<16, 3, THREADS><<<grid, THREADS, smem, s>>>(p);
    }
}

template <int THREADS>
cudaError_t set_attrs(size_t bytes) {
    cudaError_t e = set_attr<8, 2, THREADS>(bytes);
    if (e == cudaSuccess) e = set_attr<8, 3, THREADS>(bytes);
    if (e == cudaSuccess) e = set_attr<16, 2, THREADS>(bytes);
    if (e == cudaSuccess) e = set_attr<16, 3, THREADS>(bytes);
    return e;
}

}  // namespace

int bucket_threads() { return BUCKET_THREADS; }

cudaError_t launch_bucket(const BucketParams& p, int grid, int threads, size_t smem, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    if (threads == 256) launch_t<256>(p, grid, smem, s);
    else launch_t<512>(p, grid, smem, s);
    return cudaGetLastError();
}

cudaError_t set_bucket_smem_all(size_t bytes) {
    cudaError_t e = set_attrs<512>(bytes);
    if (e == cudaSuccess) e = set_attrs<256>(bytes);
    return e;
}

cudaError_t bucket_occupancy(int* blocks, int threads, size_t smem) {
    if (threads == 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_bucket<16, 3, 256>, 256, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_bucket<16, 3, 512>, 512, smem);
}

}  // namespace nn
