// Bucket pass: builds the rows of one node range per CTA from its records.
//
// For the 2^sb nodes of a bucket the CTA
//   1. counts the records (and element entries) of every node,
//   2. groups the bucket's record indices by node (a counting sort in shared
//      memory),
//   3. gives every node to one lane: 32 consecutive nodes form a group that
//      one warp finishes without block barriers.  The lane reads its node's
//      records, keeps the element ids in registers and inserts the neighbour
//      candidates into a private open-addressing hash table (a repeated
//      neighbour -- an edge shared by several elements -- hits its own slot
//      and is dropped).  A warp's tables are interleaved slot by slot, so the
//      32 lanes of a probe touch 32 different banks.  Both rows are then
//      sorted in registers by a bitonic network and staged in the group's
//      segment of shared memory.  A node with more records or distinct
//      neighbours than the registers hold is finished by its whole warp in
//      global scratch memory (bitonic sort, then adjacent-duplicate removal).
//   4. writes the element CSR at offsets known before the pass (a prefix of
//      the record counts), and leaves the node rows, each node's offset within
//      them and their total in a scratch area, at a position bounded in
//      advance (K times the bucket's first record); the compaction pass
//      places them (nn_compact.cu).  No bucket ever waits for another.
// A bucket whose record groups and element rows do not fit shared memory
// keeps them in a global spill area; so does a group whose distinct-neighbour
// rows do not fit.
//
// Rows are sets in ascending order: the paper's pipeline (Sec. 2.2.1) sorts
// pairs by key only and counts pairs per key, which lists an edge shared by
// two elements twice; one-ring neighbours are a set (Sec. 1), so repeated
// neighbours are dropped and each row is sorted.
#include "nn_device.cuh"

namespace nn {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int UNROLL = 8;   // records a thread loads before using them (counting and grouping)
constexpr int SLOT_SHIFT = 11;  // stash word: node offset (low 11 bits) | slot of the record in its node
// records a lane loads at once in the node phase
template <int IMAX> __host__ __device__ constexpr int chunk() { return IMAX >= 32 ? 4 : 8; }
constexpr uint32_t SEG_SPILL = 0x80000000u;  // group segment in the spill area
constexpr uint32_t SEG_NONE = 0xffffffffu;   // no room anywhere (status set)
constexpr uint64_t SPILL_INDEX_LIMIT = 0x7fffffffull;

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

// First 64-bit word of record r (it holds the node's offset in its bucket).
template <int RB>
__device__ __forceinline__ uint64_t load_rec_lo(const uint8_t* base, uint32_t r) {
    return __ldg(reinterpret_cast<const unsigned long long*>(base) + (size_t)r * (RB / 8));
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Ascending bitonic sorting network over a[0..N) held in registers (all
// indices are compile-time constants once unrolled).
template <int N, int M>
__device__ __forceinline__ void sort_net(uint32_t (&a)[M]) {
    static_assert(N <= M && (N & (N - 1)) == 0, "network size");
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int q = i ^ j;
                if (q > i) {
                    const uint32_t x = a[i], y = a[q];
                    const uint32_t lo = min(x, y), hi = max(x, y);
                    if ((i & k) == 0) {
                        a[i] = lo;
                        a[q] = hi;
                    } else {
                        a[i] = hi;
                        a[q] = lo;
                    }
                }
            }
        }
    }
}

// Sort the first n <= M entries (the rest are EMPTY): the smallest network
// that covers the warp's longest row (n_warp is warp-uniform).
template <int M>
__device__ __forceinline__ void sort_prefix(uint32_t (&a)[M], uint32_t n_warp) {
    if (n_warp <= 1) return;
    if (n_warp <= 4) sort_net<4>(a);
    else if (n_warp <= 8) sort_net<8>(a);
    else if constexpr (M >= 16) {
        if (n_warp <= 16 || M == 16) sort_net<16>(a);
        else sort_net<M>(a);
    }
}

// Ascending bitonic sort of a[0..n) by one warp (generic pointer), in the
// formulation whose compare-exchanges put the minimum at the lower index, so
// that indices >= n act as +infinity and are skipped.
__device__ inline void warp_bitonic_sort(uint32_t* a, uint32_t n) {
    if (n < 2) return;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t P = 1;
    while (P < n) P <<= 1;
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = lane; t < (P >> 1); t += 32) {
                const uint32_t idx = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const uint32_t q = (j == (k >> 1)) ? (idx ^ (k - 1)) : (idx ^ j);
                if (q < n) {
                    const uint32_t x = a[idx], y = a[q];
                    if (x > y) {
                        a[idx] = y;
                        a[q] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Insert y into the lane's private table (slot h at tab[h * 32]); false when
// the table already holds UCAP values (the node then takes the warp path).
// Fewer than HT values are ever stored, so a probe always ends.
template <int HT, int UCAP>
__device__ __forceinline__ bool lane_insert(uint32_t* tab, uint32_t y, uint32_t& u) {
    constexpr int LOG = HT == 16 ? 4 : 5;
    uint32_t h = (y * 0x9E3779B1u) >> (32 - LOG);
#pragma unroll 1
    for (int pr = 0; pr < HT; ++pr) {
        const uint32_t t = tab[h * 32];
        if (t == y) return true;
        if (t == EMPTY) {
            if (u >= (uint32_t)UCAP) return false;
            tab[h * 32] = y;
            ++u;
            return true;
        }
        h = (h + 1) & (HT - 1);
    }
    return false;
}

struct BucketOut {
    int64_t n_nodes, first;
    bool last;
    int64_t* rp_n; int32_t* col_n; int64_t cap_n;
    int64_t* rp_e; int32_t* col_e; int64_t cap_e;
    int32_t* status;
};

// Shared memory: per node cnt (u64) and gcur (u32); per group gseg, gtot,
// gpre (64 each); scan scratch (34 u64); misc (8 u64); the warps' tables;
// then the area (record groups, element rows, distinct-neighbour segments).
__host__ __device__ constexpr size_t fixed_bytes(int sb, int threads, int ht) {
    return ((size_t)12 << sb) + 3 * 64 * 4 + 34 * 8 + 8 * 8 + (size_t)(threads / 32) * ht * 32 * 4;
}

template <int RB, int K, int IMAX, int HT, int THREADS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS) k_bucket(BucketParams p) {
    constexpr int W = THREADS / 32;
    constexpr int UCAP = HT * 3 / 4;
    constexpr int CH = chunk<IMAX>();
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ BucketOut sh_out;
    const bool batched = p.batch.hdr != nullptr;
    const RecFmt f = batched ? p.batch.hdr->fmt : p.fmt;
    const int64_t n_buckets = batched ? p.batch.hdr->n_buckets : p.n_buckets;
    const int n_meshes = batched ? p.batch.hdr->n_meshes : 1;
    const int NB = 1 << f.sb;
    const uint32_t vmask = (uint32_t)NB - 1;
    uint64_t* cnt = reinterpret_cast<uint64_t*>(smem);  // [NB] counts, then packed offsets
    uint32_t* gcur = reinterpret_cast<uint32_t*>(cnt + NB);  // [NB] grouping cursor, then offset in group
    uint32_t* gseg = gcur + NB;                              // [64] group segment
    uint32_t* gtot = gseg + 64;                              // [64] distinct neighbours of the group
    uint32_t* gpre = gtot + 64;                              // [64] their exclusive prefix
    uint64_t* sh_scan = reinterpret_cast<uint64_t*>(gpre + 64);  // 34 words
    uint64_t* misc = sh_scan + 34;                                // 8 words
    uint32_t* tabs = reinterpret_cast<uint32_t*>(misc + 8);       // [W][HT][32]
    uint32_t* area = tabs + W * HT * 32;
    const bool want_n = f.want & NN_WANT_NODES, want_e = f.want & NN_WANT_ELEMS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* const tabw = tabs + warp * (HT * 32) + lane;

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
            // the mesh this bucket belongs to (the only one unless batched)
            BucketOut o{p.n_nodes, 0, b == n_buckets - 1, p.rp_n, p.col_n, p.cap_n, p.rp_e, p.col_e, p.cap_e, p.status};
            if (batched) {
                int lo_m = 0, hi_m = n_meshes;  // largest m with bucket_off[m] <= b
                while (hi_m - lo_m > 1) {
                    const int mid = (lo_m + hi_m) >> 1;
                    if (p.batch.bucket_off[mid] <= b) lo_m = mid;
                    else hi_m = mid;
                }
                const BatchMesh& M = p.batch.meshes[lo_m];
                o = BucketOut{M.n_nodes, p.batch.bucket_off[lo_m], b == p.batch.bucket_off[lo_m + 1] - 1, M.rp_n,
                              M.col_n, M.cap_n, M.rp_e, M.col_e, M.cap_e, M.status};
                if (*p.batch_err) set_status(o.status, *p.batch_err);
            }
            sh_out = o;
        }
        for (int l = tid; l < NB; l += THREADS) {
            cnt[l] = 0;
            gcur[l] = 0;
        }
        if (tid < 64) gtot[tid] = 0;
        __syncthreads();
        const int64_t N = sh_out.n_nodes, first = sh_out.first;
        int32_t* const status = sh_out.status;
        const int64_t v0 = (b - first) << f.sb;
        const int nb = (int)(N - v0 < (int64_t)NB ? N - v0 : (int64_t)NB);
        const uint32_t r0 = p.bstart[b], r1 = p.bstart[b + 1];
        const uint32_t R = r1 - r0;

        // 1. records per node (low word) and element entries (high word); each
        // record's slot in its node is stashed (past the largest possible
        // element rows, where distinct-neighbour rows go later) when it fits
        const bool stash_ok = 3ull * R <= p.area_words;
        uint32_t* const stash = area + 2 * R;
        if (tid == 0) misc[6] = 0;
        for (uint32_t r = r0 + tid; r < r1; r += UNROLL * THREADS) {
            uint64_t xs[UNROLL];
#pragma unroll
            for (int q = 0; q < UNROLL; ++q)
                if (r + q * THREADS < r1) xs[q] = load_rec_lo<RB>(p.rec, r + q * THREADS);
#pragma unroll
            for (int q = 0; q < UNROLL; ++q) {
                if (r + q * THREADS >= r1) break;
                const uint32_t vloc = (uint32_t)xs[q] & vmask;
                const bool is_e = want_e && !((xs[q] >> f.off_nf) & 1);  // flag bit sb < 64
                const uint32_t slot = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[vloc]),
                                                          1ull + (is_e ? 1ull << 32 : 0ull));
                if (stash_ok) stash[r + q * THREADS - r0] = vloc | (slot << SLOT_SHIFT);
            }
        }
        __syncthreads();
        const uint64_t tot = smem_array_excl_scan(cnt, NB, sh_scan);  // packed: group offset | element offset
        const uint32_t Eb = (uint32_t)(tot >> 32);
        if (tid == 0) {
            uint64_t base = 0;
            uint32_t flags = 1;  // bit 0: storage found, bit 1: in shared memory
            const uint64_t need = (uint64_t)R + Eb;
            if (need <= p.area_words) {
                flags |= 2;
            } else {
                base = atomicAdd(p.spill_cursor, (unsigned long long)need);
                if (base + need > p.spill_words) {
                    flags = 0;
                    set_status(status, NN_ERR_WORKSPACE);
                }
            }
            misc[2] = base;
            misc[4] = flags;
        }
        __syncthreads();
        const uint32_t flags = (uint32_t)misc[4];
        const bool ok = flags & 1, insm = flags & 2;
        uint32_t* const grp = insm ? area : p.spill + misc[2];
        uint32_t* const Est = grp + R;
        uint32_t* const Ust = insm ? area + R + Eb : area;
        const uint64_t ucap = insm ? (uint64_t)p.area_words - R - Eb : (uint64_t)p.area_words;

        // the element rows' offset: a prefix of the record counts, known
        // before this pass (for a batch, relative to the mesh's first bucket;
        // for a chunk, after the earlier chunks' entries)
        if (want_e && tid == 0) {
            const uint64_t ge = (uint64_t)(p.estart[b] - p.estart[first]) + (p.base ? (uint64_t)p.base[0] : 0ull);
            misc[1] = ge;
            if (ge + Eb > (uint64_t)sh_out.cap_e) set_status(status, NN_ERR_CAPACITY);
        }
        // 2. record indices grouped by node (a node with more than 2^21
        // records in one bucket cannot be stashed: any slot that large is
        // simply counted again)
        if (ok && stash_ok && R <= (1u << (32 - SLOT_SHIFT))) {
            for (uint32_t i = tid; i < R; i += THREADS) {
                const uint32_t w = stash[i];
                const uint32_t vloc = w & ((1u << SLOT_SHIFT) - 1);
                grp[(uint32_t)cnt[vloc] + (w >> SLOT_SHIFT)] = i;
            }
        } else if (ok) {
            for (uint32_t r = r0 + tid; r < r1; r += UNROLL * THREADS) {
                uint64_t xs[UNROLL];
#pragma unroll
                for (int q = 0; q < UNROLL; ++q)
                    if (r + q * THREADS < r1) xs[q] = load_rec_lo<RB>(p.rec, r + q * THREADS);
#pragma unroll
                for (int q = 0; q < UNROLL; ++q) {
                    if (r + q * THREADS >= r1) break;
                    const uint32_t vloc = (uint32_t)xs[q] & vmask;
                    const uint32_t slot = atomicAdd(&gcur[vloc], 1u);
                    grp[(uint32_t)cnt[vloc] + slot] = r + q * THREADS - r0;
                }
            }
        }
        __syncthreads();

        // 3. one lane per node, one warp per group of 32 nodes
        const int ng = (nb + 31) >> 5;
        for (int g = warp; ok && g < ng; g += W) {
            const int l = g * 32 + lane;
            const bool valid = l < nb;
            uint32_t c = 0, goff = 0, eoff = 0, ecnt = 0;
            if (valid) {
                const uint64_t a = cnt[l];
                const uint64_t z = l + 1 < NB ? cnt[l + 1] : tot;
                goff = (uint32_t)a;
                eoff = (uint32_t)(a >> 32);
                c = (uint32_t)z - goff;
                ecnt = (uint32_t)(z >> 32) - eoff;
            }
            const bool fast = valid && c <= (uint32_t)IMAX;
            const uint32_t cmax = __reduce_max_sync(FULL, fast ? c : 0u);
            // few candidates (K per record): straight into registers, sorted,
            // duplicates skipped when written; else through the lane's table
            const bool direct = (uint32_t)K * cmax <= 32u;
            uint32_t u = 0;
            bool ovf = false;
            if (want_n && !direct) {
#pragma unroll
                for (int h = 0; h < HT; ++h) tabw[h * 32] = EMPTY;
            }
            uint32_t v[IMAX], w[32];
#pragma unroll
            for (int s = 0; s < IMAX; ++s) v[s] = EMPTY;
#pragma unroll
            for (int s = 0; s < 32; ++s) w[s] = EMPTY;
#pragma unroll
            for (int s0 = 0; s0 < IMAX; s0 += CH) {
                if ((uint32_t)s0 >= cmax) break;
                Rec xs[CH];
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    if (fast && (uint32_t)(s0 + q) < c) xs[q] = load_rec<RB>(p.rec, r0 + grp[goff + s0 + q]);
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    if (fast && (uint32_t)(s0 + q) < c) {
                        const Rec& x = xs[q];
                        if (want_e && !rec_get(x, f.off_nf, 1)) v[s0 + q] = rec_get(x, f.off_e, f.eb);
                        if (want_n) {
#pragma unroll
                            for (int j = 0; j < K; ++j) {
                                const uint32_t y = rec_get(x, f.off_n + j * f.nb, f.nb);
                                if (direct) {
                                    if (K * (s0 + q) + j < 32) w[K * (s0 + q) + j] = y - 1;  // 0 (none) -> EMPTY
                                } else if (y && !ovf) {
                                    ovf = !lane_insert<HT, UCAP>(tabw, y - 1, u);
                                }
                            }
                        }
                    }
                }
            }
            if (want_e) {
                sort_prefix(v, cmax);
                if (fast) {
#pragma unroll
                    for (int s = 0; s < IMAX; ++s)
                        if ((uint32_t)s < ecnt) Est[eoff + s] = v[s];
                }
            }
            const uint32_t nw = direct ? (uint32_t)K * cmax : (uint32_t)HT;  // entries that may be set
            if (want_n) {
                if (!direct) {
#pragma unroll
                    for (int h = 0; h < HT; ++h) w[h] = tabw[h * 32];
                }
                sort_prefix(w, nw);
                u = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if ((uint32_t)j >= nw) break;
                    u += w[j] != EMPTY && (j == 0 || w[j] != w[j - 1]);
                }
            }

            // nodes beyond the registers: the whole warp, in global scratch
            const unsigned slowE = __ballot_sync(FULL, valid && want_e && !fast);
            const unsigned slowU = __ballot_sync(FULL, valid && want_n && (!fast || ovf));
            for (unsigned m = slowE; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                const uint32_t cc = __shfl_sync(FULL, c, i), go = __shfl_sync(FULL, goff, i);
                const uint32_t eo = __shfl_sync(FULL, eoff, i), ec = __shfl_sync(FULL, ecnt, i);
                uint32_t* row = Est + eo;
                uint32_t wpos = 0;
                for (uint32_t s0 = 0; s0 < cc; s0 += 32) {
                    const uint32_t s = s0 + lane;
                    bool keep = false;
                    uint32_t e = 0;
                    if (s < cc) {
                        const Rec x = load_rec<RB>(p.rec, r0 + grp[go + s]);
                        keep = !rec_get(x, f.off_nf, 1);
                        e = rec_get(x, f.off_e, f.eb);
                    }
                    const unsigned km = __ballot_sync(FULL, keep);
                    if (keep) row[wpos + __popc(km & lanemask_lt())] = e;
                    wpos += __popc(km);
                }
                __syncwarp();
                warp_bitonic_sort(row, ec);
            }
            uint32_t uscr = 0;
            for (unsigned m = slowU; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                const uint32_t cc = __shfl_sync(FULL, c, i), go = __shfl_sync(FULL, goff, i);
                const uint64_t nc = (uint64_t)K * cc;
                unsigned long long so = 0;
                if (lane == 0) so = atomicAdd(p.spill_cursor, (unsigned long long)nc);
                so = __shfl_sync(FULL, so, 0);
                uint32_t nu = 0;
                if (so + nc > p.spill_words || so + nc > SPILL_INDEX_LIMIT) {
                    if (lane == 0) set_status(status, NN_ERR_WORKSPACE);
                } else {
                    uint32_t* a = p.spill + so;
                    for (uint32_t s = lane; s < cc; s += 32) {
                        const Rec x = load_rec<RB>(p.rec, r0 + grp[go + s]);
#pragma unroll
                        for (int j = 0; j < K; ++j) {
                            const uint32_t y = rec_get(x, f.off_n + j * f.nb, f.nb);
                            a[(uint64_t)s * K + j] = y ? y - 1 : EMPTY;
                        }
                    }
                    __syncwarp();
                    warp_bitonic_sort(a, (uint32_t)nc);
                    // keep the first of every run (in place: writes never pass the chunk being read)
                    uint32_t carry = EMPTY;
                    for (uint32_t i0 = 0; i0 < nc; i0 += 32) {
                        const uint32_t idx = i0 + lane;
                        const uint32_t val = idx < nc ? a[idx] : EMPTY;
                        uint32_t prev = __shfl_up_sync(FULL, val, 1);
                        if (lane == 0) prev = carry;
                        carry = __shfl_sync(FULL, val, 31);
                        const bool keep = val != EMPTY && val != prev;
                        const unsigned km = __ballot_sync(FULL, keep);
                        __syncwarp();
                        if (keep) a[nu + __popc(km & lanemask_lt())] = val;
                        nu += __popc(km);
                        __syncwarp();
                    }
                }
                if (lane == i) {
                    u = nu;
                    uscr = (uint32_t)so;
                }
            }

            // the group's distinct-neighbour rows, contiguous in node order
            if (want_n) {
                const uint32_t uu = valid ? u : 0u;
                uint32_t incl = uu;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(FULL, incl, d);
                    if (lane >= d) incl += y;
                }
                const uint32_t ex = incl - uu, gt = __shfl_sync(FULL, incl, 31);
                uint32_t seg = 0;
                if (lane == 0) {
                    const unsigned long long s =
                        atomicAdd(reinterpret_cast<unsigned long long*>(&misc[6]), (unsigned long long)gt);
                    if (s + gt <= ucap) {
                        seg = (uint32_t)s;
                    } else {
                        const unsigned long long so = atomicAdd(p.spill_cursor, (unsigned long long)gt);
                        if (so + gt > p.spill_words || so + gt > SPILL_INDEX_LIMIT) {
                            seg = SEG_NONE;
                            set_status(status, NN_ERR_WORKSPACE);
                        } else {
                            seg = SEG_SPILL | (uint32_t)so;
                        }
                    }
                }
                seg = __shfl_sync(FULL, seg, 0);
                if (seg != SEG_NONE) {
                    uint32_t* sp = (seg & SEG_SPILL) ? p.spill + (seg & ~SEG_SPILL) : Ust + seg;
                    if (valid && !((slowU >> lane) & 1)) {
                        uint32_t* d = sp + ex;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if ((uint32_t)j >= nw) break;
                            if (w[j] != EMPTY && (j == 0 || w[j] != w[j - 1])) *d++ = w[j];
                        }
                    }
                    for (unsigned m = slowU; m; m &= m - 1) {
                        const int i = __ffs(m) - 1;
                        const uint32_t nu = __shfl_sync(FULL, u, i), so = __shfl_sync(FULL, uscr, i);
                        const uint32_t exi = __shfl_sync(FULL, ex, i);
                        for (uint32_t j = lane; j < nu; j += 32) sp[exi + j] = p.spill[(uint64_t)so + j];
                    }
                }
                if (valid) gcur[l] = ex;
                if (lane == 0) {
                    gseg[g] = seg;
                    gtot[g] = seg == SEG_NONE ? 0u : gt;
                }
            }
        }
        __syncthreads();

        // 4. element rows to their offset; node rows, with each node's offset
        // within the bucket and the bucket's total, to the scratch area (their
        // offsets are placed by the compaction pass, so no bucket waits here)
        const uint64_t Ge = misc[1];
        if (warp == 0) {
            const int NG = (NB + 31) >> 5;  // <= 64
            const uint32_t a0 = lane < NG ? gtot[lane] : 0u, a1 = lane + 32 < NG ? gtot[lane + 32] : 0u;
            uint32_t s0 = a0, s1 = a1;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y0 = __shfl_up_sync(FULL, s0, d), y1 = __shfl_up_sync(FULL, s1, d);
                if (lane >= d) {
                    s0 += y0;
                    s1 += y1;
                }
            }
            const uint32_t t0 = __shfl_sync(FULL, s0, 31);
            s1 += t0;
            if (lane < NG) gpre[lane] = s0 - a0;
            if (lane + 32 < NG) gpre[lane + 32] = s1 - a1;
            if (want_n && lane == 31) p.ubk[b] = s1;
        } else if (want_e) {
            const bool e_ok = ok && Ge + Eb <= (uint64_t)sh_out.cap_e;
            for (int l = tid - 32; l < nb; l += THREADS - 32)
                sh_out.rp_e[v0 + l] = (int64_t)(Ge + (uint32_t)(cnt[l] >> 32));
            if (e_ok) {
                int32_t* dst = sh_out.col_e + Ge;
                for (uint32_t i = tid - 32; i < Eb; i += THREADS - 32) dst[i] = (int32_t)Est[i];
            }
        }
        __syncthreads();
        if (want_n) {
            uint32_t* const loc = p.nloc + ((size_t)b << f.sb);
            for (int l = tid; l < nb; l += THREADS) loc[l] = gpre[l >> 5] + gcur[l];
            uint32_t* const rows = p.ntmp + (size_t)K * r0;
            for (int g = warp; ok && g < ng; g += W) {
                const uint32_t seg = gseg[g], n = gtot[g];
                if (seg == SEG_NONE) continue;
                const uint32_t* src = (seg & SEG_SPILL) ? p.spill + (seg & ~SEG_SPILL) : Ust + seg;
                uint32_t* dst = rows + gpre[g];
                for (uint32_t i = lane; i < n; i += 32) dst[i] = src[i];
            }
        }
        if (sh_out.last && tid == 0 && want_e) sh_out.rp_e[N] = (int64_t)(Ge + Eb);
        b_next = (int64_t)misc[5];
        __syncthreads();
    }
}

// Allow up to `bytes` of dynamic shared memory, less the kernel's own static
// shared memory (the sum may not exceed the per-block opt-in limit).
template <int RB, int K, int IMAX, int HT, int THREADS>
cudaError_t set_attr(size_t bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_bucket<RB, K, IMAX, HT, THREADS>);
    if (e != cudaSuccess) return e;
    const size_t dyn = bytes > a.sharedSizeBytes ? bytes - a.sharedSizeBytes : 0;
    return cudaFuncSetAttribute(k_bucket<RB, K, IMAX, HT, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dyn);
}

template <int IMAX, int HT, int THREADS>
void launch_w(const BucketParams& p, int grid, size_t smem, cudaStream_t s) {
    if (p.fmt.rb == 8) {
        if (p.fmt.k == 2) k_bucket<8, 2, IMAX, HT, THREADS><<<grid, THREADS, smem, s>>>(p);
        else k_bucket<8, 3, IMAX, HT, THREADS><<<grid, THREADS, smem, s>>>(p);
    } else {
        if (p.fmt.k == 2) k_bucket<16, 2, IMAX, HT, THREADS><<<grid, THREADS, smem, s>>>(p);
        else k_bucket<16, 3, IMAX, HT, THREADS><<<grid, THREADS, smem, s>>>(p);
    }
}

template <int IMAX, int HT, int THREADS>
cudaError_t set_attrs_w(size_t bytes) {
    cudaError_t e = set_attr<8, 2, IMAX, HT, THREADS>(bytes);
    if (e == cudaSuccess) e = set_attr<8, 3, IMAX, HT, THREADS>(bytes);
    if (e == cudaSuccess) e = set_attr<16, 2, IMAX, HT, THREADS>(bytes);
    if (e == cudaSuccess) e = set_attr<16, 3, IMAX, HT, THREADS>(bytes);
    return e;
}

}  // namespace

size_t bucket_fixed_bytes(int sb, int threads, int wide) { return fixed_bytes(sb, threads, wide ? 32 : 16); }

cudaError_t launch_bucket(const BucketParams& p, int grid, int threads, size_t smem, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    if (p.wide) {
        if (threads == 128) launch_w<32, 32, 128>(p, grid, smem, s);
        else launch_w<32, 32, 256>(p, grid, smem, s);
    } else {
        if (threads == 128) launch_w<16, 16, 128>(p, grid, smem, s);
        else launch_w<16, 16, 256>(p, grid, smem, s);
    }
    return cudaGetLastError();
}

cudaError_t set_bucket_smem_all(size_t bytes) {
    cudaError_t e = set_attrs_w<16, 16, 128>(bytes);
    if (e == cudaSuccess) e = set_attrs_w<16, 16, 256>(bytes);
    if (e == cudaSuccess) e = set_attrs_w<32, 32, 128>(bytes);
    if (e == cudaSuccess) e = set_attrs_w<32, 32, 256>(bytes);
    return e;
}

cudaError_t bucket_occupancy(int* blocks, int threads, int wide, size_t smem) {
    if (wide) {
        if (threads == 128)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_bucket<16, 3, 32, 32, 128>, 128, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_bucket<16, 3, 32, 32, 256>, 256, smem);
    }
    if (threads == 128)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_bucket<16, 3, 16, 16, 128>, 128, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_bucket<16, 3, 16, 16, 256>, 256, smem);
}

}  // namespace nn
