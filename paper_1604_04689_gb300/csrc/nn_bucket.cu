// Bucket pass: builds the rows of one node range per CTA from its records.
//
// For the 2^sb nodes of a bucket the CTA
//   0. copies the bucket's records into shared memory with bulk asynchronous
//      copies (cp.async.bulk, completion on an mbarrier, bounded wait).  The
//      next bucket is taken while this one is built, and its records are
//      copied in as soon as this one's records are dead, while this bucket
//      still writes its rows.  (Plans whose buckets would then hold too few
//      nodes to keep every warp busy -- nodes of many records, like tets --
//      leave the records in global memory and pull the next bucket's into L2
//      instead.)
//   1. counts the records of every node; each record keeps the slot its
//      count gave it (one shared-memory atomic per record, the only one),
//   2. groups the bucket's record indices by node (the slots make this a
//      plain scatter),
//   3. gives every node to one lane: 32 consecutive nodes form a group that
//      one warp finishes without block barriers, in two phases so that their
//      register arrays are never live together.  Element row: the lane keeps
//      the element ids of its node's records in registers and sorts them with
//      a bitonic network.  Neighbour row: few candidates go straight into
//      registers and are sorted (repeats dropped when written); otherwise
//      they go into a private open-addressing hash table (a repeated
//      neighbour -- an edge shared by several elements -- hits its own slot
//      and is dropped), whose distinct values are compacted and sorted in
//      registers.  A warp's tables are interleaved slot by slot, so the 32
//      lanes of a probe touch 32 different banks.  A node with more records
//      or distinct neighbours than the registers hold is finished by its
//      whole warp (element rows in place, neighbour rows in global scratch:
//      bitonic sort, then adjacent-duplicate removal),
//   4. writes the element CSR at offsets known before the pass (a prefix of
//      the record counts), and leaves the node rows, each node's offset within
//      them and their total in a scratch area, at a position bounded in
//      advance (K times the bucket's first record); the compaction pass
//      places them (nn_compact.cu).  No bucket ever waits for another.
// A bucket too large for shared memory reads its records from global memory
// and keeps its groups and element rows in a global spill area when they do
// not fit either; so does a group whose neighbour rows do not fit.
//
// Rows are sets in ascending order: the paper's pipeline (Sec. 2.2.1) sorts
// pairs by key only and counts pairs per key, which lists an edge shared by
// two elements twice; one-ring neighbours are a set (Sec. 1), so repeated
// neighbours are dropped and each row is sorted.
#include "nn_bulk.cuh"

namespace nn {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t BULK_CHUNK = 32768;       // bytes per bulk copy instruction
constexpr uint32_t SEG_SPILL = 0x80000000u;  // group segment in the spill area
constexpr uint32_t SEG_NONE = 0xffffffffu;   // no room anywhere (status set)
constexpr uint64_t SPILL_INDEX_LIMIT = 0x7fffffffull;

// ------------------------------------------------------------- records
// Record i of the current bucket.  `rp` points at record 0 of the bucket,
// in shared memory (the usual case) or in the record array in global memory
// (a bucket too large to copy); a generic load serves both.
template <int RB>
__device__ __forceinline__ Rec get_rec(const uint8_t* rp, uint32_t i) {
    Rec x;
    if constexpr (RB == 8) {
        x.lo = reinterpret_cast<const unsigned long long*>(rp)[i];
        x.hi = 0;
    } else {
        const ulonglong2 w = reinterpret_cast<const ulonglong2*>(rp)[i];
        x.lo = w.x;
        x.hi = w.y;
    }
    return x;
}
// First 64-bit word of record i (it holds the node's offset in its bucket).
template <int RB>
__device__ __forceinline__ uint64_t get_rec_lo(const uint8_t* rp, uint32_t i) {
    return reinterpret_cast<const unsigned long long*>(rp)[(size_t)i * (RB / 8)];
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__host__ __device__ constexpr int pow2_ceil(int n) { return n <= 1 ? 1 : 2 * pow2_ceil((n + 1) / 2); }

// Ascending sort of a[0..N) held in registers by Batcher's odd-even merge
// sort (Knuth, TAOCP vol. 3, 5.3.4), laid out for the next power of two P
// >= N and pruned to N: every comparator puts the minimum at its lower index,
// so the +infinity (EMPTY) entries at N..P-1 never move and a comparator that
// touches one of them is a no-op.  Every index is a compile-time constant
// once the loops are unrolled, so the array stays in registers.
template <int N, int M>
__device__ __forceinline__ void sort_net(uint32_t (&a)[M]) {
    static_assert(N <= M, "network size");
    constexpr int P = pow2_ceil(N);
#pragma unroll
    for (int p = 1; p < P; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
            // comparators (lo, lo + k) for lo = j + i, j = k mod p + 2k t, 0 <= i < k,
            // both ends in one block of 2p
#pragma unroll
            for (int lo = 0; lo < P; ++lo) {
                const int r = lo - k % p, hi = lo + k;
                if (r >= 0 && r % (2 * k) < k && hi < N && lo / (2 * p) == hi / (2 * p)) {
                    const uint32_t x = a[lo], y = a[hi];
                    a[lo] = min(x, y);
                    a[hi] = max(x, y);
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
    if (n_warp <= 2) sort_net<2>(a);
    else if (n_warp <= 4) sort_net<4>(a);
    else if (n_warp <= 6) sort_net<6>(a);
    else if (n_warp <= 8) sort_net<8>(a);
    else if constexpr (M >= 16) {
        if (n_warp <= 12) sort_net<12>(a);
        else if (n_warp <= 16 || M == 16) sort_net<16>(a);
        else if constexpr (M >= 24) {
            if (n_warp <= 24) sort_net<24>(a);
            else sort_net<M>(a);
        }
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

// Insert y into the lane's private table (slot h at tab[h * 32], h < HT);
// false when the table already holds UCAP values (the node then takes the
// warp path).  Fewer than HT values are ever stored, so a probe always ends
// at an empty slot or at y; every slot index is reduced mod HT, so the probe
// never leaves the lane's own HT slots.
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

// A node whose element row exceeds the registers: its whole warp collects
// the element ids of the node's c records (a repeated node's record adds
// none) into row[0..ec) and sorts them there.  Kept out of line: the fast
// path's registers stay free of it.
template <int RB>
__device__ __noinline__ void warp_elem_row(const uint8_t* rp, const uint32_t* grp, uint32_t c, uint32_t* row,
                                           uint32_t ec, int off_nf, int off_e, int eb) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t wpos = 0;
    for (uint32_t s0 = 0; s0 < c; s0 += 32) {
        const uint32_t s = s0 + lane;
        bool keep = false;
        uint32_t e = 0;
        if (s < c) {
            const Rec x = get_rec<RB>(rp, grp[s]);
            keep = !rec_get(x, off_nf, 1);
            e = rec_get(x, off_e, eb);
        }
        const unsigned km = __ballot_sync(FULL, keep);
        if (keep) row[wpos + __popc(km & lanemask_lt())] = e;
        wpos += __popc(km);
    }
    __syncwarp();
    warp_bitonic_sort(row, ec);
}

// A node with more distinct neighbours than a lane's table takes: its whole
// warp writes the K candidates of each of its c records to the spill area,
// sorts them and keeps the first of every run.  Returns the distinct count
// (the row is at spill + *so); 0 with NN_ERR_WORKSPACE when the spill area
// is exhausted.  Kept out of line like warp_elem_row.
template <int RB, int K>
__device__ __noinline__ uint32_t warp_node_row(const uint8_t* rp, const uint32_t* grp, uint32_t c, uint32_t* spill,
                                               uint64_t spill_words, unsigned long long* spill_cursor,
                                               int32_t* status, int off_n, int nb, uint32_t* so_out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nc = (uint64_t)K * c;
    unsigned long long so = 0;
    if (lane == 0) so = atomicAdd(spill_cursor, (unsigned long long)((nc + 3) & ~3ull));
    so = __shfl_sync(FULL, so, 0);
    *so_out = (uint32_t)so;
    if (so + nc > spill_words || so + nc > SPILL_INDEX_LIMIT) {
        if (lane == 0) set_status(status, NN_ERR_WORKSPACE);
        return 0;
    }
    uint32_t* a = spill + so;
    for (uint32_t s = lane; s < c; s += 32) {
        const Rec x = get_rec<RB>(rp, grp[s]);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t y = rec_get(x, off_n + j * nb, nb);
            a[(uint64_t)s * K + j] = y ? y - 1 : EMPTY;
        }
    }
    __syncwarp();
    warp_bitonic_sort(a, (uint32_t)nc);
    // keep the first of every run (in place: writes never pass the chunk being read)
    uint32_t nu = 0, carry = EMPTY;
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
    return nu;
}

struct BucketOut {
    int64_t n_nodes, first;
    bool last;
    int64_t* rp_n; int32_t* col_n; int64_t cap_n;
    int64_t* rp_e; int32_t* col_e; int64_t cap_e;
    int32_t* status;
};

// What the bucket pass knows of a bucket before it starts on it: its
// records, where its element rows go, and whether it fits shared memory.
struct BucketMeta {
    int64_t b;
    uint32_t r0, r1;
    uint64_t ge;      // element-CSR offset of its rows
    uint32_t sr;      // 1: processed in shared memory (records copied in)
    uint32_t copied;  // 1: the copy of its records is already issued
};

// Shared memory: per node the packed offsets (u64: record group low, element
// row high), the record count (u32; later the node's offset within its
// group's neighbour rows) and the repeated-node count (u32); per group of 32
// nodes the segment, total and prefix of its neighbour rows (64 each); scan
// scratch (34 u64); misc (8 u64); the warps' tables; then the area.  In the
// area a bucket's records sit at the bottom; at the top its element rows
// (which first hold each record's slot in its node), below them the record
// groups, and below those the groups' neighbour rows, allocated downwards
// while the records are still live.  Once the rows are built the records are
// dead, and the next bucket's records can be copied in at the bottom while
// this bucket writes its rows, whenever both fit.  Every part is a multiple
// of 16 bytes, so the area starts 16-byte aligned.
__host__ __device__ constexpr size_t fixed_bytes(int sb, int threads, int ht) {
    return ((size_t)16 << sb) + 3 * 64 * 4 + 34 * 8 + 8 * 8 + (size_t)(threads / 32) * ht * 32 * 4;
}
// bytes of the parts of a bucket of R records
__host__ __device__ inline uint64_t rec_bytes(uint64_t R, uint32_t roff, int RB) { return (R * RB + roff + 15) & ~15ull; }
__host__ __device__ inline uint64_t word_bytes(uint64_t n) { return (n * 4 + 15) & ~15ull; }

template <int RB, int K, int IMAX, int HT, int THREADS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS) k_bucket(BucketParams p) {
    constexpr int W = THREADS / 32;
    constexpr int UCAP = HT * 3 / 4;
    constexpr int CH = 4;  // records a lane loads at once in the row phase
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ BucketOut sh_out;
    __shared__ BucketMeta meta[2];
    __shared__ uint64_t mbar;
    const bool batched = p.batch.hdr != nullptr;
    const RecFmt f = batched ? p.batch.hdr->fmt : p.fmt;
    const int64_t n_buckets = batched ? p.batch.hdr->n_buckets : p.n_buckets;
    const int n_meshes = batched ? p.batch.hdr->n_meshes : 1;
    const int NB = 1 << f.sb;
    const uint32_t vmask = (uint32_t)NB - 1;
    uint64_t* cnt = reinterpret_cast<uint64_t*>(smem);   // [NB] packed offsets
    uint32_t* c32 = reinterpret_cast<uint32_t*>(cnt + NB);  // [NB] records, then offset within the group's rows
    uint32_t* nfc = c32 + NB;                               // [NB] repeated-node records
    uint32_t* gseg = nfc + NB;                              // [64] group segment
    uint32_t* gtot = gseg + 64;                             // [64] distinct neighbours of the group
    uint32_t* gpre = gtot + 64;                             // [64] their exclusive prefix
    uint64_t* sh_scan = reinterpret_cast<uint64_t*>(gpre + 64);  // 34 words
    uint64_t* misc = sh_scan + 34;                                // 8 words
    uint32_t* tabs = reinterpret_cast<uint32_t*>(misc + 8);       // [W][HT][32]
    uint8_t* area = reinterpret_cast<uint8_t*>(tabs + W * HT * 32);
    const uint64_t A = (uint64_t)p.area_words * 4;
    const bool want_n = f.want & NN_WANT_NODES, want_e = f.want & NN_WANT_ELEMS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* const tabw = tabs + warp * (HT * 32) + lane;

    auto issue_copy = [&](const BucketMeta& M) {
        const uint32_t roff = RB == 8 ? (M.r0 & 1u) * 8u : 0u;
        const uint64_t rbytes = rec_bytes(M.r1 - M.r0, roff, RB);
        fence_async_smem();
        mbar_expect(&mbar, (uint32_t)rbytes);
        const uint8_t* src = p.rec + (uint64_t)M.r0 * RB - roff;
        for (uint64_t a = 0; a < rbytes; a += BULK_CHUNK) {
            const uint32_t n = (uint32_t)(rbytes - a < BULK_CHUNK ? rbytes - a : BULK_CHUNK);
            bulk_load(area + a, src + a, n, &mbar);
        }
    };
    // One thread takes a bucket: its bounds and element offset, the storage
    // decision, and the bulk copy of its records into the bottom of the area
    // when that fits below `limit` bytes (the part not in use); otherwise the
    // copy is issued once the current bucket is done.  A bucket is processed
    // in shared memory when its records, slots, groups, element rows and as
    // many neighbour entries as records fit the area.
    auto take = [&](int slot, uint32_t t, uint64_t limit) {
        BucketMeta M{};
        M.b = t;
        if (t < n_buckets) {
            M.r0 = p.bstart[t];
            M.r1 = p.bstart[t + 1];
            int64_t fb = 0;  // the bucket's mesh's first bucket (batches)
            if (batched) {
                int lo_m = 0, hi_m = n_meshes;
                while (hi_m - lo_m > 1) {
                    const int mid = (lo_m + hi_m) >> 1;
                    if (p.batch.bucket_off[mid] <= (int64_t)t) lo_m = mid;
                    else hi_m = mid;
                }
                fb = p.batch.bucket_off[lo_m];
            }
            M.ge = want_e ? (uint64_t)(p.estart[t] - p.estart[fb]) + (p.base ? (uint64_t)p.base[0] : 0ull) : 0;
            const uint64_t R = M.r1 - M.r0;
            const uint64_t rb = rec_bytes(R, RB == 8 ? (M.r0 & 1u) * 8u : 0u, RB);
            M.sr = p.rec_smem && rb + 3 * word_bytes(R) <= A;
#ifdef NN_CHECKED
            const bool rec_ok = M.r1 >= M.r0 && M.r1 <= p.rec_count;  // else the bucket reads nothing
            M.sr = M.sr && rec_ok;
#else
            constexpr bool rec_ok = true;
#endif
            if (M.sr && rb <= limit) {
                issue_copy(M);
                M.copied = 1;
            } else if (!M.sr && rec_ok) {
                // read from global memory: start pulling the records into L2
                uint64_t lo = (uint64_t)M.r0 * RB, hi = (uint64_t)M.r1 * RB;
                lo &= ~15ull;
                hi = (hi + 15) & ~15ull;  // the record array is padded to 256 bytes
                for (uint64_t a = lo; a < hi; a += BULK_CHUNK) {
                    const uint32_t n = (uint32_t)(hi - a < BULK_CHUNK ? hi - a : BULK_CHUNK);
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p.rec + a), "r"(n) : "memory");
                }
            }
        }
        meta[slot] = M;
    };

    if (tid == 0) {
        mbar_init(&mbar);
        take(0, atomicAdd(p.ticket, 1u), A);
    }
    __syncthreads();
    uint32_t phase = 0;  // parity of the mbarrier phase the next bulk copy completes
    for (int it = 0;; ++it) {
        const BucketMeta M = meta[it & 1];
        const int64_t b = M.b;
        if (b >= n_buckets) break;
        uint32_t nx = 0;
        if (tid == 0) {
            nx = atomicAdd(p.ticket, 1u);  // the next bucket (taken once this one's records are read)
            // the mesh this bucket belongs to (the only one unless batched)
            BucketOut o{p.n_nodes, 0, b == n_buckets - 1, p.rp_n, p.col_n, p.cap_n, p.rp_e, p.col_e, p.cap_e, p.status};
            if (batched) {
                int lo_m = 0, hi_m = n_meshes;  // largest m with bucket_off[m] <= b
                while (hi_m - lo_m > 1) {
                    const int mid = (lo_m + hi_m) >> 1;
                    if (p.batch.bucket_off[mid] <= b) lo_m = mid;
                    else hi_m = mid;
                }
                const BatchMesh& Mm = p.batch.meshes[lo_m];
                o = BucketOut{Mm.n_nodes, p.batch.bucket_off[lo_m], b == p.batch.bucket_off[lo_m + 1] - 1, Mm.rp_n,
                              Mm.col_n, Mm.cap_n, Mm.rp_e, Mm.col_e, Mm.cap_e, Mm.status};
                if (*p.batch_err) set_status(o.status, *p.batch_err);
            }
            sh_out = o;
            misc[6] = 0;
        }
        const uint32_t r0 = M.r0, R = M.r1 - M.r0;
        const uint32_t roff = RB == 8 ? (r0 & 1u) * 8u : 0u;
        const bool sr = M.sr != 0;
        const uint64_t rbytes = sr ? rec_bytes(R, roff, RB) : 0;  // records' part of the area
        // slots / element rows at the top, record groups below them: in the
        // area, or (a bucket too large) in the spill area
        const uint64_t sbytes = word_bytes(R);
        const bool top_in = sr || 2 * sbytes <= A;
        if (!top_in && tid == 0) {
            const uint64_t need = 2 * sbytes / 4;
            const uint64_t base = atomicAdd(p.spill_cursor, (unsigned long long)need);
            misc[2] = base;
            misc[4] = base + need <= p.spill_words;
            if (base + need > p.spill_words) set_status(sh_out.status, NN_ERR_WORKSPACE);
        }
        for (int l = tid; l < NB; l += THREADS) {
            c32[l] = 0;
            nfc[l] = 0;
        }
        if (tid < 64) gtot[tid] = 0;
        bool lost = false;
        if (sr) {
            lost = !mbar_wait(&mbar, phase);
            phase ^= 1u;
        }
        if (__syncthreads_or(lost)) {
            // the copy never completed: report it and stop (never observed;
            // the bounded wait only keeps a lost copy from hanging the GPU)
            if (tid == 0) set_status(sh_out.status, NN_ERR_TIMEOUT);
            return;
        }
#ifdef NN_CHECKED
        // the bucket's records lie inside the record array (else none is read)
        const bool recs_in = M.r1 >= M.r0 && NN_IN((uint64_t)M.r1, p.rec_count + 1, sh_out.status);
#else
        constexpr bool recs_in = true;
#endif
        const bool ok = (top_in || misc[4] != 0) && recs_in;
        uint32_t* const Est = top_in ? reinterpret_cast<uint32_t*>(area + A - sbytes) : p.spill + misc[2];
        uint32_t* const grp = top_in ? reinterpret_cast<uint32_t*>(area + A - 2 * sbytes) : Est + sbytes / 4;
        uint8_t* const ust_top = area + (top_in ? A - 2 * sbytes : A);  // neighbour rows grow down from here
        const uint64_t ucap = (uint64_t)(ust_top - area - rbytes) / 4;   // ... to the records' end (words)
        const uint8_t* const rp = sr ? area + roff : p.rec + (uint64_t)r0 * RB;
        const int64_t N = sh_out.n_nodes;
        int32_t* const status = sh_out.status;
        const int64_t v0 = (b - sh_out.first) << f.sb;
        const int nb = (int)(N - v0 < (int64_t)NB ? N - v0 : (int64_t)NB);

        // 1. records per node, each record's slot in its node (kept in the
        // element-row space), repeated-node records
        for (uint32_t r = tid; ok && r < R; r += THREADS) {
            const uint64_t lo = get_rec_lo<RB>(rp, r);
            const uint32_t vloc = (uint32_t)lo & vmask;
            Est[r] = atomicAdd(&c32[vloc], 1u);
            if (want_e && ((lo >> f.off_nf) & 1)) atomicAdd(&nfc[vloc], 1u);  // flag bit sb < 64
        }
        __syncthreads();
        for (int l = tid; l < NB; l += THREADS) cnt[l] = (uint64_t)c32[l] | ((uint64_t)(c32[l] - nfc[l]) << 32);
        __syncthreads();
        const uint64_t tot = smem_array_excl_scan(cnt, NB, sh_scan);  // packed: group offset | element offset
        const uint32_t Eb = (uint32_t)(tot >> 32);
        if (want_e && tid == 0 && ok && M.ge + Eb > (uint64_t)sh_out.cap_e) set_status(status, NN_ERR_CAPACITY);
        // 2. record indices grouped by node
        for (uint32_t r = tid; ok && r < R; r += THREADS) {
            const uint32_t vloc = (uint32_t)get_rec_lo<RB>(rp, r) & vmask;
            grp[(uint32_t)cnt[vloc] + Est[r]] = r;
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
            // 3a. element row: the element ids of the node's records (a
            // repeated node's record adds none), sorted in registers
            if (want_e) {
                const bool fast = valid && c <= (uint32_t)IMAX;
                const uint32_t cmax = __reduce_max_sync(FULL, fast ? c : 0u);
                uint32_t v[IMAX];
#pragma unroll
                for (int s = 0; s < IMAX; ++s) v[s] = EMPTY;
#pragma unroll
                for (int s0 = 0; s0 < IMAX; s0 += CH) {
                    if ((uint32_t)s0 >= cmax) break;
                    Rec xs[CH];
#pragma unroll
                    for (int q = 0; q < CH; ++q)
                        if (fast && (uint32_t)(s0 + q) < c) xs[q] = get_rec<RB>(rp, grp[goff + s0 + q]);
#pragma unroll
                    for (int q = 0; q < CH; ++q)
                        if (fast && (uint32_t)(s0 + q) < c && !rec_get(xs[q], f.off_nf, 1))
                            v[s0 + q] = rec_get(xs[q], f.off_e, f.eb);
                }
                sort_prefix(v, cmax);
                if (fast) {
#pragma unroll
                    for (int s = 0; s < IMAX; ++s)
                        if ((uint32_t)s < ecnt) Est[eoff + s] = v[s];
                }
                // nodes beyond the registers: the whole warp, in place
                for (unsigned m = __ballot_sync(FULL, valid && !fast); m; m &= m - 1) {
                    const int i = __ffs(m) - 1;
                    const uint32_t cc = __shfl_sync(FULL, c, i), go = __shfl_sync(FULL, goff, i);
                    const uint32_t eo = __shfl_sync(FULL, eoff, i), ec = __shfl_sync(FULL, ecnt, i);
                    warp_elem_row<RB>(rp, grp + go, cc, Est + eo, ec, f.off_nf, f.off_e, f.eb);
                }
            }
            if (!want_n) continue;

            // 3b. neighbour row
            const uint32_t cmax = __reduce_max_sync(FULL, valid ? c : 0u);
            // few candidates (K per record): straight into registers,
            // sorted, repeats skipped when written; else the lane's table
            const bool direct = (uint64_t)K * cmax <= 32u;
            constexpr int DMAX = 32 / K;  // records of a direct row
            uint32_t u = 0, nw = 0;
            bool ovf = valid && c > 4u * IMAX;  // very many records: the warp path at once
            uint32_t w[32];
#pragma unroll
            for (int s = 0; s < 32; ++s) w[s] = EMPTY;
            if (direct) {
#pragma unroll
                for (int s0 = 0; s0 < DMAX; s0 += CH) {
                    if ((uint32_t)s0 >= cmax) break;
                    Rec xs[CH];
#pragma unroll
                    for (int q = 0; q < CH; ++q)
                        if (s0 + q < DMAX && (uint32_t)(s0 + q) < c) xs[q] = get_rec<RB>(rp, grp[goff + s0 + q]);
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        if (s0 + q < DMAX && (uint32_t)(s0 + q) < c) {
#pragma unroll
                            for (int j = 0; j < K; ++j)
                                w[K * (s0 + q) + j] = rec_get(xs[q], f.off_n + j * f.nb, f.nb) - 1;  // 0 (none) -> EMPTY
                        }
                    }
                }
                nw = K * cmax;
                sort_prefix(w, nw);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if ((uint32_t)j >= nw) break;
                    u += w[j] != EMPTY && (j == 0 || w[j] != w[j - 1]);
                }
            } else {
#pragma unroll
                for (int h = 0; h < HT; ++h) tabw[h * 32] = EMPTY;
                for (uint32_t s = 0; valid && s < c && !ovf; ++s) {
                    const Rec x = get_rec<RB>(rp, grp[goff + s]);
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const uint32_t y = rec_get(x, f.off_n + j * f.nb, f.nb);
                        if (y && !ovf) ovf = !lane_insert<HT, UCAP>(tabw, y - 1, u);
                    }
                }
                // distinct values to the front of the table, then sorted
                // in registers (they are already free of repeats)
                uint32_t j = 0;
#pragma unroll
                for (int h = 0; h < HT; ++h) {
                    const uint32_t t = tabw[h * 32];
                    if (t != EMPTY) {
                        tabw[j * 32] = t;
                        ++j;
                    }
                }
                nw = __reduce_max_sync(FULL, ovf ? 0u : j);
#pragma unroll
                for (int h = 0; h < HT; ++h)
                    if ((uint32_t)h < j && !ovf) w[h] = tabw[h * 32];
                sort_prefix(w, nw);
            }

            // nodes beyond the table: the whole warp, in global scratch
            const unsigned slowU = __ballot_sync(FULL, valid && ovf);
            uint32_t uscr = 0;
            for (unsigned m = slowU; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                const uint32_t cc = __shfl_sync(FULL, c, i), go = __shfl_sync(FULL, goff, i);
                uint32_t so = 0;
                const uint32_t nu = warp_node_row<RB, K>(rp, grp + go, cc, p.spill, p.spill_words, p.spill_cursor,
                                                         status, f.off_n, f.nb, &so);
                if (lane == i) {
                    u = nu;
                    uscr = so;
                }
            }

            // the group's distinct-neighbour rows, contiguous in node order,
            // in a segment allocated downwards from ust_top (or spilled)
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
                    seg = (uint32_t)(s + gt);  // the segment ends seg words below ust_top
                } else {
                    const unsigned long long so = atomicAdd(p.spill_cursor, (unsigned long long)((gt + 3) & ~3u));
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
                uint32_t* sp = (seg & SEG_SPILL) ? p.spill + (seg & ~SEG_SPILL)
                                                 : reinterpret_cast<uint32_t*>(ust_top) - seg;
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
            if (valid) c32[l] = ex;
            if (lane == 0) {
                gseg[g] = seg;
                gtot[g] = seg == SEG_NONE ? 0u : gt;
            }
        }
        __syncthreads();
        // the records are dead: the next bucket (copied in below the rows
        // when it fits there)
        if (tid == 0) take((it + 1) & 1, nx, sr || top_in ? (uint64_t)(ust_top - area) - 4 * misc[6] : A);

        // 4. element rows to their offset; node rows, with each node's offset
        // within the bucket and the bucket's total, to the scratch area (their
        // offsets are placed by the compaction pass, so no bucket waits here)
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
            if (want_n && lane == 31 && NN_IN(b, p.ubk_words, status)) p.ubk[b] = s1;
        } else if (want_e) {
            const bool e_ok = ok && M.ge + Eb <= (uint64_t)sh_out.cap_e;
            for (int l = tid - 32; l < nb; l += THREADS - 32)
                if (NN_IN(v0 + l, N + 1, status)) sh_out.rp_e[v0 + l] = (int64_t)(M.ge + (uint32_t)(cnt[l] >> 32));
            if (e_ok) {
                int32_t* dst = sh_out.col_e + M.ge;
                for (uint32_t i = tid - 32; i < Eb; i += THREADS - 32) dst[i] = (int32_t)Est[i];
            }
        }
        __syncthreads();
        if (want_n) {
            uint32_t* const loc = p.nloc + ((size_t)b << f.sb);
            for (int l = tid; l < nb; l += THREADS)
                if (NN_IN(((size_t)b << f.sb) + l, p.nloc_words, status)) loc[l] = gpre[l >> 5] + c32[l];
            uint32_t* const rows = p.ntmp + (size_t)K * r0;
            for (int g = warp; ok && g < ng; g += W) {
                const uint32_t seg = gseg[g], n = gtot[g];
                if (seg == SEG_NONE) continue;
                if (n && !NN_IN((size_t)K * r0 + gpre[g] + n - 1, p.ntmp_words, status)) continue;
                const uint32_t* src = (seg & SEG_SPILL) ? p.spill + (seg & ~SEG_SPILL)
                                                        : reinterpret_cast<const uint32_t*>(ust_top) - seg;
                uint32_t* dst = rows + gpre[g];
                for (uint32_t i = lane; i < n; i += 32) dst[i] = src[i];
            }
        }
        if (sh_out.last && tid == 0 && want_e && NN_IN(N, N + 1, status)) sh_out.rp_e[N] = (int64_t)(M.ge + Eb);
        __syncthreads();
        // the next bucket's copy, if it did not fit beside this one's rows
        if (tid == 0 && meta[(it + 1) & 1].sr && !meta[(it + 1) & 1].copied) issue_copy(meta[(it + 1) & 1]);
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
