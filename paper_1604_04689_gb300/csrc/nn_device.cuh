// Device helpers shared by the libnn kernels: status reporting, bounded
// decoupled lookback, block scans, record packing and element edge tables.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "nn_internal.h"

namespace nn {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
// A bounded wait gives up after this long without progress (ns).
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

__device__ __forceinline__ void set_status(int32_t* st, int32_t code) { atomicCAS(st, 0, code); }

// Bounds-checked build (compiled with -DNN_CHECKED into libnn_checked.so):
// NN_IN(i, n, status) is false when index i lies outside a buffer of n
// elements, after recording NN_ERR_BOUNDS; the caller then skips the access.
// In the ordinary build it is the constant true and costs nothing.
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n, int32_t* st) {
    if (i < n) return true;
    set_status(st, NN_ERR_BOUNDS);
    return false;
}
#ifdef NN_CHECKED
#define NN_IN(i, n, st) (::nn::in_bounds((uint64_t)(i), (uint64_t)(n), (st)))
#else
#define NN_IN(i, n, st) true
#endif

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- lookback
// Single-pass scan across tiles taken in ticket order.  Word layout: bits
// 62-63 flag (0 not ready, 1 tile aggregate, 2 inclusive prefix), bits 0-61
// the value.  Every predecessor of a tile holds an earlier ticket, so it is
// running or done; the wait is still bounded and reports NN_ERR_TIMEOUT.
constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_VAL = (1ull << 62) - 1;

// Warp-parallel lookback in two halves.  lb_publish (one thread) makes the
// tile's aggregate visible as soon as it is known; lb_resolve (all 32 lanes
// of one warp, possibly much later) walks back over the predecessors, 32 at
// a time, consuming the ready ones nearest to t and stopping at the first
// inclusive prefix, then publishes t's inclusive prefix.  Only the nearest
// not-yet-ready predecessor is ever waited for.
// `first` is the first tile of t's chain (a batch restarts the scan at every
// mesh): tiles before it count as an inclusive zero.
__device__ __forceinline__ void lb_publish(uint64_t* state, uint64_t t, uint64_t agg, uint64_t first = 0) {
    st_release(&state[t], (t == first ? LB_INC : LB_AGG) | agg);
}

__device__ inline uint64_t lb_resolve(uint64_t* state, uint64_t t, uint64_t agg, int32_t* status,
                                      uint64_t first = 0) {
    const int lane = threadIdx.x & 31;
    if (t == first) return 0;
    uint64_t excl = 0;
    int64_t p = (int64_t)t - 1;
    uint64_t t0 = 0;
    for (;;) {
        const int64_t idx = p - lane;
        const uint64_t s = idx >= (int64_t)first ? ld_acquire(&state[idx]) : LB_INC;  // before the chain: zero
        const unsigned not_ready = __ballot_sync(0xffffffffu, (s >> 62) == 0);
        const int k = not_ready ? __ffs(not_ready) - 1 : 32;  // lanes 0..k-1 are ready
        const unsigned ready_mask = k == 32 ? 0xffffffffu : ((1u << k) - 1);
        const unsigned inc = __ballot_sync(0xffffffffu, (s >> 62) == 2) & ready_mask;
        const int stop = inc ? __ffs(inc) - 1 : k - 1;
        uint64_t v = lane <= stop ? (s & LB_VAL) : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        excl += v;
        if (inc) break;
        p -= k;
        if (k == 0) {  // nearest predecessor not ready yet: bounded wait
            const uint64_t now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > WAIT_LIMIT_NS) {
                if (lane == 0) set_status(status, NN_ERR_TIMEOUT);
                break;
            }
            __nanosleep(100);
        } else {
            t0 = 0;
        }
    }
    if (lane == 0) st_release(&state[t], LB_INC | ((excl + agg) & LB_VAL));
    __syncwarp();
    return excl;
}

__device__ inline uint64_t warp_lookback(uint64_t* state, uint64_t t, uint64_t agg, int32_t* status) {
    if ((threadIdx.x & 31) == 0) lb_publish(state, t, agg);
    __syncwarp();
    return lb_resolve(state, t, agg, status);
}

// ------------------------------------------------------------ block scans
// Exclusive scan of one 64-bit value per thread; *total gets the block sum.
// `sh` needs 33 words.  All threads must call.
__device__ inline uint64_t block_excl_scan(uint64_t x, uint64_t* total, uint64_t* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    uint64_t v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += y;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < nw) sh[lane] = w;
        if (lane == 31) sh[32] = w;
    }
    __syncthreads();
    uint64_t r = v - x + (warp > 0 ? sh[warp - 1] : 0);
    *total = sh[32];
    __syncthreads();
    return r;
}

// Exclusive scan in place of a shared array of n 64-bit values; returns the sum.
__device__ inline uint64_t smem_array_excl_scan(uint64_t* a, int n, uint64_t* sh) {
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    uint64_t s = 0;
    for (int i = lo; i < hi; ++i) s += a[i];
    uint64_t total;
    uint64_t run = block_excl_scan(s, &total, sh);
    for (int i = lo; i < hi; ++i) {
        uint64_t t = a[i];
        a[i] = run;
        run += t;
    }
    __syncthreads();
    return total;
}

// --------------------------------------------------------------- records
struct Rec {
    uint64_t lo, hi;
};

__device__ __forceinline__ void rec_put(Rec& r, uint64_t val, int off) {  // val < 2^32
    if (off < 64) {
        r.lo |= val << off;
        if (off > 32) r.hi |= val >> (64 - off);
    } else {
        r.hi |= val << (off - 64);
    }
}
// Field of `width` <= 32 bits at bit `off` of the 128-bit record (no field
// crosses bit 128).  Branch-free: the field starts in 32-bit word off / 32
// and a funnel shift takes it across into the next word.
__device__ __forceinline__ uint32_t rec_get(const Rec& r, int off, int width) {
    const uint32_t w0 = (uint32_t)r.lo, w1 = (uint32_t)(r.lo >> 32), w2 = (uint32_t)r.hi, w3 = (uint32_t)(r.hi >> 32);
    const int q = off >> 5;
    const uint32_t a = q == 0 ? w0 : (q == 1 ? w1 : (q == 2 ? w2 : w3));
    const uint32_t b = q == 0 ? w1 : (q == 1 ? w2 : (q == 2 ? w3 : 0u));
    const uint32_t v = __funnelshift_r(a, b, (uint32_t)off & 31u);
    return width >= 32 ? v : v & ((1u << width) - 1u);
}

// ------------------------------------------------ element local edge tables
// Edge-neighbors of local node i (the other end of each local edge at i).
// tri: the two others; quad: the two cyclic neighbours; tet: the three others;
// hex (VTK): the two cyclic neighbours in i's face plus the node across.
template <int TYPE>
struct ElemT;
template <>
struct ElemT<NN_TRI> {
    static constexpr int NPE = 3, K = 2;
    __device__ static int nbr(int i, int s) { return (i + 1 + s) % 3; }
};
template <>
struct ElemT<NN_QUAD> {
    static constexpr int NPE = 4, K = 2;
    __device__ static int nbr(int i, int s) { return (i + (s ? 3 : 1)) & 3; }
};
template <>
struct ElemT<NN_TET> {
    static constexpr int NPE = 4, K = 3;
    __device__ static int nbr(int i, int s) { return (i + 1 + s) & 3; }
};
template <>
struct ElemT<NN_HEX> {
    static constexpr int NPE = 8, K = 3;
    __device__ static int nbr(int i, int s) {
        return s == 2 ? (i ^ 4) : ((i & 4) | ((i + (s ? 3 : 1)) & 3));
    }
};

__device__ __forceinline__ int npe_of(int t) { return t == NN_TRI ? 3 : (t == NN_HEX ? 8 : 4); }
__device__ __forceinline__ int nbr_of(int t, int i, int s) {
    switch (t) {
        case NN_TRI: return ElemT<NN_TRI>::nbr(i, s);
        case NN_QUAD: return ElemT<NN_QUAD>::nbr(i, s);
        case NN_TET: return ElemT<NN_TET>::nbr(i, s);
        default: return ElemT<NN_HEX>::nbr(i, s);
    }
}
__device__ __forceinline__ int k_of(int t) { return (t == NN_TRI || t == NN_QUAD) ? 2 : 3; }
// The node at the far end of local edge s at local node i of an element of
// run-time type t, read from the element's nodes nd[0..8).  Called with i and
// s fixed by unrolled loops, every index below is a compile-time constant, so
// nd stays in registers (an index computed at run time, as nbr_of gives,
// would put the array in local memory).  Every index is below 8.
__device__ __forceinline__ int32_t nbr_node(int t, const int32_t* nd, int i, int s) {
    switch (t) {
        case NN_TRI: return nd[ElemT<NN_TRI>::nbr(i, s)];
        case NN_QUAD: return nd[ElemT<NN_QUAD>::nbr(i, s)];
        case NN_TET: return nd[ElemT<NN_TET>::nbr(i, s)];
        default: return nd[ElemT<NN_HEX>::nbr(i, s)];
    }
}

}  // namespace nn
