// Seeded synthetic grid generator on the device (input generation for the
// serving loop and benchmarks; not part of the neighbour-finding method).
//
// Reproduces paper_1604_04689_gb300/meshgen.py bit for bit: splitmix64
// (Steele, Lea and Flood, OOPSLA 2014, with the published constants) keyed by
// (seed, stream), node relabelling and element reordering by a 4-round
// Feistel network over the next even power of two with cycle walking, one
// seeded diagonal per triangle-grid quad, and the six Kuhn tetrahedra of each
// cube cell.  One thread per natural-order element.
#include <cstdint>

#include "nn_internal.h"

namespace nn {

namespace {

constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;
constexpr uint64_t ROUND_STEP = 0xD1B54A32D192ED03ull;
constexpr int STREAM_NODE_PERM = 1, STREAM_ELEM_PERM = 2, STREAM_DIAG = 3;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return splitmix64(splitmix64(seed) ^ (stream * GOLDEN));
}

struct Feistel {
    uint64_t n;
    int h;
    uint64_t mask;
    uint64_t rk[4];
};

__host__ inline Feistel make_feistel(uint64_t n, uint64_t key) {
    Feistel f{};
    f.n = n;
    int bits = 2;
    while (bits < 64 && n > 1 && ((n - 1) >> bits)) ++bits;
    f.h = (bits + 1) / 2;
    f.mask = (1ull << f.h) - 1;
    for (int r = 0; r < 4; ++r) f.rk[r] = splitmix64(key + (uint64_t)r * ROUND_STEP);
    return f;
}

__device__ __forceinline__ uint64_t feistel_enc(const Feistel& f, uint64_t v) {
    uint64_t L = v >> f.h, R = v & f.mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint64_t x = splitmix64(R ^ f.rk[r]) & f.mask;
        const uint64_t nl = R;
        R = L ^ x;
        L = nl;
    }
    return (L << f.h) | R;
}

// pi(x) for x in [0, n): encrypt, then walk the cycle until back inside [0, n)
// (the orbit of x returns to x, so the walk ends; expected < 4 steps).
__device__ __forceinline__ uint64_t feistel_perm(const Feistel& f, uint64_t x) {
    uint64_t y = feistel_enc(f, x);
    for (int guard = 0; y >= f.n && guard < (1 << 24); ++guard) y = feistel_enc(f, y);
    return y;
}

struct GenParams {
    int type;
    int64_t n;      // nodes per side
    int64_t m;      // cells per side
    int64_t n_nodes, n_elems;
    int permute_nodes, permute_elems;
    Feistel node_pi, elem_pi;
    uint64_t diag_key;
    int32_t* conn;
};

__global__ void k_gen(GenParams p) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n_elems) return;
    const int64_t n = p.n, m = p.m;
    int64_t nat[8];
    int npe;
    if (p.type == NN_TRI) {
        npe = 3;
        const int64_t q = t >> 1, i = q % m, j = q / m;
        const int64_t a = i + n * j, b = a + 1, c = a + 1 + n, d = a + n;
        const bool bit = (splitmix64((uint64_t)q ^ p.diag_key) & 1ull) != 0;
        if ((t & 1) == 0) { nat[0] = a; nat[1] = b; nat[2] = bit ? d : c; }
        else { nat[0] = bit ? b : a; nat[1] = c; nat[2] = d; }
    } else if (p.type == NN_QUAD) {
        npe = 4;
        const int64_t i = t % m, j = t / m, a = i + n * j;
        nat[0] = a; nat[1] = a + 1; nat[2] = a + 1 + n; nat[3] = a + n;
    } else {
        const int64_t ci = p.type == NN_TET ? t / 6 : t;
        const int64_t i = ci % m, j = (ci / m) % m, k = ci / (m * m);
        const int64_t base = i + n * j + n * n * k;
        const int64_t off[8] = {0, 1, 1 + n, n, n * n, n * n + 1, n * n + 1 + n, n * n + n};
        if (p.type == NN_HEX) {
            npe = 8;
            for (int q = 0; q < 8; ++q) nat[q] = base + off[q];
        } else {
            // Kuhn tets of a VTK-ordered cube: one per axis order, all on the 0-6 diagonal
            const int8_t kuhn[6][4] = {{0, 1, 2, 6}, {0, 1, 5, 6}, {0, 3, 2, 6}, {0, 3, 7, 6}, {0, 4, 5, 6}, {0, 4, 7, 6}};
            const int s = (int)(t % 6);
            npe = 4;
            for (int q = 0; q < 4; ++q) nat[q] = base + off[kuhn[s][q]];
        }
    }
    const int64_t pos = p.permute_elems ? (int64_t)feistel_perm(p.elem_pi, (uint64_t)t) : t;
    int32_t* out = p.conn + pos * npe;
    for (int q = 0; q < npe; ++q)
        out[q] = (int32_t)(p.permute_nodes ? feistel_perm(p.node_pi, (uint64_t)nat[q]) : (uint64_t)nat[q]);
}

}  // namespace

}  // namespace nn

extern "C" nn_status nn_generate_grid(int32_t type, int64_t n, uint64_t seed, int permute_nodes, int permute_elems,
                                      int32_t* conn, int64_t conn_capacity, int64_t* n_nodes, int64_t* n_elems,
                                      nn_stream_t stream) {
    using namespace nn;
    if (!(type == NN_TRI || type == NN_QUAD || type == NN_TET || type == NN_HEX) || n < 2 || n > (1 << 20))
        return NN_ERR_ARG;
    GenParams p{};
    p.type = type;
    p.n = n;
    p.m = n - 1;
    const bool d3 = type == NN_TET || type == NN_HEX;
    p.n_nodes = d3 ? n * n * n : n * n;
    const int64_t cells = d3 ? p.m * p.m * p.m : p.m * p.m;
    p.n_elems = type == NN_TRI ? 2 * cells : (type == NN_TET ? 6 * cells : cells);
    const int npe = type == NN_TRI ? 3 : (type == NN_HEX ? 8 : 4);
    if (n_nodes) *n_nodes = p.n_nodes;
    if (n_elems) *n_elems = p.n_elems;
    if (p.n_nodes >= (1ll << 31) || p.n_elems * npe >= (1ll << 31)) return NN_ERR_ARG;
    if (!conn) return conn_capacity < 0 ? NN_ERR_ARG : NN_OK;  // size query
    if (conn_capacity < p.n_elems * npe) return NN_ERR_CAPACITY;
    p.permute_nodes = permute_nodes;
    p.permute_elems = permute_elems;
    p.node_pi = make_feistel((uint64_t)p.n_nodes, stream_key(seed, STREAM_NODE_PERM));
    p.elem_pi = make_feistel((uint64_t)p.n_elems, stream_key(seed, STREAM_ELEM_PERM));
    p.diag_key = stream_key(seed, STREAM_DIAG);
    p.conn = conn;
    if (p.n_elems == 0) return NN_OK;
    k_gen<<<(unsigned)((p.n_elems + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(p);
    return cudaGetLastError() == cudaSuccess ? NN_OK : NN_ERR_CUDA;
}
