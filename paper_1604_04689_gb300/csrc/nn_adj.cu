// Element face adjacency from the node -> element CSR.
//
// Sec. 1 lists the neighbours of each element among the local connectivity a
// mesh code needs; the paper works out only the per-node ones.  Reading: two
// distinct elements are face neighbours when every node of some face of one
// of them belongs to the other (faces: tri and quad edges, tet triangles, hex
// quads in VTK order; a face with a repeated node is no face).  For a
// conforming mesh this is the dual graph; a hex face split into two tet
// triangles borders both tets.
//
// One thread per element merges the (sorted) element rows of its distinct
// nodes, which yields every element sharing a node with it once, in
// ascending order, with the number of shared nodes; the face tests run only
// where that number allows a shared face.  Three kernels: count, exclusive
// scan (decoupled lookback over tiles of elements), and write.
#include "nn_device.cuh"

namespace nn {

namespace {

constexpr int ADJ_THREADS = 256;
constexpr int ADJ_SCAN_THREADS = 128;

__constant__ int8_t c_nfaces[4] = {3, 4, 4, 6};
__constant__ int8_t c_fsize[4] = {2, 2, 3, 4};
__constant__ int8_t c_faces[4][6][4] = {
    {{0, 1}, {1, 2}, {2, 0}},
    {{0, 1}, {1, 2}, {2, 3}, {3, 0}},
    {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}},
    {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}},
};

// Type and nodes of element e (-1: invalid element, skipped).
__device__ __forceinline__ int load_element(const AdjParams& p, int64_t e, int32_t* nd) {
    int t = p.type;
    int64_t a;
    if (t == NN_MIXED) {
        t = p.elem_type[e];
        if (t > NN_HEX) return -1;
        a = p.elem_ptr[e];
        if (a < 0 || p.elem_ptr[e + 1] - a != npe_of(t) || p.elem_ptr[e + 1] > p.n_conn) return -1;
    } else {
        a = e * npe_of(t);
    }
    const int n = npe_of(t);
    for (int i = 0; i < n; ++i) {
        nd[i] = p.conn[a + i];
        if (nd[i] < 0 || (int64_t)nd[i] >= p.n_nodes) return -1;
    }
    return t;
}

__device__ __forceinline__ bool contains(const int32_t* nd, int n, int32_t v) {
    for (int i = 0; i < n; ++i)
        if (nd[i] == v) return true;
    return false;
}

// Some face of element a (type ta, nodes na) has all its nodes in b (nb nodes).
__device__ __forceinline__ bool face_in(int ta, const int32_t* na, const int32_t* nbd, int nb) {
    const int nf = c_nfaces[ta], fs = c_fsize[ta];
    for (int k = 0; k < nf; ++k) {
        bool ok = true;
        for (int q = 0; q < fs && ok; ++q) {
            const int32_t v = na[c_faces[ta][k][q]];
            for (int r = 0; r < q; ++r)
                if (na[c_faces[ta][k][r]] == v) ok = false;  // repeated node: no face
            if (ok && !contains(nbd, nb, v)) ok = false;
        }
        if (ok) return true;
    }
    return false;
}

// Calls emit(f) for every face neighbour f of element e, once each, in
// ascending order.  The element rows of e's distinct nodes are sorted, so a
// k-way merge of them visits every element sharing a node with e once and
// counts the nodes they share; only an element sharing at least as many nodes
// as the smallest face that could join them has its nodes gathered and the
// face tests run (a tet sees ~96 row entries but ~4 such candidates).
template <class F>
__device__ __forceinline__ void for_each_neighbour(const AdjParams& p, int64_t e, F&& emit) {
    constexpr int32_t END = 0x7fffffff;
    int32_t nd[8];
    const int t = load_element(p, e, nd);
    if (t < 0) return;
    const int n = npe_of(t);
    // one row per node slot (a repeated node, or a slot past the element, gets an empty one)
    int64_t pos[8], end[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        bool use = i < n;
#pragma unroll
        for (int j = 0; j < i; ++j) use = use && !(j < n && nd[j] == nd[i]);
        pos[i] = use ? p.ne_rp[nd[i]] : 0;
        end[i] = use ? p.ne_rp[nd[i] + 1] : 0;
    }
    int32_t head[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) head[i] = pos[i] < end[i] ? p.ne_col[pos[i]] : END;
    // any face of e, and any face of a neighbour of another type (2-node faces in a mixed mesh)
    const int dmin = p.type == NN_MIXED ? 2 : c_fsize[t];
    for (;;) {
        int32_t m = END;
#pragma unroll
        for (int j = 0; j < 8; ++j) m = min(m, head[j]);
        if (m == END) break;
        int shared = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (head[j] == m) {
                ++shared;
                ++pos[j];
                head[j] = pos[j] < end[j] ? p.ne_col[pos[j]] : END;
            }
        }
        if ((int64_t)m == e || shared < dmin || m < 0 || (int64_t)m >= p.n_elems) continue;
        int32_t fd[8];
        const int tf = load_element(p, m, fd);
        if (tf < 0) continue;
        if (face_in(t, nd, fd, npe_of(tf)) || face_in(tf, fd, nd, n)) emit(m);
    }
}

__global__ void __launch_bounds__(ADJ_THREADS) k_adj_count(AdjParams p) {
    for (int64_t e = (int64_t)blockIdx.x * ADJ_THREADS + threadIdx.x; e < p.n_elems;
         e += (int64_t)gridDim.x * ADJ_THREADS) {
        uint32_t c = 0;
        for_each_neighbour(p, e, [&](int32_t) { ++c; });
        p.cnt[e] = c;
    }
}

__global__ void __launch_bounds__(ADJ_SCAN_THREADS) k_adj_scan(AdjParams p) {
    __shared__ uint64_t sh_scan[33];
    __shared__ uint32_t sh_tile;
    __shared__ uint64_t sh_base;
    if (threadIdx.x == 0) sh_tile = atomicAdd(p.ticket, 1u);
    __syncthreads();
    const uint32_t tile = sh_tile;
    const int64_t e = (int64_t)tile * ADJ_SCAN_THREADS + threadIdx.x;
    const uint64_t x = e < p.n_elems ? p.cnt[e] : 0;
    uint64_t agg;
    const uint64_t ex = block_excl_scan(x, &agg, sh_scan);
    if (threadIdx.x < 32) {
        const uint64_t base = warp_lookback(p.lb_state, tile, agg, p.status);
        if (threadIdx.x == 0) sh_base = base;
    }
    __syncthreads();
    if (e < p.n_elems) p.rp[e] = (int64_t)(sh_base + ex);
    if (e == p.n_elems - 1) {
        p.rp[p.n_elems] = (int64_t)(sh_base + ex + x);
        if ((int64_t)(sh_base + ex + x) > p.cap) set_status(p.status, NN_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(ADJ_THREADS) k_adj_write(AdjParams p) {
    for (int64_t e = (int64_t)blockIdx.x * ADJ_THREADS + threadIdx.x; e < p.n_elems;
         e += (int64_t)gridDim.x * ADJ_THREADS) {
        const int64_t a = p.rp[e], n = p.rp[e + 1] - a;
        if (a + n > p.cap) continue;
        int32_t* row = p.col + a;
        int64_t k = 0;
        for_each_neighbour(p, e, [&](int32_t f) {
            if (k < n) row[k] = f;
            ++k;
        });
    }
}

}  // namespace

cudaError_t launch_adjacency(const AdjParams& p, int grid, cudaStream_t s) {
    if (p.n_elems <= 0) return cudaSuccess;
    k_adj_count<<<grid, ADJ_THREADS, 0, s>>>(p);
    const unsigned tiles = (unsigned)((p.n_elems + ADJ_SCAN_THREADS - 1) / ADJ_SCAN_THREADS);
    k_adj_scan<<<tiles, ADJ_SCAN_THREADS, 0, s>>>(p);
    k_adj_write<<<grid, ADJ_THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

size_t adjacency_scan_tiles(int64_t n_elems) { return (size_t)((n_elems + ADJ_SCAN_THREADS - 1) / ADJ_SCAN_THREADS); }

}  // namespace nn
