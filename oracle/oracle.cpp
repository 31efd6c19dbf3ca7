// CPU oracle for one-ring neighbor finding -- TEST INFRASTRUCTURE ONLY.
//
// Only tests, the smoke check and the CPU-baseline leg of the benchmark load
// this file's library; the product path never does.  It shares no code with
// the CUDA library: its own status numbers, its own edge tables, no headers.
//
// What it computes (Mei et al., "A Parallel Solution to Finding Nodal
// Neighbors in Generic Meshes", Sec. 1 and Sec. 2.1):
//   * neighbor nodes of v   = every node joined to v by an element edge
//                             (Sec. 2.1.1: an edge makes its two nodes
//                             neighbors of each other);
//   * neighbor elements of v = every element that contains v (Sec. 2.1.2).
// It follows the serial method the paper compares against (Sec. 1, loop over
// all elements; Sec. 3.2.2, one growable container per vertex), with ordered
// sets in place of vector<int> so each neighbor is listed once, ascending
// (readings of the paper: neighbors form a set; rows are emitted sorted).
//
// Edge tables (local node indices):
//   tri  {01,12,20}   quad {01,12,23,30}   tet: all six pairs
//   hex (VTK order, 0-3 bottom, 4-7 top) {01,12,23,30,45,56,67,74,04,15,26,37}
// For triangles, inserting both directions of each edge is the paper's
// "three CCW plus three CW pairs" per triangle (Sec. 2.2.1).
// An edge whose two ends are the same node (degenerate element) is dropped.
//
// Errors (first one met, in element order, is returned; the element is skipped):
//   4 node id outside [0, n_nodes)
//   5 mixed mesh: element type unknown, or elem_ptr range inconsistent with it
#include <cstdint>
#include <cstdlib>
#include <set>
#include <vector>
#include <unordered_map>
#include <algorithm>

namespace {

const int ST_OK = 0, ST_NODE_RANGE = 4, ST_ELEM_PTR = 5;
const int T_TRI = 0, T_QUAD = 1, T_TET = 2, T_HEX = 3, T_MIXED = 255;

struct EdgeTable { int npe; int ne; int e[12][2]; };

const EdgeTable TABLES[4] = {
    {3, 3, {{0, 1}, {1, 2}, {2, 0}}},
    {4, 4, {{0, 1}, {1, 2}, {2, 3}, {3, 0}}},
    {4, 6, {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}}},
    {8, 12, {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6}, {6, 7}, {7, 4},
             {0, 4}, {1, 5}, {2, 6}, {3, 7}}},
};

struct MeshIn {
    int32_t type; int64_t n_nodes, n_elems, n_conn;
    const int32_t* conn; const int64_t* elem_ptr; const uint8_t* elem_type;
};

// Calls visit_elem(e, type, nodes) for every valid element in array order.
// Returns the first error status met (elements with errors are skipped).
template <class F>
int for_each_element(const MeshIn& m, F visit_elem) {
    int status = ST_OK;
    for (int64_t e = 0; e < m.n_elems; ++e) {
        int t;
        const int32_t* nodes;
        if (m.type == T_MIXED) {
            int tt = m.elem_type[e];
            int64_t a = m.elem_ptr[e], b = m.elem_ptr[e + 1];
            if (tt < 0 || tt > 3 || a < 0 || b > m.n_conn || b - a != TABLES[tt].npe) {
                if (status == ST_OK) status = ST_ELEM_PTR;
                continue;
            }
            t = tt;
            nodes = m.conn + a;
        } else {
            t = m.type;
            nodes = m.conn + e * TABLES[t].npe;
        }
        bool ok = true;
        for (int i = 0; i < TABLES[t].npe; ++i)
            if (nodes[i] < 0 || nodes[i] >= m.n_nodes) ok = false;
        if (!ok) {
            if (status == ST_OK) status = ST_NODE_RANGE;
            continue;
        }
        visit_elem(e, t, nodes);
    }
    return status;
}

struct Result {
    int status = ST_OK;
    std::vector<int64_t> node_row_ptr, elem_row_ptr;
    std::vector<int32_t> node_col, elem_col;
};

void emit(const std::vector<std::set<int32_t>>& sets, std::vector<int64_t>& rp,
          std::vector<int32_t>& col) {
    rp.assign(sets.size() + 1, 0);
    for (size_t v = 0; v < sets.size(); ++v) rp[v + 1] = rp[v] + (int64_t)sets[v].size();
    col.clear();
    col.reserve((size_t)rp.back());
    for (const auto& s : sets) col.insert(col.end(), s.begin(), s.end());
}

}  // namespace

extern "C" {

// Full build.  want: 1 nodes, 2 elements, 3 both.  Returns an opaque handle.
void* oracle_build(int32_t type, int64_t n_nodes, int64_t n_elems, int64_t n_conn,
                   const int32_t* conn, const int64_t* elem_ptr, const uint8_t* elem_type,
                   int want) {
    MeshIn m{type, n_nodes, n_elems, n_conn, conn, elem_ptr, elem_type};
    Result* r = new Result();
    std::vector<std::set<int32_t>> nn((want & 1) ? n_nodes : 0), ne((want & 2) ? n_nodes : 0);
    r->status = for_each_element(m, [&](int64_t e, int t, const int32_t* nodes) {
        const EdgeTable& tb = TABLES[t];
        if (want & 2)
            for (int i = 0; i < tb.npe; ++i) ne[nodes[i]].insert((int32_t)e);
        if (want & 1)
            for (int k = 0; k < tb.ne; ++k) {
                int32_t a = nodes[tb.e[k][0]], b = nodes[tb.e[k][1]];
                if (a == b) continue;
                nn[a].insert(b);
                nn[b].insert(a);
            }
    });
    if (want & 1) emit(nn, r->node_row_ptr, r->node_col);
    if (want & 2) emit(ne, r->elem_row_ptr, r->elem_col);
    return r;
}

int oracle_status(void* h) { return static_cast<Result*>(h)->status; }

// which: 1 node CSR, 2 element CSR.  Returns nnz (or -1 if not built).
int64_t oracle_nnz(void* h, int which) {
    Result* r = static_cast<Result*>(h);
    const auto& rp = which == 1 ? r->node_row_ptr : r->elem_row_ptr;
    return rp.empty() ? -1 : rp.back();
}

void oracle_copy(void* h, int which, int64_t* row_ptr, int32_t* col) {
    Result* r = static_cast<Result*>(h);
    const auto& rp = which == 1 ? r->node_row_ptr : r->elem_row_ptr;
    const auto& c = which == 1 ? r->node_col : r->elem_col;
    std::copy(rp.begin(), rp.end(), row_ptr);
    std::copy(c.begin(), c.end(), col);
}

void oracle_free(void* h) { delete static_cast<Result*>(h); }

// Rows of a sample of nodes only, by the same element walk (one pass over all
// elements, keeping only pairs whose key node is sampled).  Output is a CSR
// over the sample, in sample order.  Used to check full-size builds row by row.
void* oracle_rows(int32_t type, int64_t n_nodes, int64_t n_elems, int64_t n_conn,
                  const int32_t* conn, const int64_t* elem_ptr, const uint8_t* elem_type,
                  int want, const int32_t* sample, int64_t n_sample) {
    MeshIn m{type, n_nodes, n_elems, n_conn, conn, elem_ptr, elem_type};
    std::unordered_map<int32_t, int64_t> slot;
    slot.reserve((size_t)n_sample * 2);
    for (int64_t i = 0; i < n_sample; ++i) slot.emplace(sample[i], i);
    Result* r = new Result();
    std::vector<std::set<int32_t>> nn((want & 1) ? n_sample : 0), ne((want & 2) ? n_sample : 0);
    r->status = for_each_element(m, [&](int64_t e, int t, const int32_t* nodes) {
        const EdgeTable& tb = TABLES[t];
        if (want & 2)
            for (int i = 0; i < tb.npe; ++i) {
                auto it = slot.find(nodes[i]);
                if (it != slot.end()) ne[it->second].insert((int32_t)e);
            }
        if (want & 1)
            for (int k = 0; k < tb.ne; ++k) {
                int32_t a = nodes[tb.e[k][0]], b = nodes[tb.e[k][1]];
                if (a == b) continue;
                auto ia = slot.find(a);
                if (ia != slot.end()) nn[ia->second].insert(b);
                auto ib = slot.find(b);
                if (ib != slot.end()) nn[ib->second].insert(a);
            }
    });
    // duplicated sample entries share one row; copy it to every slot
    for (int64_t i = 0; i < n_sample; ++i) {
        int64_t j = slot[sample[i]];
        if (j != i) {
            if (want & 1) nn[i] = nn[j];
            if (want & 2) ne[i] = ne[j];
        }
    }
    if (want & 1) emit(nn, r->node_row_ptr, r->node_col);
    if (want & 2) emit(ne, r->elem_row_ptr, r->elem_col);
    return r;
}

// Element face adjacency (the element-to-element neighbours that Sec. 1 lists
// among the local connectivity a mesh code needs "for each node or element";
// the paper works out only the per-node neighbours).  Faces: tri and quad
// edges, tet triangles, hex (VTK) quads.  Elements e != f are face neighbours
// when every node of some face of one lies in the other (a face with a
// repeated node is no face).  For a conforming mesh this is the dual graph; a
// hex face split into two tet triangles borders both tets.  Plain definition:
// node -> element sets, then for every element each candidate sharing a node
// is tested face by face.  sample == NULL: all elements, else only the
// sampled ones (CSR over the sample, in sample order).
void* oracle_elem_adjacency(int32_t type, int64_t n_nodes, int64_t n_elems, int64_t n_conn,
                            const int32_t* conn, const int64_t* elem_ptr, const uint8_t* elem_type,
                            const int32_t* sample, int64_t n_sample) {
    static const int NF[4] = {3, 4, 4, 6};
    static const int FS[4] = {2, 2, 3, 4};
    static const int FACES[4][6][4] = {
        {{0, 1}, {1, 2}, {2, 0}},
        {{0, 1}, {1, 2}, {2, 3}, {3, 0}},
        {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}},
        {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}},
    };
    MeshIn m{type, n_nodes, n_elems, n_conn, conn, elem_ptr, elem_type};
    Result* r = new Result();
    // every valid element's type and nodes
    std::vector<int> et(n_elems, -1);
    std::vector<std::vector<int32_t>> en(n_elems);
    std::vector<std::set<int32_t>> ne(n_nodes);
    r->status = for_each_element(m, [&](int64_t e, int t, const int32_t* nodes) {
        et[e] = t;
        en[e].assign(nodes, nodes + TABLES[t].npe);
        for (int i = 0; i < TABLES[t].npe; ++i) ne[nodes[i]].insert((int32_t)e);
    });
    // some face of a lies in b
    auto face_in = [&](int64_t a, int64_t b) {
        const int t = et[a];
        for (int k = 0; k < NF[t]; ++k) {
            std::set<int32_t> face;
            for (int q = 0; q < FS[t]; ++q) face.insert(en[a][FACES[t][k][q]]);
            if ((int)face.size() < FS[t]) continue;  // repeated node: no face
            bool all = true;
            for (int32_t v : face)
                if (std::find(en[b].begin(), en[b].end(), v) == en[b].end()) all = false;
            if (all) return true;
        }
        return false;
    };
    const int64_t rows = sample ? n_sample : n_elems;
    std::vector<std::set<int32_t>> adj(rows);
    for (int64_t i = 0; i < rows; ++i) {
        const int64_t e = sample ? sample[i] : i;
        if (e < 0 || e >= n_elems || et[e] < 0) continue;
        for (int32_t v : en[e])
            for (int32_t f : ne[v])
                if (f != e && (face_in(e, f) || face_in(f, e))) adj[i].insert(f);
    }
    emit(adj, r->elem_row_ptr, r->elem_col);
    return r;
}

}  // extern "C"
