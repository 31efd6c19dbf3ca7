/* A plain C99 user of the C ABI (include/nn.h), built and run by
 * tests/test_c_consumer.py on a host without a GPU.  It uses only the
 * host-only calls: an offline sizing handle, workspace and capacity queries,
 * chunk slabs, tuning and status strings.  Prints one line per check and
 * exits non-zero on the first failure. */
#include <stdio.h>
#include <stdint.h>

#include "nn.h"

#define CHECK(cond, what)                           \
    do {                                            \
        if (!(cond)) {                              \
            fprintf(stderr, "FAILED: %s\n", what);  \
            return 1;                               \
        }                                           \
        printf("ok %s\n", what);                    \
    } while (0)

int main(void) {
    nn_handle* h = NULL;
    CHECK(nn_create_offline(&h, 152, 232448, 233472) == NN_OK && h != NULL, "offline handle");

    /* a 2048 x 2048 triangle grid, described only (the pointer is never read) */
    nn_mesh m;
    m.type = NN_TRI;
    m.n_nodes = 4194304;
    m.n_elems = 8380418;
    m.n_conn = 3 * m.n_elems;
    m.conn = (const int32_t*)(uintptr_t)(1u << 20);
    m.elem_ptr = NULL;
    m.elem_type = NULL;

    size_t ws = 0;
    int64_t node_cap = 0, elem_cap = 0;
    CHECK(nn_query(h, &m, NN_WANT_BOTH, &ws, &node_cap, &elem_cap) == NN_OK, "query");
    CHECK(node_cap == 6 * m.n_elems && elem_cap == m.n_conn, "capacity bounds");
    CHECK(ws > (size_t)m.n_conn * 8, "workspace holds the records");
    printf("workspace %zu bytes, node col %lld, elem col %lld\n", ws, (long long)node_cap, (long long)elem_cap);

    int64_t info[9];
    CHECK(nn_plan_info(h, &m, NN_WANT_BOTH, info, 9) == NN_OK, "plan info");
    CHECK(((info[1] - 1) << info[0]) < m.n_nodes && m.n_nodes <= (info[1] << info[0]), "buckets cover the nodes");

    nn_tuning t = {8, 128, 4};
    CHECK(nn_set_tuning(h, &t) == NN_OK, "tuning");
    CHECK(nn_plan_info(h, &m, NN_WANT_BOTH, info, 1) == NN_OK && info[0] == 8, "tuned bucket width");
    CHECK(nn_set_tuning(h, NULL) == NN_OK, "tuning reset");

    int shift = -1, n_slabs = -1;
    CHECK(nn_chunk_slabs(&m, &shift, &n_slabs) == NN_OK && n_slabs <= NN_CHUNK_SLABS_MAX, "chunk slabs");
    CHECK(((int64_t)(n_slabs - 1) << shift) < m.n_nodes, "slabs cover the nodes");

    nn_mesh bad = m;
    bad.type = 7;
    CHECK(nn_query(h, &bad, NN_WANT_BOTH, &ws, NULL, NULL) == NN_ERR_ARG, "bad type refused");
    CHECK(nn_neighbors_both(h, &m, NULL, NULL, NULL, 0, NULL, NULL) == NN_ERR_ARG, "offline handle refuses compute");
    printf("status text: %s\n", nn_status_str(NN_ERR_NODE_RANGE));

    nn_destroy(h);
    return 0;
}
