/*
 * nn.h -- one-ring neighbor nodes and neighbor elements of generic meshes,
 * built on an NVIDIA GB300 (sm_103a).  C ABI of libnn.so.
 *
 * The operation (Mei et al., "A Parallel Solution to Finding Nodal Neighbors
 * in Generic Meshes", Sec. 1 and Sec. 2.1):
 *   - the neighbor NODES of node v are the nodes joined to v by an element
 *     edge (Sec. 2.1.1; each edge makes its two nodes neighbors of each other);
 *   - the neighbor ELEMENTS of v are the elements that contain v (Sec. 2.1.2).
 * Both are returned as canonical CSR over all n_nodes nodes: row_ptr int64
 * [n_nodes+1] with row_ptr[0] = 0, col int32, each row strictly ascending
 * (a set: no repeats, no self entry).  Nodes that no element touches have
 * empty rows.  An edge whose two ends are the same node is ignored.
 *
 * Element types and their local edge tables (local node indices):
 *   NN_TRI  (3 nodes)  01 12 20
 *   NN_QUAD (4 nodes)  01 12 23 30          (diagonals are not edges)
 *   NN_TET  (4 nodes)  all six pairs
 *   NN_HEX  (8 nodes, VTK order: 0-3 bottom face, 4-7 top face, i above i-4)
 *                      01 12 23 30 45 56 67 74 04 15 26 37
 *   NN_MIXED           per-element type in elem_type[], nodes of element e at
 *                      conn[elem_ptr[e] .. elem_ptr[e+1])
 * Element ids are positions in the element list (0-based); node ids are
 * 0-based and must lie in [0, n_nodes).
 *
 * Memory and streams.  Every pointer in nn_mesh / nn_csr and the workspace
 * are DEVICE pointers owned by the caller.  Compute calls only enqueue work
 * on `stream` and return; nothing synchronises.  The library allocates no
 * device memory on these paths (all scratch lives in the caller's workspace).
 *
 * Errors.  A call returns a host status for errors it can see without
 * touching the device (bad arguments, workspace too small).  Errors found on
 * the device are written to *d_status (device int32; the call first sets it
 * to 0): node id out of range, inconsistent elem_ptr/elem_type, output
 * capacity exceeded, spill workspace exhausted, or a bounded wait that timed
 * out.  Kernels never trap; output contents are unspecified when *d_status
 * is not NN_OK.  The number of entries written is row_ptr[n_nodes].
 *
 * Limits of this version: n_nodes, n_elems and n_conn each < 2^31; conn
 * 16-byte aligned; the packed per-incidence record (see nn_query) must fit
 * 128 bits, which holds for meshes up to roughly 2^27 nodes and elements.
 */
#ifndef NN_H
#define NN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the CUDA runtime's stream handle); 0 = legacy default stream. */
typedef struct CUstream_st* nn_stream_t;

typedef enum { NN_TRI = 0, NN_QUAD = 1, NN_TET = 2, NN_HEX = 3, NN_MIXED = 255 } nn_elem_type;

typedef enum {
    NN_OK = 0,
    NN_ERR_ARG = 1,        /* null/misaligned pointer, bad type, size out of range  */
    NN_ERR_WORKSPACE = 2,  /* ws_bytes below nn_query's minimum (host), or the spill
                              part of the workspace ran out (device)                 */
    NN_ERR_CAPACITY = 3,   /* an output col buffer is smaller than the result        */
    NN_ERR_NODE_RANGE = 4, /* a node id outside [0, n_nodes) (device)                */
    NN_ERR_ELEM_PTR = 5,   /* mixed mesh: unknown type or elem_ptr range of the wrong
                              length / outside conn (device)                         */
    NN_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up (device)            */
    NN_ERR_BUDGET = 7,     /* serving layer: request larger than the memory budget   */
    NN_ERR_CUDA = 8,       /* a CUDA launch or driver call failed                    */
    NN_ERR_BOUNDS = 9      /* a bounds-checked build (libnn_checked.so) found an index
                              outside its buffer and skipped the access (device)     */
} nn_status;

/* want flags */
#define NN_WANT_NODES 1
#define NN_WANT_ELEMS 2
#define NN_WANT_BOTH 3

typedef struct {
    int32_t type;              /* nn_elem_type                                        */
    int64_t n_nodes;           /* rows of the result                                  */
    int64_t n_elems;           /* elements                                            */
    int64_t n_conn;            /* length of conn (n_elems * nodes-per-element unless
                                  NN_MIXED)                                           */
    const int32_t* conn;       /* device, int32 node ids, 16-byte aligned             */
    const int64_t* elem_ptr;   /* device, [n_elems+1], NN_MIXED only (else NULL)      */
    const uint8_t* elem_type;  /* device, [n_elems], NN_MIXED only (else NULL)        */
} nn_mesh;

typedef struct {
    int64_t* row_ptr;          /* device, int64 [n_nodes+1]                           */
    int32_t* col;              /* device, int32 [col_capacity]                        */
    int64_t col_capacity;      /* entries available in col                            */
} nn_csr;

typedef struct nn_handle nn_handle;

/* Create a handle bound to the current CUDA device (reads its SM count and
 * shared-memory limits; holds launch tuning).  Host allocation only. */
nn_status nn_create(nn_handle** h);
void nn_destroy(nn_handle* h);

/* A handle for sizing and planning only, on a host with or without a GPU:
 * nn_query, nn_plan_info, nn_chunk_plan, nn_batch_query and
 * nn_element_neighbors_query size for a device with `sms` SMs, `smem_optin`
 * bytes of opt-in shared memory per block and `smem_per_sm` per SM (a GB300:
 * 152, 232448, 233472).  Compute calls return NN_ERR_ARG on it.  Host
 * allocation only; free with nn_destroy. */
nn_status nn_create_offline(nn_handle** h, int32_t sms, int32_t smem_optin, int32_t smem_per_sm);

/* Host-only sizing for a mesh (no device access).  want = NN_WANT_*.
 * *ws_bytes: workspace that a compute call needs (the minimum plus a spill
 * area sized for meshes of ordinary valence; meshes with a few nodes of very
 * high valence may need more, reported as NN_ERR_WORKSPACE on the device).
 * *node_col_cap / *elem_col_cap: upper bounds on the result sizes (the sum
 * of local edge ends over all elements, and n_conn).  Any pointer may be NULL. */
nn_status nn_query(nn_handle* h, const nn_mesh* mesh, int want, size_t* ws_bytes,
                   int64_t* node_col_cap, int64_t* elem_col_cap);

/* Launch tuning held by a handle, applied to its later calls (0 = the
 * library's automatic choice).  sb: log2 of the bucket width in nodes (4..11);
 * bucket_threads: 128 or 256 threads per bucket CTA; bucket_ctas_per_sm: 1..8
 * bucket CTAs sharing an SM (sets the shared memory per CTA, which caps the
 * bucket width).  Results never depend on tuning, only speed and workspace size.
 * nn_set_tuning(h, NULL) restores the automatic choice. */
typedef struct {
    int32_t sb;
    int32_t bucket_threads;
    int32_t bucket_ctas_per_sm;
} nn_tuning;
nn_status nn_set_tuning(nn_handle* h, const nn_tuning* tuning);

/* Element face adjacency (the neighbours "for each element" that Sec. 1
 * lists beside the per-node ones; the paper works out only the latter).
 * Two distinct elements are face neighbours when every node of some face of
 * one of them belongs to the other.  Faces are tri and quad edges, tet
 * triangles and hex quads (VTK order); a face with a repeated node is no
 * face.  For a conforming mesh this is the dual graph; a hex face split into
 * two tet triangles borders both tets.
 * node_elems: the mesh's node -> element CSR on the device (as built by
 * nn_neighbor_elements or nn_neighbors_both; col_capacity is not used).
 * out: row_ptr [n_elems+1] int64 and col, rows ascending; NN_ERR_CAPACITY on
 * the device if col_capacity is too small (nn_element_neighbors_query gives
 * a bound that holds when every face borders at most two elements of each
 * side).  Workspace: nn_element_neighbors_query.  Asynchronous on stream;
 * elements with invalid nodes or offsets are skipped (the neighbour build
 * reports them). */
nn_status nn_element_neighbors_query(nn_handle* h, const nn_mesh* mesh, size_t* ws_bytes, int64_t* col_cap);
nn_status nn_element_neighbors(nn_handle* h, const nn_mesh* mesh, const nn_csr* node_elems, nn_csr* out,
                               void* ws, size_t ws_bytes, int32_t* d_status, nn_stream_t stream);

/* Parameters of the build plan for a mesh (host-only; for tooling and
 * traffic accounting).  Fills up to n of: info[0] bucket shift (a bucket is
 * 2^info[0] consecutive node ids), [1] number of buckets, [2] CTAs of the
 * element walk, [3] bytes per incidence record, [4] minimum workspace bytes,
 * [5] CTAs of the bucket pass, [6] threads per bucket CTA, [7] shared memory
 * per bucket CTA, [8] partition mode (-1 scattered, 0 one sorted pass, k > 0
 * coarse + fine sorted passes with 2^k buckets per coarse region). */
nn_status nn_plan_info(nn_handle* h, const nn_mesh* mesh, int want, int64_t* info, int n);

/* Neighbor nodes of every node (Sec. 2.1.1, Sec. 2.2.1) into *out. */
nn_status nn_neighbor_nodes(nn_handle* h, const nn_mesh* mesh, nn_csr* out, void* ws,
                            size_t ws_bytes, int32_t* d_status, nn_stream_t stream);

/* Neighbor elements of every node (Sec. 2.1.2, Sec. 2.2.2) into *out. */
nn_status nn_neighbor_elements(nn_handle* h, const nn_mesh* mesh, nn_csr* out, void* ws,
                               size_t ws_bytes, int32_t* d_status, nn_stream_t stream);

/* Both results from one pass over the connectivity (shares the element walk). */
nn_status nn_neighbors_both(nn_handle* h, const nn_mesh* mesh, nn_csr* nodes, nn_csr* elems,
                            void* ws, size_t ws_bytes, int32_t* d_status, nn_stream_t stream);

/* ------------------------------------------------------- chunked builds
 * The same results as nn_neighbor_nodes / nn_neighbor_elements /
 * nn_neighbors_both (want = NN_WANT_*) with a workspace of the caller's
 * chosen size, for meshes whose whole-mesh workspace would not fit.  The
 * paper names its extra device memory as the method's shortcoming and its
 * future work (Sec. 3.2.2, Sec. 4).  The nodes are cut into chunks of
 * consecutive ids; each chunk is built in turn, walking all elements but
 * keeping only its own nodes' incidences, into its rows of the caller's
 * CSRs.  Peak workspace follows the largest chunk, not the mesh.
 *
 * Three steps:
 *  1. nn_chunk_count (device, asynchronous): incidences per node slab.  A
 *     slab is 2^shift consecutive node ids; nn_chunk_slabs gives shift and
 *     the slab count (<= NN_CHUNK_SLABS_MAX).  d_counts: device uint32
 *     [n_slabs], overwritten.  d_status: set to 0, then any node-range or
 *     elem_ptr error.
 *  2. nn_chunk_plan (host only): group consecutive slabs into chunks whose
 *     workspace, including the spill area nn_query would add, fits ws_bytes.
 *     counts: the slab counts, copied to the host.  Fills chunks[0 ..
 *     max_chunks) and *n_chunks.  *ws_needed (may be NULL) is the smallest
 *     workspace that admits a plan (the largest single slab).  Errors:
 *     NN_ERR_WORKSPACE when ws_bytes is below that; NN_ERR_CAPACITY when
 *     more than max_chunks chunks are needed (*n_chunks says how many);
 *     NN_ERR_ARG when the counts sum above n_conn.
 *  3. nn_neighbors_chunked (device, asynchronous): build the chunks in
 *     order on `stream`.  The chunks must tile [0, n_nodes) in order; their
 *     boundaries need not fall on slabs (nn_chunk_query sizes any chunk).
 *     Each one's records must be the incidence count of its nodes.
 *     Wrong counts give NN_ERR_WORKSPACE on the device, not a bad write.
 *     ws: device memory, 256-byte aligned, at least the plan's ws_bytes.
 *     Its first 256 bytes hold the running CSR offsets between chunks.
 * The mesh and output pointers may also be host memory the GPU can address:
 * pinned (cudaHostAlloc / cudaHostRegister), or pageable on a system that
 * reports pageable memory access.  That is an out-of-core build, with only
 * the workspace in device memory.  ws and d_status must be device memory.
 * The chunks' results equal the single build's bit for bit. */
#define NN_CHUNK_SLABS_MAX 4096
typedef struct {
    int64_t node_lo, node_hi;  /* nodes [node_lo, node_hi) */
    int64_t records;           /* incidences of those nodes (sum of their slabs' counts) */
} nn_chunk;
nn_status nn_chunk_slabs(const nn_mesh* mesh, int* shift, int* n_slabs);
nn_status nn_chunk_count(nn_handle* h, const nn_mesh* mesh, uint32_t* d_counts, int32_t* d_status,
                         nn_stream_t stream);
nn_status nn_chunk_plan(nn_handle* h, const nn_mesh* mesh, int want, const uint32_t* counts, size_t ws_bytes,
                        nn_chunk* chunks, int max_chunks, int* n_chunks, size_t* ws_needed);
/* Host only: the workspace one chunk needs in nn_neighbors_chunked.  That is
 * 256 bytes of running offsets plus what nn_query would give for the chunk's
 * nodes and records.  For callers that choose their own node ranges. */
nn_status nn_chunk_query(nn_handle* h, const nn_mesh* mesh, int want, const nn_chunk* chunk, size_t* ws_bytes);
nn_status nn_neighbors_chunked(nn_handle* h, const nn_mesh* mesh, int want, const nn_chunk* chunks, int n_chunks,
                               nn_csr* nodes, nn_csr* elems, void* ws, size_t ws_bytes, int32_t* d_status,
                               nn_stream_t stream);

/* ------------------------------------------------------------- batches
 * Many meshes of any types, each with its own outputs, built by ONE launch
 * sequence (batch init, histogram, offsets, partition, bucket pass) over the
 * disjoint union of the meshes: every mesh owns a contiguous range of node
 * buckets and its CSRs are mesh-local (row_ptr from 0, local node and element
 * ids).  The batch's description is written by nn_batch_prepare into HOST
 * staging memory that the caller owns (pinned, so the copy is asynchronous
 * and can be captured), and nn_batch_launch copies it to the workspace and
 * enqueues the kernels, whose grids depend only on the capacities: one CUDA
 * graph captured around nn_batch_launch replays for every batch prepared into
 * the same staging buffer with the same capacities and workspace.
 * Results equal those of nn_neighbors_both on each mesh alone. */
typedef struct {
    int32_t max_meshes;  /* meshes per batch                                      */
    int32_t want;        /* NN_WANT_*                                             */
    int64_t max_elems;   /* elements of all meshes of a batch                     */
    int64_t max_nodes;   /* nodes of all meshes of a batch                        */
    int64_t max_conn;    /* connectivity entries of all meshes of a batch         */
    int32_t sb;          /* log2 of the bucket width in nodes (0 = default, 4..11) */
} nn_batch_caps;

/* Sizes for a capacity: workspace bytes (device) and staging bytes (host). */
nn_status nn_batch_query(nn_handle* h, const nn_batch_caps* caps, size_t* ws_bytes, size_t* staging_bytes);

/* Host only: validate the meshes and write the batch description into
 * `staging`.  node_out / elem_out are arrays of n_meshes CSRs (either may be
 * NULL if not wanted); d_status is a device array of n_meshes status words
 * (mesh m's device-detected errors go to d_status[m]).  The caller must not
 * rewrite `staging` while a launch that reads it may still be pending. */
nn_status nn_batch_prepare(nn_handle* h, const nn_batch_caps* caps, const nn_mesh* meshes,
                           const nn_csr* node_out, const nn_csr* elem_out, int32_t* d_status, int n_meshes,
                           void* staging, size_t staging_bytes);

/* Enqueue the batch described in `staging` on `stream` (no host sync). */
nn_status nn_batch_launch(nn_handle* h, const nn_batch_caps* caps, const void* staging, void* ws,
                          size_t ws_bytes, nn_stream_t stream);

/* One-call batch (the same results as the three calls above), for callers
 * that do not capture graphs.  Builds the n_meshes meshes into their own
 * outputs with one launch sequence.  The wanted results are the non-NULL
 * ones of node_out / elem_out (arrays of n_meshes CSRs; at least one must be
 * given).  The capacity is the meshes' own totals: size ws with
 * nn_batch_submit_query for the same meshes and want.  ws: device memory,
 * 256-byte aligned.  d_status: device int32[n_meshes], one status word per
 * mesh, as in nn_batch_prepare.  The batch description is staged in host
 * memory that the call allocates; the stream frees it after the batch has
 * run (a host function enqueued on `stream`).  So the call is asynchronous
 * but cannot be captured in a CUDA graph: use nn_batch_prepare /
 * nn_batch_launch for that; a stream that is capturing is refused with
 * NN_ERR_ARG.  n_meshes == 0 enqueues nothing.  Host errors:
 * NN_ERR_ARG (bad mesh or pointers, no output wanted), NN_ERR_WORKSPACE
 * (ws_bytes below the minimum), NN_ERR_BUDGET (host memory for the staging
 * exhausted), NN_ERR_CUDA. */
nn_status nn_batch_submit_query(nn_handle* h, const nn_mesh* meshes, int n_meshes, int want, size_t* ws_bytes);
nn_status nn_batch_submit(nn_handle* h, const nn_mesh* meshes, nn_csr* node_out, nn_csr* elem_out, int n_meshes,
                          void* ws, size_t ws_bytes, int32_t* d_status, nn_stream_t stream);

/* Seeded synthetic grid meshes generated on the device -- input generation
 * for benchmarks and the serving loop, not part of the method.  The result is
 * identical to the host generator (paper_1604_04689_gb300/meshgen.py):
 * n x n (tri/quad) or n x n x n (tet/hex) nodes, triangles split along a
 * seeded diagonal per quad, cube cells split into 6 Kuhn tetrahedra, node ids
 * (permute_nodes) and element order (permute_elems) relabelled by seeded
 * bijections.  With conn == NULL only *n_nodes and *n_elems are returned. */
nn_status nn_generate_grid(int32_t type, int64_t n, uint64_t seed, int permute_nodes, int permute_elems,
                           int32_t* conn, int64_t conn_capacity, int64_t* n_nodes, int64_t* n_elems,
                           nn_stream_t stream);

/* Per-stage device timing (used by the benchmark).  While enabled, compute
 * calls record CUDA events on their stream between their stages:
 *   0 workspace/status init, 1 bucket histogram, 2 bucket offsets,
 *   3 partition (record write; the coarse pass of a two-level partition),
 *   4 fine partition pass (empty for a one-level partition), 5 bucket pass
 *   (element CSR, node rows to scratch), 6 node-row placement.
 * nn_profile_read waits for the recorded events and returns, per stage, the
 * summed milliseconds over the calls since profiling was enabled, and the
 * number of calls.  n_stages <= NN_PROFILE_STAGES.  Enabling twice resets the
 * sums.  Chunked builds and batches record no stages. */
#define NN_PROFILE_STAGES 7
nn_status nn_profile_enable(nn_handle* h, int enable);
nn_status nn_profile_read(nn_handle* h, double* ms, int64_t* calls, int n_stages);

/* Allocation-free build of both results, for callers that may not allocate
 * device memory (code that runs inside an application owning all device
 * memory through its own pool, or a loop that must never enter the CUDA
 * allocator).  The paper has no counterpart: it is a deployment variant of
 * nn_neighbors_both.  Instead of a caller workspace it uses one scratch array
 * of NN_NOALLOC_SCRATCH_BYTES that the library keeps in device memory; every
 * GPU that loads libnn holds that array until the process exits.  The caller
 * still passes the mesh, both output CSRs and d_status (all device memory it
 * owns) and the stream.  The first call on a device (with that device
 * current) looks up the array's device address; make that first call before
 * any stream capture.  A call in a new context of the device (after
 * cudaDeviceReset) looks the address up again.  Meshes whose build needs more scratch than the array
 * holds (roughly 1.5 million node-element incidences) are rejected with
 * NN_ERR_WORKSPACE before anything is enqueued.  All calls share the array
 * and it keeps the last call's contents: calls whose work overlaps on the GPU
 * race, so the caller must serialise them (one stream, or events). */
#define NN_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
nn_status nn_neighbors_both_noalloc(const nn_mesh* mesh, nn_csr* nodes, nn_csr* elems, int32_t* d_status,
                                    nn_stream_t stream);

/* Diagnostic of the bounded device-side waits; the paper has no counterpart.
 * The single-pass scans of a build wait for predecessor tiles (a decoupled
 * lookback).  Such a wait gives up after about 2 s without progress, writes
 * NN_ERR_TIMEOUT to the call's status word and returns, so a lost
 * predecessor never hangs the GPU.  This call runs that same wait for a tile
 * whose predecessor never publishes, so that a test can watch it end.
 * d_state: device, 3 x uint64, 8-byte aligned, overwritten: word 0 is the
 * predecessor (set to 0, never published), word 1 receives the probed tile's
 * published prefix when the wait ends, word 2 the wait's duration in ns.
 * d_status: device int32, set to 0, then NN_ERR_TIMEOUT.  Asynchronous on
 * stream; the kernel runs about 2 s.  Host errors: NN_ERR_ARG for a null or
 * misaligned pointer, NN_ERR_CUDA if the launch fails. */
nn_status nn_diag_wait_timeout(uint64_t* d_state, int32_t* d_status, nn_stream_t stream);

/* Short English text for a status code (static storage). */
const char* nn_status_str(nn_status s);

#ifdef __cplusplus
}
#endif

#endif /* NN_H */
