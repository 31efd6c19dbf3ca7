// Internal host/device interface of libnn: the build plan, kernel parameter
// blocks and the launchers defined in the kernel translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "nn.h"

namespace nn {

// Layout of one packed incidence record (node v is local node i of element e).
// Bit fields, low to high:
//   vloc   : v mod 2^sb (the record's bucket is v >> sb)            [sb bits]
//   nf     : 1 if v already occurred earlier in e (degenerate e)   [1 bit, elems wanted]
//   e      : element id                                            [eb bits, elems wanted]
//   n_0..  : k edge-neighbors of v in e, stored as id+1, 0 = none  [nb bits each, nodes wanted]
// The record is 8 bytes when the fields fit 64 bits, else 16 bytes.
struct RecFmt {
    int sb;
    int want;
    int k;
    int off_nf, off_e, eb;
    int off_n, nb;
    int rb;  // 8 or 16
    // Partition: cshift < 0 -> one scattered pass (one store per record);
    // cshift == 0 -> one tile-sorted pass with the bucket as radix digit
    // (at most 256 buckets); cshift > 0 -> a tile-sorted pass on the coarse
    // digit (bucket >> cshift) into a temporary array, then a tile-sorted
    // pass per coarse region on the fine digit, stored in the record at off_fb.
    int cshift;
    int off_fb;
};

// Element walk: the kernels that read the connectivity (histogram and
// partition passes).  Each CTA owns a fixed range of work units; a unit is 4
// triangles (three 16-byte loads) or one element of any other type.
struct EmitParams {
    int type;
    int64_t n_nodes, n_elems, n_conn;
    const int32_t* conn;
    const int64_t* elem_ptr;
    const uint8_t* elem_type;
    RecFmt fmt;
    // node range of this build: incidences of nodes outside [node_lo,
    // node_lo + node_span) are skipped, buckets count from node_lo (a whole
    // mesh: 0 and n_nodes; a chunked build: one chunk)
    int64_t node_lo, node_span;
    int64_t n_buckets;
    int64_t hist_chunk;  // buckets counted per walk of the histogram pass (shared counters)
    int n_cta;        // CTAs of the histogram pass (rows of hist)
    int n_cta_part;   // CTAs of the partition pass
    uint32_t* hist;   // [n_cta][n_buckets] record counts of each CTA's element slice
    uint32_t* nfc;    // [n_buckets] records of a node already seen in its element (they add no element entry)
    uint32_t* gcur;   // [n_buckets] write cursor of each bucket (starts at the bucket start)
    uint32_t* gcur_coarse;  // [256] write cursor of each coarse region (two-level partition)
    uint8_t* rec_tmp; // records grouped by coarse region (two-level partition)
    uint8_t* rec;     // records, grouped by bucket
    uint64_t rec_cap; // records that fit; more only when elem_ptr is invalid
    int32_t* status;
    uint64_t hist_words;  // length of hist (bounds-checked builds)
};

struct BatchHeader;

struct OffsetsParams {
    uint32_t* hist;
    int n_cta;
    int64_t n_buckets;
    uint32_t* bstart;       // [n_buckets+1] first record of each bucket
    const uint32_t* nfc;    // [n_buckets] repeated-node records (nullptr: no element offsets)
    uint32_t* estart;       // [n_buckets+1] first element-CSR entry of each bucket (with nfc)
    uint32_t* gcur;         // [n_buckets] set to the bucket starts
    uint32_t* gcur_coarse;  // [256] set to the coarse region starts (when cshift > 0)
    int cshift;
    uint64_t* lb_state;     // lookback words, one per tile of buckets
    uint32_t* ticket;
    uint64_t rec_cap;       // bucket starts are clamped to the record array
    int32_t* status;
    const BatchHeader* hdr; // batches: the bucket count comes from the header
};

// ------------------------------------------------------------------ batches
// A batch is the disjoint union of many meshes built by one launch sequence.
// Its description lives in device memory (copied from host staging by the
// launch), so the same captured sequence serves any batch that fits the
// workspace capacity: header, then one BatchMesh per mesh, then the element
// and bucket offsets of the meshes (n_meshes + 1 each).
struct BatchMesh {
    int32_t type;
    int32_t k;
    int64_t n_nodes, n_elems, n_conn;
    const int32_t* conn;
    const int64_t* elem_ptr;
    const uint8_t* elem_type;
    int64_t* rp_n; int32_t* col_n; int64_t cap_n;
    int64_t* rp_e; int32_t* col_e; int64_t cap_e;
    int32_t* status;
};

struct BatchHeader {
    RecFmt fmt;
    int32_t n_meshes;
    int64_t n_elems;    // elements of all meshes
    int64_t n_buckets;  // buckets of all meshes (each mesh starts a new bucket)
    int64_t n_records;  // record capacity (incidences of all meshes)
};

struct BatchTables {
    const BatchHeader* hdr;
    const BatchMesh* meshes;
    const int64_t* elem_off;    // [n_meshes+1]
    const int64_t* bucket_off;  // [n_meshes+1]
};

// Bucket pass: one CTA per bucket (persistent, buckets taken in order),
// builds the rows of the bucket's 2^sb nodes and writes both CSRs.
struct BucketParams {
    RecFmt fmt;
    int64_t n_nodes;
    int64_t n_buckets;
    const uint8_t* rec;
    const uint32_t* bstart;
    const uint32_t* estart; // element-CSR offset of each bucket, batch-wide (required when element rows are wanted)
    uint32_t* ticket;
    uint32_t* spill;        // global scratch for buckets too large for shared memory
    uint64_t spill_words;
    unsigned long long* spill_cursor;
    int64_t* rp_n; int32_t* col_n; int64_t cap_n;
    int64_t* rp_e; int32_t* col_e; int64_t cap_e;
    int32_t* status;
    uint32_t area_words;    // shared-memory words available for record groups and rows
    uint32_t* ntmp;         // node rows of bucket b at ntmp + k * bstart[b] (k = neighbours per record)
    uint32_t* ubk;          // [n_buckets] node-row total of each bucket
    uint32_t* nloc;         // [n_buckets << sb] each node's offset within its bucket's rows
    int32_t wide;           // 1: 32 records and a 32-slot table per node in registers, 0: 16 and 16
    int32_t rec_smem;       // 1: copy each bucket's records into shared memory when they fit, 0: read them from L2
    BatchTables batch;      // batch.hdr != nullptr: format, bucket count and meshes come from the tables
    const int32_t* batch_err;  // batches: status of the shared offsets scan, copied to every mesh
    const int64_t* base;    // chunked builds: {element-CSR, node-CSR} entries of the earlier chunks (else nullptr)
    // buffer lengths, for bounds-checked builds
    uint64_t rec_count;     // records the record array holds
    uint64_t ntmp_words;    // words of ntmp
    uint64_t nloc_words;    // words of nloc
    uint64_t ubk_words;     // words of ubk
};

constexpr int EMIT_THREADS = 1024;
constexpr int PART_THREADS = 512;
constexpr int SORT_THREADS = 256;   // tile-sorted partition passes
constexpr int OFFSETS_THREADS = 128;

// Placement of the node rows the bucket pass left in scratch (nn_compact.cu).
struct CompactParams {
    int64_t n_buckets;       // single mesh (batches: from the header)
    int64_t n_buckets_cap;   // grid of the scan (batches: capacity)
    int sb, k;               // single mesh (batches: from the header; k = 3)
    int64_t n_nodes;
    const uint32_t* bstart;
    const uint32_t* ubk;
    const uint32_t* nloc;
    const uint32_t* ntmp;
    uint64_t* nstart;        // [n_buckets+1] exclusive scan of ubk (batch-wide)
    uint64_t* lb_state;      // lookback words, one per tile of buckets
    uint32_t* ticket;
    int64_t* rp_n; int32_t* col_n; int64_t cap_n;
    int32_t* status;
    BatchTables batch;
    const int64_t* base;     // chunked builds: {element-CSR, node-CSR} entries of the earlier chunks (else nullptr)
    // buffer lengths, for bounds-checked builds
    uint64_t ntmp_words;     // words of ntmp
    uint64_t nloc_words;     // words of nloc
};

// Element face adjacency (nn_adj.cu).
struct AdjParams {
    int type;
    int64_t n_nodes, n_elems, n_conn;
    const int32_t* conn;
    const int64_t* elem_ptr;
    const uint8_t* elem_type;
    const int64_t* ne_rp;    // node -> element CSR
    const int32_t* ne_col;
    uint32_t* cnt;           // [n_elems] neighbours per element
    uint64_t* lb_state;      // lookback words, one per tile of elements
    uint32_t* ticket;
    int64_t* rp; int32_t* col; int64_t cap;
    int32_t* status;
};

// launchers (return the CUDA error of the launch)
cudaError_t launch_adjacency(const AdjParams& p, int grid, cudaStream_t s);
size_t adjacency_scan_tiles(int64_t n_elems);
cudaError_t launch_node_compact(const CompactParams& p, int copy_grid, cudaStream_t s);
// chunked builds: base[0] += estart[B], base[1] += nstart[B] (either may be nullptr)
cudaError_t launch_chunk_advance(int64_t* base, const uint32_t* estart, const uint64_t* nstart, int64_t B,
                                 cudaStream_t s);
// incidences per node slab of 2^shift nodes, added to counts[0 .. n_slabs) (n_slabs <= NN_CHUNK_SLABS_MAX)
cudaError_t launch_slab_count(const EmitParams& p, int shift, int n_slabs, uint32_t* counts, cudaStream_t s);
cudaError_t launch_hist(const EmitParams& p, size_t smem, cudaStream_t s);
cudaError_t launch_part(const EmitParams& p, cudaStream_t s);
cudaError_t launch_part_sorted(const EmitParams& p, const uint32_t* bstart, int sms, cudaStream_t s);
// the two passes of launch_part_sorted on their own (the fine pass only when cshift > 0)
cudaError_t launch_part_coarse(const EmitParams& p, cudaStream_t s);
cudaError_t launch_part_fine(const EmitParams& p, const uint32_t* bstart, int sms, cudaStream_t s);
cudaError_t launch_offsets(const OffsetsParams& p, cudaStream_t s);
cudaError_t launch_bucket(const BucketParams& p, int grid, int threads, size_t smem, cudaStream_t s);
size_t bucket_fixed_bytes(int sb, int threads, int wide);  // shared memory of the bucket kernel outside its area
cudaError_t bucket_occupancy(int* blocks, int threads, int wide, size_t smem);
cudaError_t launch_batch_emit(const BatchTables& bt, uint32_t* bcount, uint32_t* nfc, uint32_t* gcur, uint8_t* rec,
                              uint64_t* lb_off, uint32_t* ctrl, int grid, int stage, cudaStream_t s,
                              uint64_t* lb_ns = nullptr);
int batch_threads();
cudaError_t set_emit_smem_all(size_t bytes);
cudaError_t set_bucket_smem_all(size_t bytes);
bool handle_offline(const nn_handle* h);  // a sizing-only handle (nn_create_offline)
nn_status build_with_limits(int sms, size_t smem_optin, size_t smem_per_sm, const nn_mesh* m, int want,
                            nn_csr* nodes, nn_csr* elems, void* ws, size_t ws_bytes, int32_t* d_status,
                            cudaStream_t s, size_t* ws_min);

}  // namespace nn
