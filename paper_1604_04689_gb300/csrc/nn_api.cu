// Host side of libnn: argument checks, the build plan (bucket width, record
// format, workspace layout) and the launch sequence.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "nn_internal.h"

namespace nn {
cudaError_t set_emit_smem_all(size_t bytes);
cudaError_t set_bucket_smem_all(size_t bytes);
}  // namespace nn

struct nn_handle {
    int device = 0;
    bool offline = false;      // nn_create_offline: sizing and planning only, no compute calls
    int sms = 0;
    size_t smem_optin = 0;     // max dynamic shared memory per block
    size_t bucket_smem = 0;    // largest dynamic shared memory of the bucket kernel
    size_t smem_per_sm = 0;
    int sb_override = -1;      // fixed bucket width (tests / tuning), -1 = automatic
    int part_mode = -1;        // -1 automatic, 0 one scattered store per record (tests)
    int64_t hist_chunk_override = 0;  // > 0: count at most this many buckets per walk (tests)
    int emit_ctas_override = 0;       // > 0: at most this many element-walk CTAs (tests)
    nn_tuning tuning{};        // nn_set_tuning: bucket width, block size, CTAs per SM (0 = automatic)
    // per-stage timing (nn_profile_*)
    bool prof = false;
    bool pending = false;
    cudaEvent_t ev[NN_PROFILE_STAGES + 1] = {};
    double acc[NN_PROFILE_STAGES] = {};
    int64_t calls = 0;
};

bool nn::handle_offline(const nn_handle* h) { return h && h->offline; }

namespace {

using namespace nn;

constexpr size_t ALIGN = 256;
constexpr int SB_MIN = 4, SB_MAX = 11;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }
int bits_for(uint64_t x) {  // bits needed to hold values 0..x (>= 1)
    int b = 1;
    while (b < 64 && (x >> b)) ++b;
    return b;
}
int npe_host(int t) { return t == NN_TRI ? 3 : (t == NN_HEX ? 8 : 4); }

struct Plan {
    int type = 0, want = 0, k = 0;
    // N: nodes of this build's range (first node `lo`); n_conn: its records
    // (incidences of those nodes); a whole mesh has lo = 0 and both totals
    int64_t N = 0, T = 0, n_conn = 0, lo = 0;
    RecFmt fmt{};
    int64_t B = 0;
    int64_t hist_chunk = 1;
    int G = 1;
    int G_part = 1;
    int G_fine = 1;
    size_t emit_smem = 0;
    size_t off_estart = 0, off_nfc = 0, off_ntmp = 0, off_ubk = 0, off_nloc = 0, off_nstart = 0, off_lb_ns = 0;
    size_t off_hist = 0, off_bstart = 0, off_gcur = 0, off_gcur_c = 0, off_rec_tmp = 0, off_rec = 0, off_lb_off = 0,
           off_ctrl = 0, off_spill = 0, zero_begin = 0, zero_end = 0;
    size_t ws_min = 0, ws_rec = 0;
    int bucket_grid = 0;
    int bucket_threads = 256;
    int wide = 0;
    int rec_smem = 1;
    size_t bucket_smem = 0;
    uint32_t area_words = 0;
};

nn_status check_mesh(const nn_mesh* m) {
    if (!m) return NN_ERR_ARG;
    const int t = m->type;
    if (!(t == NN_TRI || t == NN_QUAD || t == NN_TET || t == NN_HEX || t == NN_MIXED)) return NN_ERR_ARG;
    if (m->n_nodes < 0 || m->n_elems < 0 || m->n_conn < 0) return NN_ERR_ARG;
    if (m->n_nodes >= (1ll << 31) || m->n_elems >= (1ll << 31) || m->n_conn >= (1ll << 31)) return NN_ERR_ARG;
    if (t != NN_MIXED && m->n_conn != m->n_elems * npe_host(t)) return NN_ERR_ARG;
    if (m->n_conn > 0 && !m->conn) return NN_ERR_ARG;
    if (t != NN_MIXED && (reinterpret_cast<uintptr_t>(m->conn) & 15)) return NN_ERR_ARG;
    if (t == NN_MIXED && m->n_elems > 0 && (!m->elem_ptr || !m->elem_type)) return NN_ERR_ARG;
    if (t == NN_MIXED && (reinterpret_cast<uintptr_t>(m->elem_ptr) & 7)) return NN_ERR_ARG;
    return NN_OK;
}

// Plan of a build over the nodes [lo, lo + span) of mesh m, which have
// `records` incidences: the element walk covers the whole mesh, the record
// arrays and node tables only this range.  Record fields stay sized by the
// whole mesh (node and element ids are global).
nn_status make_plan_range(const nn_handle* h, const nn_mesh* m, int want, int64_t lo, int64_t span, int64_t records,
                          Plan* P) {
    nn_status st = check_mesh(m);
    if (st != NN_OK) return st;
    if (want < 1 || want > 3) return NN_ERR_ARG;
    if (lo < 0 || span < 0 || lo + span > m->n_nodes || records < 0 || records > m->n_conn) return NN_ERR_ARG;
    Plan p;
    p.type = m->type;
    p.want = want;
    p.N = span;
    p.lo = lo;
    p.T = m->n_elems;
    p.n_conn = records;
    p.k = (m->type == NN_TRI || m->type == NN_QUAD) ? 2 : 3;

    // bucket kernel shape.  Every node goes to one lane, which holds up to
    // 16 (or, "wide", 32) records and a 16 (32) slot neighbour table;
    // meshes whose nodes have more than ten incidences on average (tets,
    // mixed) take the wide form.  256-thread CTAs, two per SM.  A bucket's
    // records are copied into the CTA's shared memory beside each record's
    // slot, its record groups, element rows and neighbour rows; the bucket
    // width is as many nodes as fit with room to spare for buckets of higher
    // than average record counts.
    const double inc = p.N > 0 ? (double)p.n_conn / (double)p.N : 0.0;
    p.wide = inc > 10.0 ? 1 : 0;
    const int ucap = p.wide ? 24 : 12;  // distinct neighbours a lane's table takes
    p.bucket_threads = h->tuning.bucket_threads ? h->tuning.bucket_threads : 256;
    const int bcps = h->tuning.bucket_ctas_per_sm ? h->tuning.bucket_ctas_per_sm : (p.bucket_threads == 128 ? 4 : 2);
    size_t bsmem = std::min(h->bucket_smem, h->smem_per_sm / (size_t)bcps - 2048);
    // distinct neighbours per node: half the candidates, at most two thirds
    // of what a lane's table takes (a Kuhn tet grid has 14 for 72 candidates)
    const double U = (want & NN_WANT_NODES) ? std::min(p.k * inc / 2.0, ucap * 2.0 / 3.0) : 0.0;
    // record width of a bucket shift s (the fine-digit field of a two-level
    // partition included, at most 12 bits)
    const int eb_ = bits_for(p.T > 0 ? (uint64_t)(p.T - 1) : 0), nb_ = bits_for((uint64_t)m->n_nodes);
    auto rb_of = [&](int s) {
        const int bits = s + ((want & NN_WANT_ELEMS) ? 1 + eb_ : 0) + ((want & NN_WANT_NODES) ? p.k * nb_ : 0);
        int cs_ = 0;
        while ((((p.N + (1ll << s) - 1) >> s) + (1ll << cs_) - 1) >> cs_ > 256) ++cs_;
        return bits + cs_ <= 64 ? 8 : 16;
    };
    // shared memory of a bucket of 2^s nodes with 15 % more records than
    // average: the records themselves (when copied in), a slot and a group
    // entry per record, element rows, neighbour rows
    bool rec_smem = true;
    auto bucket_bytes = [&](int s) {
        const double n = (double)(1 << s) * 1.15;
        return n * (inc * ((rec_smem ? rb_of(s) : 0) + 8.0) + 4.0 * (rec_smem ? std::max(U, inc) : U)) + 64.0;
    };
    // (many buckets are fine: the histogram pass counts them in chunks that
    // fit its shared memory; the hard cap below only bounds workspace tables)
    const int64_t B_lim = (int64_t)1 << 20;
    auto fixed_of = [&](int s) { return bucket_fixed_bytes(s, p.bucket_threads, p.wide); };
    auto widest = [&]() {
        for (int s = SB_MAX; s >= SB_MIN; --s) {
            if (((p.N + (1ll << s) - 1) >> s) > B_lim) break;
            const double area = (double)bsmem - (double)fixed_of(s);
            if (area > 0 && bucket_bytes(s) <= area) return s;
        }
        return -1;
    };
    // records in shared memory unless that leaves a bucket fewer nodes than
    // the CTA has lanes
    int sb = widest();
    if (sb >= 0 && (32 << (sb - 5)) < p.bucket_threads && sb < SB_MAX) {
        rec_smem = false;
        const int s2 = widest();
        if (s2 > sb) sb = s2;
        else rec_smem = true;
    }
    p.rec_smem = rec_smem ? 1 : 0;
    if (sb < 0) sb = SB_MIN;
    if (h->tuning.sb >= SB_MIN && h->tuning.sb <= SB_MAX) sb = h->tuning.sb;
    if (h->sb_override >= SB_MIN && h->sb_override <= SB_MAX) sb = h->sb_override;
    const size_t min_area = 1024 * 4;
    while (fixed_of(sb) + min_area > bsmem && bsmem < h->bucket_smem) bsmem = h->bucket_smem;
    p.bucket_smem = bsmem;
    while (sb > SB_MIN && fixed_of(sb) + min_area > p.bucket_smem) --sb;
    const int64_t B_max = B_lim;
    auto nbk = [&](int s) { return (p.N + (1ll << s) - 1) >> s; };
    while (nbk(sb) > B_max && sb < SB_MAX) ++sb;
    if (nbk(sb) > B_max || fixed_of(sb) + min_area > p.bucket_smem) return NN_ERR_ARG;
    p.B = nbk(sb);

    RecFmt& f = p.fmt;
    f.sb = sb;
    f.want = want;
    f.k = p.k;
    f.eb = bits_for(p.T > 0 ? (uint64_t)(p.T - 1) : 0);
    f.nb = bits_for((uint64_t)m->n_nodes);
    f.off_nf = sb;
    f.off_e = sb + 1;
    f.off_n = (want & NN_WANT_ELEMS) ? sb + 1 + f.eb : sb;
    int total = (want & NN_WANT_NODES) ? f.off_n + p.k * f.nb : sb + 1 + f.eb;
    if (total > 128) return NN_ERR_ARG;
    // partition: tile-sorted (one pass for <= 256 buckets, else coarse + fine
    // with the fine digit kept in the record) unless that field does not fit
    int cs = 0;
    while (((p.B + (1ll << cs) - 1) >> cs) > 256) ++cs;
    f.cshift = -1;
    f.off_fb = total;
    if (h->part_mode != 0 && total + cs <= 128 && cs <= 12) {  // <= 4096 buckets per coarse region
        f.cshift = cs;
        total += cs;
    }
    f.rb = total <= 64 ? 8 : 16;

    // element-walk CTAs: one or two per SM, each a fixed slice of elements
    const int unit = p.type == NN_TRI ? 4 : 1;
    const int64_t n_units = (p.T + unit - 1) / unit;
    p.hist_chunk = std::min<int64_t>(p.B, (int64_t)((h->smem_optin - 1024) / 4));
    if (h->hist_chunk_override > 0) p.hist_chunk = std::min<int64_t>(p.hist_chunk, h->hist_chunk_override);
    p.emit_smem = std::max<size_t>(16, (size_t)p.hist_chunk * 4);
    const int cps = p.emit_smem + 2048 <= 113 * 1024 ? 2 : 1;
    p.G = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sms * cps, (n_units + 2047) / 2048));
    if (h->emit_ctas_override > 0) p.G = std::min(p.G, h->emit_ctas_override);
    p.G_part = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sms * 2, (n_units + 511) / 512));
    if (f.cshift >= 0)  // tile-sorted passes: 256-thread CTAs, several per SM
        p.G_part = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sms * 4, (n_units + 511) / 512));
    p.G_fine = h->sms;  // the fine pass sizes its grid by its occupancy

    p.area_words = (uint32_t)((p.bucket_smem - fixed_of(sb)) / 4);
    int per_sm = 1;
    if (h->offline || bucket_occupancy(&per_sm, p.bucket_threads, p.wide, p.bucket_smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    p.bucket_grid = (int)std::min<int64_t>(p.B, (int64_t)h->sms * per_sm);

    // workspace layout
    size_t o = 0;
    p.off_hist = o; o = align_up(o + (size_t)p.G * p.B * 4);
    p.off_bstart = o; o = align_up(o + ((size_t)p.B + 1) * 4);
    p.off_estart = o; o = align_up(o + ((want & NN_WANT_ELEMS) ? ((size_t)p.B + 1) * 4 : 0));
    p.off_gcur = o; o = align_up(o + (size_t)p.B * 4);
    p.off_gcur_c = o; o = align_up(o + 256 * 4);
    p.off_rec_tmp = o; o = align_up(o + (f.cshift > 0 ? (size_t)p.n_conn * f.rb : 0));
    p.off_rec = o; o = align_up(o + (size_t)p.n_conn * f.rb);
    // node rows in scratch (at most k per record), per-node offsets within
    // their bucket, bucket totals and their scan
    const bool wn = want & NN_WANT_NODES;
    const size_t ntmp_bytes = wn ? (size_t)p.k * p.n_conn * 4 + 16 : 0;
    if (f.cshift > 0 && (size_t)p.n_conn * f.rb >= ntmp_bytes) {
        p.off_ntmp = p.off_rec_tmp;  // the coarse-sorted records are dead once the fine pass has run
    } else {
        p.off_ntmp = o; o = align_up(o + ntmp_bytes);
    }
    p.off_ubk = o; o = align_up(o + (wn ? (size_t)p.B * 4 : 0));
    p.off_nloc = o; o = align_up(o + (wn ? ((size_t)p.B << sb) * 4 : 0));
    p.off_nstart = o; o = align_up(o + (wn ? ((size_t)p.B + 1) * 8 : 0));
    p.zero_begin = o;
    p.off_nfc = o; o = align_up(o + ((want & NN_WANT_ELEMS) ? (size_t)p.B * 4 : 0));
    p.off_lb_off = o; o = align_up(o + (size_t)((p.B + OFFSETS_THREADS - 1) / OFFSETS_THREADS) * 8 + 8);
    p.off_lb_ns = o; o = align_up(o + (wn ? (size_t)((p.B + 127) / 128) * 8 + 8 : 0));
    p.off_ctrl = o; o = align_up(o + 64);
    p.zero_end = o;
    p.off_spill = o;
    p.ws_min = o;
    // spill area: buckets larger than the bucket pass's shared memory keep
    // their record groups and rows there (16 MB and 8 bytes per record covers
    // the odd oversized bucket, a node of very high valence included); a
    // plan whose typical bucket does not fit (a tuning that widens the
    // buckets) gets room for all of them
    size_t spill = ((size_t)16 << 20) + (size_t)p.n_conn * 8;
    if (bucket_bytes(sb) > (double)p.area_words * 4.0)
        spill += (size_t)p.n_conn * (8 + 4 * (size_t)p.k) + (size_t)p.B * 64;
    p.ws_rec = o + spill;

    *P = p;
    return NN_OK;
}

nn_status make_plan(const nn_handle* h, const nn_mesh* m, int want, Plan* P) {
    nn_status st = check_mesh(m);
    if (st != NN_OK) return st;
    return make_plan_range(h, m, want, 0, m->n_nodes, m->n_conn, P);
}

void prof_flush(nn_handle* h) {
    if (!h->pending) return;
    h->pending = false;
    if (cudaEventSynchronize(h->ev[NN_PROFILE_STAGES]) != cudaSuccess) return;
    for (int i = 0; i < NN_PROFILE_STAGES; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) == cudaSuccess) h->acc[i] += ms;
    }
    h->calls += 1;
}

void prof_mark(nn_handle* h, int i, cudaStream_t s) {
    if (h->prof) cudaEventRecord(h->ev[i], s);
}

nn_status enqueue(nn_handle* h, const nn_mesh* m, const Plan& p, nn_csr* nodes, nn_csr* elems, uint8_t* w,
                  size_t ws_bytes, const int64_t* base, int32_t* d_status, bool prof, cudaStream_t s);

// Argument checks shared by the single and chunked builds.
nn_status check_outputs(int want, const nn_csr* nodes, const nn_csr* elems) {
    if ((want & NN_WANT_NODES) && (!nodes || !nodes->row_ptr || nodes->col_capacity < 0 ||
                                   (nodes->col_capacity > 0 && !nodes->col)))
        return NN_ERR_ARG;
    if ((want & NN_WANT_ELEMS) && (!elems || !elems->row_ptr || elems->col_capacity < 0 ||
                                   (elems->col_capacity > 0 && !elems->col)))
        return NN_ERR_ARG;
    return NN_OK;
}

nn_status run(nn_handle* h, const nn_mesh* m, int want, nn_csr* nodes, nn_csr* elems, void* ws,
              size_t ws_bytes, int32_t* d_status, cudaStream_t s) {
    if (!h || h->offline || !d_status) return NN_ERR_ARG;
    Plan p;
    nn_status st = make_plan(h, m, want, &p);
    if (st != NN_OK) return st;
    st = check_outputs(want, nodes, elems);
    if (st != NN_OK) return st;
    if (ws_bytes < p.ws_min || (!ws && p.ws_min > 0)) return NN_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & (ALIGN - 1)) return NN_ERR_ARG;

    uint8_t* w = static_cast<uint8_t*>(ws);
    if (h->prof) prof_flush(h);
    prof_mark(h, 0, s);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return NN_ERR_CUDA;
    if (p.N == 0) {
        if ((want & NN_WANT_NODES) && cudaMemsetAsync(nodes->row_ptr, 0, 8, s) != cudaSuccess) return NN_ERR_CUDA;
        if ((want & NN_WANT_ELEMS) && cudaMemsetAsync(elems->row_ptr, 0, 8, s) != cudaSuccess) return NN_ERR_CUDA;
        return NN_OK;
    }
    st = enqueue(h, m, p, nodes, elems, w, ws_bytes, nullptr, d_status, h->prof, s);
    if (st == NN_OK && h->prof) h->pending = true;
    return st;
}

// Enqueue the kernels of plan p: rows p.lo .. p.lo + p.N - 1 of the CSRs.
// base: the running {element, node} CSR bases of a chunked build on the
// device, added to every row pointer and col position (nullptr: 0).
nn_status enqueue(nn_handle* h, const nn_mesh* m, const Plan& p, nn_csr* nodes, nn_csr* elems, uint8_t* w,
                  size_t ws_bytes, const int64_t* base, int32_t* d_status, bool prof, cudaStream_t s) {
    const int want = p.want;
    auto mark = [&](int i) {
        if (prof) prof_mark(h, i, s);
    };
    if (cudaMemsetAsync(w + p.zero_begin, 0, p.zero_end - p.zero_begin, s) != cudaSuccess) return NN_ERR_CUDA;

    uint32_t* ctrl = reinterpret_cast<uint32_t*>(w + p.off_ctrl);
    EmitParams ep{};
    ep.type = p.type;
    ep.n_nodes = m->n_nodes;
    ep.n_elems = p.T;
    ep.n_conn = m->n_conn;
    ep.node_lo = p.lo;
    ep.node_span = p.N;
    ep.conn = m->conn;
    ep.elem_ptr = m->elem_ptr;
    ep.elem_type = m->elem_type;
    ep.fmt = p.fmt;
    ep.n_buckets = p.B;
    ep.hist_chunk = std::max<int64_t>(1, p.hist_chunk);
    ep.n_cta = p.G;
    ep.n_cta_part = p.G_part;
    ep.hist = reinterpret_cast<uint32_t*>(w + p.off_hist);
    ep.nfc = (want & NN_WANT_ELEMS) ? reinterpret_cast<uint32_t*>(w + p.off_nfc) : nullptr;
    ep.gcur = reinterpret_cast<uint32_t*>(w + p.off_gcur);
    ep.gcur_coarse = reinterpret_cast<uint32_t*>(w + p.off_gcur_c);
    ep.rec_tmp = w + p.off_rec_tmp;
    ep.rec = w + p.off_rec;
    ep.rec_cap = (uint64_t)p.n_conn;
    ep.status = d_status;
    ep.hist_words = (uint64_t)p.G * (uint64_t)p.B;

    OffsetsParams op{};
    op.hist = ep.hist;
    op.n_cta = p.G;
    op.n_buckets = p.B;
    op.bstart = reinterpret_cast<uint32_t*>(w + p.off_bstart);
    op.nfc = ep.nfc;
    op.estart = (want & NN_WANT_ELEMS) ? reinterpret_cast<uint32_t*>(w + p.off_estart) : nullptr;
    op.gcur = ep.gcur;
    op.gcur_coarse = ep.gcur_coarse;
    op.cshift = p.fmt.cshift;
    op.lb_state = reinterpret_cast<uint64_t*>(w + p.off_lb_off);
    op.ticket = ctrl + 0;
    op.rec_cap = (uint64_t)p.n_conn;
    op.status = d_status;

    BucketParams bp{};
    bp.fmt = p.fmt;
    bp.n_nodes = p.N;
    bp.n_buckets = p.B;
    bp.rec = ep.rec;
    bp.bstart = op.bstart;
    bp.estart = op.estart;
    bp.ticket = ctrl + 1;
    bp.spill_cursor = reinterpret_cast<unsigned long long*>(ctrl + 2);
    bp.spill = reinterpret_cast<uint32_t*>(w + p.off_spill);
    const size_t spill_bytes = ws_bytes > p.off_spill ? ws_bytes - p.off_spill : 0;
    bp.spill_words = spill_bytes / 4;
    if (want & NN_WANT_NODES) {
        bp.rp_n = nodes->row_ptr + p.lo;
        bp.col_n = nodes->col;
        bp.cap_n = nodes->col_capacity;
    }
    if (want & NN_WANT_ELEMS) {
        bp.rp_e = elems->row_ptr + p.lo;
        bp.col_e = elems->col;
        bp.cap_e = elems->col_capacity;
    }
    bp.base = base;
    bp.status = d_status;
    bp.area_words = p.area_words;
    bp.wide = p.wide;
    bp.rec_smem = p.rec_smem;
    bp.ntmp = reinterpret_cast<uint32_t*>(w + p.off_ntmp);
    bp.ubk = reinterpret_cast<uint32_t*>(w + p.off_ubk);
    bp.nloc = reinterpret_cast<uint32_t*>(w + p.off_nloc);
    bp.rec_count = (uint64_t)p.n_conn;
    bp.ntmp_words = (want & NN_WANT_NODES) ? (uint64_t)p.k * p.n_conn + 4 : 0;
    bp.nloc_words = (want & NN_WANT_NODES) ? (uint64_t)p.B << p.fmt.sb : 0;
    bp.ubk_words = (want & NN_WANT_NODES) ? (uint64_t)p.B : 0;

    mark(1);
    if (launch_hist(ep, p.emit_smem, s) != cudaSuccess) return NN_ERR_CUDA;
    mark(2);
    if (launch_offsets(op, s) != cudaSuccess) return NN_ERR_CUDA;
    mark(3);
    if (p.fmt.cshift >= 0) {
        if (launch_part_coarse(ep, s) != cudaSuccess) return NN_ERR_CUDA;
        mark(4);
        if (launch_part_fine(ep, op.bstart, p.G_fine, s) != cudaSuccess) return NN_ERR_CUDA;
    } else {
        if (launch_part(ep, s) != cudaSuccess) return NN_ERR_CUDA;
        mark(4);
    }
    mark(5);
    if (launch_bucket(bp, p.bucket_grid, p.bucket_threads, p.bucket_smem, s) != cudaSuccess)
        return NN_ERR_CUDA;
    mark(6);
    if (want & NN_WANT_NODES) {
        CompactParams cp{};
        cp.n_buckets = p.B;
        cp.n_buckets_cap = p.B;
        cp.sb = p.fmt.sb;
        cp.k = p.k;
        cp.n_nodes = p.N;
        cp.base = base;
        cp.bstart = bp.bstart;
        cp.ubk = bp.ubk;
        cp.nloc = bp.nloc;
        cp.ntmp = bp.ntmp;
        cp.nstart = reinterpret_cast<uint64_t*>(w + p.off_nstart);
        cp.lb_state = reinterpret_cast<uint64_t*>(w + p.off_lb_ns);
        cp.ticket = ctrl + 4;
        cp.rp_n = nodes->row_ptr + p.lo;
        cp.col_n = nodes->col;
        cp.cap_n = nodes->col_capacity;
        cp.status = d_status;
        cp.ntmp_words = bp.ntmp_words;
        cp.nloc_words = bp.nloc_words;
        if (launch_node_compact(cp, (int)std::min<int64_t>(p.B, (int64_t)h->sms * 8), s) != cudaSuccess)
            return NN_ERR_CUDA;
    }
    mark(7);
    return NN_OK;
}

// --------------------------------------------------------------- batches

struct BatchPlan {
    int sb = 7;
    int64_t B_cap = 0;
    size_t hdr_bytes = 0, meshes_off = 0, elem_off_off = 0, bucket_off_off = 0, table_bytes = 0;
    size_t off_bcount = 0, off_bstart = 0, off_gcur = 0, off_rec = 0, off_lb_off = 0, off_ctrl = 0, off_spill = 0, ws_min = 0, ws_rec = 0, off_nfc = 0,
           off_estart = 0, off_ntmp = 0, off_ubk = 0, off_nloc = 0, off_nstart = 0, off_lb_ns = 0;
    size_t bucket_smem = 0;
    uint32_t area_words = 0;
    int bucket_grid = 0, emit_grid = 0, bucket_threads = 128;
    int64_t tiles_cap = 0;
};

nn_status batch_plan(const nn_handle* h, const nn_batch_caps* c, BatchPlan* out) {
    if (!h || !c || c->max_meshes < 1 || c->max_elems < 0 || c->max_nodes < 0 || c->max_conn < 0 ||
        c->want < 1 || c->want > 3)
        return NN_ERR_ARG;
    if (c->max_conn >= (1ll << 31) || c->max_elems >= (1ll << 31)) return NN_ERR_ARG;
    BatchPlan p;
    p.sb = c->sb ? c->sb : 7;
    if (p.sb < SB_MIN || p.sb > SB_MAX) return NN_ERR_ARG;
    p.B_cap = (c->max_nodes >> p.sb) + c->max_meshes + 1;
    p.hdr_bytes = align_up(sizeof(BatchHeader));
    p.meshes_off = p.hdr_bytes;
    p.elem_off_off = p.meshes_off + align_up((size_t)c->max_meshes * sizeof(BatchMesh));
    p.bucket_off_off = p.elem_off_off + align_up(((size_t)c->max_meshes + 1) * 8);
    p.table_bytes = p.bucket_off_off + align_up(((size_t)c->max_meshes + 1) * 8);
    // bucket kernel: wide lanes (a batch may hold any element type), 256
    // threads, two CTAs per SM, so that a bucket's records (copied into
    // shared memory) fit beside its tables
    p.bucket_threads = 256;
    const size_t fixed = bucket_fixed_bytes(p.sb, p.bucket_threads, 1);
    p.bucket_smem = std::min(h->bucket_smem, h->smem_per_sm / 2 - 2048);
    if (fixed + 8192 * 4 > p.bucket_smem) p.bucket_smem = h->bucket_smem;
    if (fixed + 4096 * 4 > p.bucket_smem) return NN_ERR_ARG;
    p.area_words = (uint32_t)((p.bucket_smem - fixed) / 4);
    int per_sm = 1;
    if (bucket_occupancy(&per_sm, p.bucket_threads, 1, p.bucket_smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    p.bucket_grid = h->sms * per_sm;
    size_t o = p.table_bytes;
    p.off_bcount = o; o = align_up(o + (size_t)p.B_cap * 4);
    p.off_nfc = o; o = align_up(o + (size_t)p.B_cap * 4);
    p.off_bstart = o; o = align_up(o + ((size_t)p.B_cap + 1) * 4);
    p.off_estart = o; o = align_up(o + ((size_t)p.B_cap + 1) * 4);
    p.off_gcur = o; o = align_up(o + (size_t)p.B_cap * 4);
    p.off_rec = o; o = align_up(o + (size_t)c->max_conn * 16);
    const bool wn = c->want & NN_WANT_NODES;
    p.off_ntmp = o; o = align_up(o + (wn ? (size_t)3 * c->max_conn * 4 + 16 : 0));
    p.off_ubk = o; o = align_up(o + (wn ? (size_t)p.B_cap * 4 : 0));
    p.off_nloc = o; o = align_up(o + (wn ? ((size_t)p.B_cap << p.sb) * 4 : 0));
    p.off_nstart = o; o = align_up(o + (wn ? ((size_t)p.B_cap + 1) * 8 : 0));
    p.off_lb_ns = o; o = align_up(o + (wn ? (size_t)((p.B_cap + 127) / 128) * 8 + 8 : 0));
    p.tiles_cap = (p.B_cap + OFFSETS_THREADS - 1) / OFFSETS_THREADS;
    p.off_lb_off = o; o = align_up(o + ((size_t)p.tiles_cap + 1) * 8);
    p.off_ctrl = o; o = align_up(o + 64);
    p.off_spill = o;
    p.ws_min = o;
    p.ws_rec = o + (((size_t)16 << 20) + (size_t)c->max_conn * 8);
    p.emit_grid = h->sms * (2048 / batch_threads());
    *out = p;
    return NN_OK;
}

nn_status batch_prepare(nn_handle* h, const nn_batch_caps* c, const nn_mesh* meshes, const nn_csr* node_out,
                        const nn_csr* elem_out, int32_t* d_status, int n, void* staging, size_t staging_bytes) {
    BatchPlan bp;
    nn_status st = batch_plan(h, c, &bp);
    if (st != NN_OK) return st;
    if (n < 0 || n > c->max_meshes || !staging || staging_bytes < bp.table_bytes || (n > 0 && (!meshes || !d_status)))
        return NN_ERR_ARG;
    if ((c->want & NN_WANT_NODES) && n > 0 && !node_out) return NN_ERR_ARG;
    if ((c->want & NN_WANT_ELEMS) && n > 0 && !elem_out) return NN_ERR_ARG;
    uint8_t* sg = static_cast<uint8_t*>(staging);
    BatchHeader* hdr = reinterpret_cast<BatchHeader*>(sg);
    BatchMesh* bm = reinterpret_cast<BatchMesh*>(sg + bp.meshes_off);
    int64_t* eoff = reinterpret_cast<int64_t*>(sg + bp.elem_off_off);
    int64_t* boff = reinterpret_cast<int64_t*>(sg + bp.bucket_off_off);
    int64_t E = 0, Bk = 0, C = 0, Nn = 0, maxT = 0, maxN = 0;
    for (int m = 0; m < n; ++m) {
        const nn_mesh& M = meshes[m];
        if ((st = check_mesh(&M)) != NN_OK) return st;
        BatchMesh& d = bm[m];
        d = BatchMesh{};
        d.type = M.type;
        d.k = (M.type == NN_TRI || M.type == NN_QUAD) ? 2 : 3;
        d.n_nodes = M.n_nodes;
        d.n_elems = M.n_elems;
        d.n_conn = M.n_conn;
        d.conn = M.conn;
        d.elem_ptr = M.elem_ptr;
        d.elem_type = M.elem_type;
        if (c->want & NN_WANT_NODES) {
            const nn_csr& o = node_out[m];
            if (!o.row_ptr || o.col_capacity < 0 || (o.col_capacity > 0 && !o.col)) return NN_ERR_ARG;
            d.rp_n = o.row_ptr; d.col_n = o.col; d.cap_n = o.col_capacity;
        }
        if (c->want & NN_WANT_ELEMS) {
            const nn_csr& o = elem_out[m];
            if (!o.row_ptr || o.col_capacity < 0 || (o.col_capacity > 0 && !o.col)) return NN_ERR_ARG;
            d.rp_e = o.row_ptr; d.col_e = o.col; d.cap_e = o.col_capacity;
        }
        d.status = d_status + m;
        eoff[m] = E;
        boff[m] = Bk;
        E += M.n_elems;
        Bk += (M.n_nodes + (1ll << bp.sb) - 1) >> bp.sb;
        C += M.n_conn;
        Nn += M.n_nodes;
        maxT = std::max<int64_t>(maxT, M.n_elems);
        maxN = std::max<int64_t>(maxN, M.n_nodes);
    }
    eoff[n] = E;
    boff[n] = Bk;
    if (E > c->max_elems || C > c->max_conn || Nn > c->max_nodes || Bk > bp.B_cap) return NN_ERR_BUDGET;
    RecFmt f{};
    f.sb = bp.sb;
    f.want = c->want;
    f.k = 3;
    f.eb = bits_for(maxT > 0 ? (uint64_t)(maxT - 1) : 0);
    f.nb = bits_for((uint64_t)maxN);
    f.off_nf = f.sb;
    f.off_e = f.sb + 1;
    f.off_n = (c->want & NN_WANT_ELEMS) ? f.sb + 1 + f.eb : f.sb;
    const int total = (c->want & NN_WANT_NODES) ? f.off_n + 3 * f.nb : f.sb + 1 + f.eb;
    if (total > 128) return NN_ERR_ARG;
    f.rb = 16;
    f.cshift = -1;
    f.off_fb = total;
    hdr->fmt = f;
    hdr->n_meshes = n;
    hdr->n_elems = E;
    hdr->n_buckets = Bk;
    hdr->n_records = C;
    return NN_OK;
}

nn_status batch_launch(nn_handle* h, const nn_batch_caps* c, const void* staging, void* ws, size_t ws_bytes,
                       cudaStream_t s) {
    if (!h || h->offline) return NN_ERR_ARG;
    BatchPlan bp;
    nn_status st = batch_plan(h, c, &bp);
    if (st != NN_OK) return st;
    if (!staging || !ws || (reinterpret_cast<uintptr_t>(ws) & (ALIGN - 1))) return NN_ERR_ARG;
    if (ws_bytes < bp.ws_min) return NN_ERR_WORKSPACE;
    uint8_t* w = static_cast<uint8_t*>(ws);
    if (cudaMemcpyAsync(w, staging, bp.table_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return NN_ERR_CUDA;
    BatchTables bt;
    bt.hdr = reinterpret_cast<const BatchHeader*>(w);
    bt.meshes = reinterpret_cast<const BatchMesh*>(w + bp.meshes_off);
    bt.elem_off = reinterpret_cast<const int64_t*>(w + bp.elem_off_off);
    bt.bucket_off = reinterpret_cast<const int64_t*>(w + bp.bucket_off_off);
    uint32_t* bcount = reinterpret_cast<uint32_t*>(w + bp.off_bcount);
    uint32_t* nfc = reinterpret_cast<uint32_t*>(w + bp.off_nfc);
    uint32_t* gcur = reinterpret_cast<uint32_t*>(w + bp.off_gcur);
    uint32_t* ctrl = reinterpret_cast<uint32_t*>(w + bp.off_ctrl);
    uint64_t* lb_off = reinterpret_cast<uint64_t*>(w + bp.off_lb_off);
    uint8_t* rec = w + bp.off_rec;
    if (launch_batch_emit(bt, bcount, nfc, gcur, rec, lb_off, ctrl, bp.emit_grid, 0, s,
                          reinterpret_cast<uint64_t*>(w + bp.off_lb_ns)) != cudaSuccess)
        return NN_ERR_CUDA;
    if (launch_batch_emit(bt, bcount, nfc, gcur, rec, lb_off, ctrl, bp.emit_grid, 1, s) != cudaSuccess)
        return NN_ERR_CUDA;
    OffsetsParams op{};
    op.hist = bcount;
    op.n_cta = 1;
    op.n_buckets = bp.B_cap;
    op.bstart = reinterpret_cast<uint32_t*>(w + bp.off_bstart);
    op.nfc = nfc;
    op.estart = (c->want & NN_WANT_ELEMS) ? reinterpret_cast<uint32_t*>(w + bp.off_estart) : nullptr;
    op.gcur = gcur;
    op.lb_state = lb_off;
    op.ticket = ctrl + 0;
    op.rec_cap = (uint64_t)c->max_conn;
    op.status = reinterpret_cast<int32_t*>(ctrl + 8);  // passed on to every mesh by the bucket pass
    op.hdr = bt.hdr;
    if (launch_offsets(op, s) != cudaSuccess) return NN_ERR_CUDA;
    if (launch_batch_emit(bt, bcount, nfc, gcur, rec, lb_off, ctrl, bp.emit_grid, 2, s) != cudaSuccess)
        return NN_ERR_CUDA;
    BucketParams kp{};
    kp.n_buckets = 0;
    kp.rec = rec;
    kp.bstart = op.bstart;
    kp.estart = op.estart;
    kp.ticket = ctrl + 1;
    kp.spill_cursor = reinterpret_cast<unsigned long long*>(ctrl + 2);
    kp.spill = reinterpret_cast<uint32_t*>(w + bp.off_spill);
    const size_t spill_bytes = ws_bytes > bp.off_spill ? ws_bytes - bp.off_spill : 0;
    kp.spill_words = spill_bytes / 4;
    kp.area_words = bp.area_words;
    kp.batch = bt;
    kp.batch_err = reinterpret_cast<const int32_t*>(ctrl + 8);
    kp.fmt.rb = 16;
    kp.fmt.k = 3;
    kp.wide = 1;
    kp.rec_smem = 1;
    kp.ntmp = reinterpret_cast<uint32_t*>(w + bp.off_ntmp);
    kp.ubk = reinterpret_cast<uint32_t*>(w + bp.off_ubk);
    kp.nloc = reinterpret_cast<uint32_t*>(w + bp.off_nloc);
    kp.rec_count = (uint64_t)c->max_conn;
    kp.ntmp_words = (c->want & NN_WANT_NODES) ? 3 * (uint64_t)c->max_conn + 4 : 0;
    kp.nloc_words = (c->want & NN_WANT_NODES) ? (uint64_t)bp.B_cap << bp.sb : 0;
    kp.ubk_words = (c->want & NN_WANT_NODES) ? (uint64_t)bp.B_cap : 0;
    if (launch_bucket(kp, bp.bucket_grid, bp.bucket_threads, bp.bucket_smem, s) != cudaSuccess) return NN_ERR_CUDA;
    if (c->want & NN_WANT_NODES) {
        CompactParams cp{};
        cp.n_buckets_cap = bp.B_cap;
        cp.bstart = kp.bstart;
        cp.ubk = kp.ubk;
        cp.nloc = kp.nloc;
        cp.ntmp = kp.ntmp;
        cp.nstart = reinterpret_cast<uint64_t*>(w + bp.off_nstart);
        cp.lb_state = reinterpret_cast<uint64_t*>(w + bp.off_lb_ns);
        cp.ticket = ctrl + 4;
        cp.status = reinterpret_cast<int32_t*>(ctrl + 8);
        cp.batch = bt;
        cp.ntmp_words = kp.ntmp_words;
        cp.nloc_words = kp.nloc_words;
        if (launch_node_compact(cp, h->sms * 8, s) != cudaSuccess) return NN_ERR_CUDA;
    }
    return NN_OK;
}

}  // namespace

namespace nn {

// Build with a handle described by plain device limits (no handle object on
// the heap): used by the allocation-free entry point.
nn_status build_with_limits(int sms, size_t smem_optin, size_t smem_per_sm, const nn_mesh* m, int want,
                            nn_csr* nodes, nn_csr* elems, void* ws, size_t ws_bytes, int32_t* d_status,
                            cudaStream_t s, size_t* ws_min) {
    nn_handle h;
    h.sms = sms;
    h.smem_optin = smem_optin;
    h.smem_per_sm = smem_per_sm;
    h.bucket_smem = smem_optin - 1024;  // the bucket kernel has a little static shared memory
    Plan p;
    nn_status st = make_plan(&h, m, want, &p);
    if (st != NN_OK) return st;
    if (ws_min) *ws_min = p.ws_min;
    if (p.ws_min > ws_bytes) return NN_ERR_WORKSPACE;
    return run(&h, m, want, nodes, elems, ws, ws_bytes, d_status, s);
}

}  // namespace nn

extern "C" {

nn_status nn_create(nn_handle** out) {
    if (!out) return NN_ERR_ARG;
    nn_handle* h = new (std::nothrow) nn_handle();
    if (!h) return NN_ERR_ARG;
    int optin = 0, per_sm = 0;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
        delete h;
        return NN_ERR_CUDA;
    }
    h->smem_optin = (size_t)optin;
    h->smem_per_sm = (size_t)per_sm;
    h->bucket_smem = h->smem_optin - 1024;  // the bucket kernel has a little static shared memory
    if (const char* e = std::getenv("NN_SB")) h->sb_override = std::atoi(e);
    if (const char* e = std::getenv("NN_PART")) h->part_mode = std::strcmp(e, "scatter") == 0 ? 0 : -1;
    if (const char* e = std::getenv("NN_HIST_CHUNK")) h->hist_chunk_override = std::atoll(e);
    if (const char* e = std::getenv("NN_EMIT_CTAS")) h->emit_ctas_override = std::atoi(e);
    if (const char* e = std::getenv("NN_BUCKET_SMEM_KB")) {
        size_t kb = (size_t)std::atol(e);
        if (kb >= 32 && kb * 1024 <= h->smem_optin - 1024) h->bucket_smem = kb * 1024;
    }
    if (set_emit_smem_all(h->smem_optin) != cudaSuccess || set_bucket_smem_all(h->smem_optin) != cudaSuccess) {
        delete h;
        return NN_ERR_CUDA;
    }
    *out = h;
    return NN_OK;
}

nn_status nn_create_offline(nn_handle** out, int32_t sms, int32_t smem_optin, int32_t smem_per_sm) {
    if (!out || sms < 1 || smem_optin < 64 * 1024 || smem_per_sm < smem_optin) return NN_ERR_ARG;
    nn_handle* h = new (std::nothrow) nn_handle();
    if (!h) return NN_ERR_ARG;
    h->device = -1;
    h->offline = true;
    h->sms = sms;
    h->smem_optin = (size_t)smem_optin;
    h->smem_per_sm = (size_t)smem_per_sm;
    h->bucket_smem = h->smem_optin - 1024;
    *out = h;
    return NN_OK;
}

void nn_destroy(nn_handle* h) {
    if (!h) return;
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

nn_status nn_profile_enable(nn_handle* h, int enable) {
    if (!h || h->offline) return NN_ERR_ARG;
    if (enable && !h->ev[0])
        for (cudaEvent_t& e : h->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return NN_ERR_CUDA;
    h->pending = false;
    h->prof = enable != 0;
    for (double& a : h->acc) a = 0.0;
    h->calls = 0;
    return NN_OK;
}

nn_status nn_profile_read(nn_handle* h, double* ms, int64_t* calls, int n_stages) {
    if (!h || n_stages < 0 || n_stages > NN_PROFILE_STAGES) return NN_ERR_ARG;
    prof_flush(h);
    for (int i = 0; i < n_stages; ++i) ms[i] = h->acc[i];
    if (calls) *calls = h->calls;
    return NN_OK;
}

nn_status nn_query(nn_handle* h, const nn_mesh* mesh, int want, size_t* ws_bytes, int64_t* node_col_cap,
                   int64_t* elem_col_cap) {
    if (!h) return NN_ERR_ARG;
    Plan p;
    nn_status st = make_plan(h, mesh, want, &p);
    if (st != NN_OK) return st;
    if (ws_bytes) *ws_bytes = p.ws_rec;
    // bound on node entries: every incidence has at most k edge ends (2 tri/quad, 3 tet/hex)
    if (node_col_cap) *node_col_cap = (int64_t)p.k * p.n_conn;
    if (elem_col_cap) *elem_col_cap = p.n_conn;
    return NN_OK;
}

nn_status nn_plan_info(nn_handle* h, const nn_mesh* mesh, int want, int64_t* info, int n) {
    if (!h || (!info && n > 0) || n < 0) return NN_ERR_ARG;
    Plan p;
    nn_status st = make_plan(h, mesh, want, &p);
    if (st != NN_OK) return st;
    const int64_t v[9] = {p.fmt.sb, p.B, p.G, p.fmt.rb, (int64_t)p.ws_min, p.bucket_grid, p.bucket_threads,
                          (int64_t)p.bucket_smem, p.fmt.cshift};
    for (int i = 0; i < n && i < 9; ++i) info[i] = v[i];
    return NN_OK;
}

nn_status nn_element_neighbors_query(nn_handle* h, const nn_mesh* mesh, size_t* ws_bytes, int64_t* col_cap) {
    if (!h) return NN_ERR_ARG;
    nn_status st = check_mesh(mesh);
    if (st != NN_OK) return st;
    const size_t T = (size_t)mesh->n_elems;
    if (ws_bytes) *ws_bytes = align_up(T * 4) + align_up((adjacency_scan_tiles((int64_t)T) + 1) * 8) + ALIGN;
    // faces per element (6 at most) times two
    if (col_cap) *col_cap = (int64_t)T * (mesh->type == NN_TRI ? 6 : mesh->type == NN_HEX || mesh->type == NN_MIXED ? 12 : 8);
    return NN_OK;
}

nn_status nn_element_neighbors(nn_handle* h, const nn_mesh* mesh, const nn_csr* node_elems, nn_csr* out, void* ws,
                               size_t ws_bytes, int32_t* d_status, nn_stream_t stream) {
    if (!h || h->offline || !node_elems || !node_elems->row_ptr || !out || !out->row_ptr || !d_status) return NN_ERR_ARG;
    nn_status st = check_mesh(mesh);
    if (st != NN_OK) return st;
    if (out->col_capacity < 0 || (out->col_capacity > 0 && !out->col)) return NN_ERR_ARG;
    if (mesh->n_conn > 0 && !node_elems->col) return NN_ERR_ARG;
    size_t need = 0;
    nn_element_neighbors_query(h, mesh, &need, nullptr);
    if (ws_bytes < need || !ws || (reinterpret_cast<uintptr_t>(ws) & (ALIGN - 1))) return NN_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* w = static_cast<uint8_t*>(ws);
    const size_t T = (size_t)mesh->n_elems;
    const size_t off_lb = align_up(T * 4), off_ticket = off_lb + align_up((adjacency_scan_tiles((int64_t)T) + 1) * 8);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return NN_ERR_CUDA;
    if (cudaMemsetAsync(w + off_lb, 0, off_ticket + ALIGN - off_lb, s) != cudaSuccess) return NN_ERR_CUDA;
    if (T == 0) return cudaMemsetAsync(out->row_ptr, 0, 8, s) == cudaSuccess ? NN_OK : NN_ERR_CUDA;
    AdjParams p{};
    p.type = mesh->type;
    p.n_nodes = mesh->n_nodes;
    p.n_elems = mesh->n_elems;
    p.n_conn = mesh->n_conn;
    p.conn = mesh->conn;
    p.elem_ptr = mesh->elem_ptr;
    p.elem_type = mesh->elem_type;
    p.ne_rp = node_elems->row_ptr;
    p.ne_col = node_elems->col;
    p.cnt = reinterpret_cast<uint32_t*>(w);
    p.lb_state = reinterpret_cast<uint64_t*>(w + off_lb);
    p.ticket = reinterpret_cast<uint32_t*>(w + off_ticket);
    p.rp = out->row_ptr;
    p.col = out->col;
    p.cap = out->col_capacity;
    p.status = d_status;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sms * 8, ((int64_t)T + 255) / 256));
    return launch_adjacency(p, grid, s) == cudaSuccess ? NN_OK : NN_ERR_CUDA;
}

nn_status nn_set_tuning(nn_handle* h, const nn_tuning* t) {
    if (!h) return NN_ERR_ARG;
    if (!t) {
        h->tuning = nn_tuning{};
        return NN_OK;
    }
    if ((t->sb != 0 && (t->sb < SB_MIN || t->sb > SB_MAX)) ||
        (t->bucket_threads != 0 && t->bucket_threads != 128 && t->bucket_threads != 256) ||
        t->bucket_ctas_per_sm < 0 || t->bucket_ctas_per_sm > 8)
        return NN_ERR_ARG;
    h->tuning = *t;
    return NN_OK;
}

nn_status nn_neighbor_nodes(nn_handle* h, const nn_mesh* mesh, nn_csr* out, void* ws, size_t ws_bytes,
                            int32_t* d_status, nn_stream_t stream) {
    return run(h, mesh, NN_WANT_NODES, out, nullptr, ws, ws_bytes, d_status, reinterpret_cast<cudaStream_t>(stream));
}

nn_status nn_neighbor_elements(nn_handle* h, const nn_mesh* mesh, nn_csr* out, void* ws, size_t ws_bytes,
                               int32_t* d_status, nn_stream_t stream) {
    return run(h, mesh, NN_WANT_ELEMS, nullptr, out, ws, ws_bytes, d_status, reinterpret_cast<cudaStream_t>(stream));
}

nn_status nn_neighbors_both(nn_handle* h, const nn_mesh* mesh, nn_csr* nodes, nn_csr* elems, void* ws,
                            size_t ws_bytes, int32_t* d_status, nn_stream_t stream) {
    return run(h, mesh, NN_WANT_BOTH, nodes, elems, ws, ws_bytes, d_status, reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------ chunked builds

namespace {

// Whether kernels on device `dev` may dereference ptr: device or managed
// memory, pinned host memory mapped at the same address (unified
// addressing), or any host memory where the device reads pageable memory.
bool addressable(const void* ptr, int dev) {
    if (!ptr) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return true;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer == ptr;
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) return false;
    return pageable != 0;
}

bool on_device(const void* ptr) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool mesh_addressable(const nn_mesh* m, int dev) {
    return addressable(m->conn, dev) && addressable(m->elem_ptr, dev) && addressable(m->elem_type, dev);
}

}  // namespace

nn_status nn_chunk_slabs(const nn_mesh* mesh, int* shift, int* n_slabs) {
    nn_status st = check_mesh(mesh);
    if (st != NN_OK) return st;
    int sh = 0;
    while (((mesh->n_nodes + (1ll << sh) - 1) >> sh) > NN_CHUNK_SLABS_MAX) ++sh;
    if (shift) *shift = sh;
    if (n_slabs) *n_slabs = (int)((mesh->n_nodes + (1ll << sh) - 1) >> sh);
    return NN_OK;
}

nn_status nn_chunk_count(nn_handle* h, const nn_mesh* mesh, uint32_t* d_counts, int32_t* d_status,
                         nn_stream_t stream) {
    if (!h || h->offline || !d_status) return NN_ERR_ARG;
    int shift = 0, ns = 0;
    nn_status st = nn_chunk_slabs(mesh, &shift, &ns);
    if (st != NN_OK) return st;
    if (ns > 0 && !d_counts) return NN_ERR_ARG;
    if (!on_device(d_status) || (ns > 0 && !on_device(d_counts)) || !mesh_addressable(mesh, h->device))
        return NN_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return NN_ERR_CUDA;
    if (ns == 0) return NN_OK;
    if (cudaMemsetAsync(d_counts, 0, (size_t)ns * 4, s) != cudaSuccess) return NN_ERR_CUDA;
    if (mesh->n_elems == 0) return NN_OK;
    EmitParams ep{};
    ep.type = mesh->type;
    ep.n_nodes = mesh->n_nodes;
    ep.n_elems = mesh->n_elems;
    ep.n_conn = mesh->n_conn;
    ep.conn = mesh->conn;
    ep.elem_ptr = mesh->elem_ptr;
    ep.elem_type = mesh->elem_type;
    // element-walk CTAs as in a build: two per SM, each a fixed slice of elements
    const int64_t n_units = (mesh->n_elems + (mesh->type == NN_TRI ? 3 : 0)) / (mesh->type == NN_TRI ? 4 : 1);
    ep.n_cta = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sms * 2, (n_units + 2047) / 2048));
    ep.status = d_status;
    return launch_slab_count(ep, shift, ns, d_counts, s) == cudaSuccess ? NN_OK : NN_ERR_CUDA;
}

nn_status nn_chunk_query(nn_handle* h, const nn_mesh* mesh, int want, const nn_chunk* chunk, size_t* ws_bytes) {
    if (!h || !chunk || chunk->node_hi <= chunk->node_lo) return NN_ERR_ARG;
    Plan p;
    nn_status st = make_plan_range(h, mesh, want, chunk->node_lo, chunk->node_hi - chunk->node_lo, chunk->records, &p);
    if (st != NN_OK) return st;
    if (ws_bytes) *ws_bytes = ALIGN + p.ws_rec;  // the running CSR bases, then the chunk's plan
    return NN_OK;
}

nn_status nn_chunk_plan(nn_handle* h, const nn_mesh* mesh, int want, const uint32_t* counts, size_t ws_bytes,
                        nn_chunk* chunks, int max_chunks, int* n_chunks, size_t* ws_needed) {
    if (!h || !n_chunks || max_chunks < 0 || (max_chunks > 0 && !chunks)) return NN_ERR_ARG;
    int shift = 0, ns = 0;
    nn_status st = nn_chunk_slabs(mesh, &shift, &ns);
    if (st != NN_OK) return st;
    if (want < 1 || want > 3 || (ns > 0 && !counts)) return NN_ERR_ARG;
    const int64_t N = mesh->n_nodes;
    int64_t total = 0;
    for (int i = 0; i < ns; ++i) total += counts[i];
    if (total > mesh->n_conn) return NN_ERR_ARG;  // not this mesh's counts
    // workspace of the chunk of slabs i..j
    auto need = [&](int i, int j, int64_t rec, size_t* out) {
        const nn_chunk k{(int64_t)i << shift, std::min<int64_t>(N, (int64_t)(j + 1) << shift), rec};
        return nn_chunk_query(h, mesh, want, &k, out);
    };
    // the smallest workspace that admits a plan: the largest single slab
    size_t worst = ALIGN;
    for (int i = 0; i < ns; ++i) {
        size_t w1 = 0;
        if ((st = need(i, i, counts[i], &w1)) != NN_OK) return st;
        worst = std::max(worst, w1);
    }
    if (ws_needed) *ws_needed = worst;
    if (worst > ws_bytes) {
        *n_chunks = 0;
        return NN_ERR_WORKSPACE;
    }
    // greedy: each chunk takes slabs while its plan still fits the workspace
    int n = 0;
    for (int i = 0; i < ns;) {
        int j = i;
        int64_t rec = counts[i];
        while (j + 1 < ns) {
            size_t w2 = 0;
            if (need(i, j + 1, rec + counts[j + 1], &w2) != NN_OK || w2 > ws_bytes) break;
            ++j;
            rec += counts[j];
        }
        if (n < max_chunks)
            chunks[n] = nn_chunk{(int64_t)i << shift, std::min<int64_t>(N, (int64_t)(j + 1) << shift), rec};
        ++n;
        i = j + 1;
    }
    *n_chunks = n;
    return n > max_chunks ? NN_ERR_CAPACITY : NN_OK;
}

nn_status nn_neighbors_chunked(nn_handle* h, const nn_mesh* mesh, int want, const nn_chunk* chunks, int n_chunks,
                               nn_csr* nodes, nn_csr* elems, void* ws, size_t ws_bytes, int32_t* d_status,
                               nn_stream_t stream) {
    if (!h || h->offline || !d_status || n_chunks < 0 || (n_chunks > 0 && !chunks)) return NN_ERR_ARG;
    nn_status st = check_mesh(mesh);
    if (st != NN_OK) return st;
    if (want < 1 || want > 3) return NN_ERR_ARG;
    st = check_outputs(want, nodes, elems);
    if (st != NN_OK) return st;
    if (!ws) return NN_ERR_WORKSPACE;
    if ((reinterpret_cast<uintptr_t>(ws) & (ALIGN - 1)) || !on_device(ws) || !on_device(d_status) || !mesh_addressable(mesh, h->device)) return NN_ERR_ARG;
    if ((want & NN_WANT_NODES) && (!addressable(nodes->row_ptr, h->device) || !addressable(nodes->col, h->device)))
        return NN_ERR_ARG;
    if ((want & NN_WANT_ELEMS) && (!addressable(elems->row_ptr, h->device) || !addressable(elems->col, h->device)))
        return NN_ERR_ARG;
    const int64_t N = mesh->n_nodes;
    // the chunks must tile [0, N) in order
    if (N > 0 && (n_chunks == 0 || chunks[0].node_lo != 0 || chunks[n_chunks - 1].node_hi != N)) return NN_ERR_ARG;
    for (int c = 0; c < n_chunks; ++c) {
        const nn_chunk& k = chunks[c];
        if (k.node_hi <= k.node_lo || (c > 0 && k.node_lo != chunks[c - 1].node_hi) || k.records < 0 ||
            k.records > mesh->n_conn)
            return NN_ERR_ARG;
        Plan p;
        if ((st = make_plan_range(h, mesh, want, k.node_lo, k.node_hi - k.node_lo, k.records, &p)) != NN_OK)
            return st;
        if (ALIGN + p.ws_min > ws_bytes) return NN_ERR_WORKSPACE;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* w = static_cast<uint8_t*>(ws);
    int64_t* base = reinterpret_cast<int64_t*>(w);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return NN_ERR_CUDA;
    if (cudaMemsetAsync(base, 0, 2 * sizeof(int64_t), s) != cudaSuccess) return NN_ERR_CUDA;
    if (N == 0) {
        if ((want & NN_WANT_NODES) && cudaMemsetAsync(nodes->row_ptr, 0, 8, s) != cudaSuccess) return NN_ERR_CUDA;
        if ((want & NN_WANT_ELEMS) && cudaMemsetAsync(elems->row_ptr, 0, 8, s) != cudaSuccess) return NN_ERR_CUDA;
        return NN_OK;
    }
    uint8_t* cw = w + ALIGN;
    for (int c = 0; c < n_chunks; ++c) {
        Plan p;
        make_plan_range(h, mesh, want, chunks[c].node_lo, chunks[c].node_hi - chunks[c].node_lo, chunks[c].records, &p);
        if ((st = enqueue(h, mesh, p, nodes, elems, cw, ws_bytes - ALIGN, base, d_status, false, s)) != NN_OK)
            return st;
        const uint32_t* estart = (want & NN_WANT_ELEMS) ? reinterpret_cast<const uint32_t*>(cw + p.off_estart) : nullptr;
        const uint64_t* nstart = (want & NN_WANT_NODES) ? reinterpret_cast<const uint64_t*>(cw + p.off_nstart) : nullptr;
        if (launch_chunk_advance(base, estart, nstart, p.B, s) != cudaSuccess) return NN_ERR_CUDA;
    }
    return NN_OK;
}

nn_status nn_batch_query(nn_handle* h, const nn_batch_caps* caps, size_t* ws_bytes, size_t* staging_bytes) {
    BatchPlan bp;
    nn_status st = batch_plan(h, caps, &bp);
    if (st != NN_OK) return st;
    if (ws_bytes) *ws_bytes = bp.ws_rec;
    if (staging_bytes) *staging_bytes = bp.table_bytes;
    return NN_OK;
}

nn_status nn_batch_prepare(nn_handle* h, const nn_batch_caps* caps, const nn_mesh* meshes, const nn_csr* node_out,
                           const nn_csr* elem_out, int32_t* d_status, int n_meshes, void* staging,
                           size_t staging_bytes) {
    return batch_prepare(h, caps, meshes, node_out, elem_out, d_status, n_meshes, staging, staging_bytes);
}

nn_status nn_batch_launch(nn_handle* h, const nn_batch_caps* caps, const void* staging, void* ws, size_t ws_bytes,
                          nn_stream_t stream) {
    return batch_launch(h, caps, staging, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

const char* nn_status_str(nn_status s) {
    switch (s) {
        case NN_OK: return "ok";
        case NN_ERR_ARG: return "invalid argument";
        case NN_ERR_WORKSPACE: return "workspace too small";
        case NN_ERR_CAPACITY: return "output capacity too small";
        case NN_ERR_NODE_RANGE: return "node id out of range";
        case NN_ERR_ELEM_PTR: return "element offsets inconsistent with element types";
        case NN_ERR_TIMEOUT: return "device wait timed out";
        case NN_ERR_BUDGET: return "request exceeds memory budget";
        case NN_ERR_CUDA: return "CUDA error";
        case NN_ERR_BOUNDS: return "index outside its buffer (checked build)";
    }
    return "unknown status";
}

}  // extern "C"
