"""Host-side rules of the C ABI, checked without a GPU on the offline sizing
handle: argument validation, the documented capacity bounds, tuning limits,
size-only queries of the grid generator, compute calls refused on an
offline handle, and no fallback when libnn.so is missing.

Mesh pointers are never dereferenced by these host-only calls, so fake
addresses stand in for device memory (16-byte aligned unless a test wants
otherwise)."""
import ctypes as C

import pytest

from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn

FAKE = 1 << 20
ARG, WS, CAP = 1, 2, 3


@pytest.fixture(scope="module")
def h():
    from paper_1604_04689_gb300 import build
    build.build()
    handle = nn.nn_create_offline()
    yield handle
    nn.nn_destroy(handle)


def uniform(etype, n_nodes, n_elems, conn=FAKE, n_conn=None):
    if n_conn is None:
        n_conn = n_elems * nn.NPE[etype]
    return nn.NNMesh(etype, n_nodes, n_elems, n_conn, conn if n_conn else None, None, None)


def query_status(h, mesh, want=nn.WANT_BOTH):
    ws, nc, ec = C.c_size_t(), C.c_int64(), C.c_int64()
    return nn.lib().nn_query(h, C.byref(mesh), want, C.byref(ws), C.byref(nc), C.byref(ec))


# ------------------------------------------------------------ capacity bounds

@pytest.mark.parametrize("etype,edge_ends", [(nn.TRI, 6), (nn.QUAD, 8), (nn.TET, 12), (nn.HEX, 24)])
def test_capacity_bounds_are_the_edge_ends(h, etype, edge_ends):
    """Node col bound = both ends of every local edge of every element (tri 3
    edges, quad 4, tet 6, hex 12); element col bound = one entry per incidence."""
    T = 1000
    ws, nc, ec = nn.nn_query(h, uniform(etype, 5000, T), nn.WANT_BOTH)
    assert nc == edge_ends * T
    assert ec == nn.NPE[etype] * T
    assert ws >= nn.nn_plan_info(h, uniform(etype, 5000, T), nn.WANT_BOTH)["ws_min"] > 0


def test_capacity_bounds_hold_on_a_real_mesh(h):
    """The bounds are at least the true result sizes (oracle-free: closed forms
    of the hex grid, E = 3 m n^2 edges, 8 incidences per cell)."""
    m = mg.hex_grid(9, 1)
    s = nn.NNMesh(nn.HEX, m.n_nodes, m.n_elems, m.conn.size, FAKE, None, None)
    _, nc, ec = nn.nn_query(h, s, nn.WANT_BOTH)
    assert nc >= 2 * 3 * 8 * 81
    assert ec == 8 * m.n_elems


def test_mixed_bound_uses_three_edge_ends_per_incidence(h):
    m = mg.mixed_grid(7, 3)
    s = nn.NNMesh(nn.MIXED, m.n_nodes, m.n_elems, m.conn.size, FAKE, FAKE, FAKE)
    _, nc, ec = nn.nn_query(h, s, nn.WANT_BOTH)
    assert nc == 3 * m.conn.size and ec == m.conn.size


def test_empty_mesh_is_valid(h):
    ws, nc, ec = nn.nn_query(h, uniform(nn.TRI, 0, 0), nn.WANT_BOTH)
    assert (nc, ec) == (0, 0) and ws > 0
    ws, nc, ec = nn.nn_query(h, uniform(nn.TET, 17, 0), nn.WANT_NODES)
    assert (nc, ec) == (0, 0)


# ------------------------------------------------------------ argument errors

@pytest.mark.parametrize("case", [
    "type", "neg_nodes", "nodes_2_31", "elems_2_31", "conn_mismatch", "null_conn", "misaligned_conn",
    "mixed_no_ptr", "mixed_no_types", "mixed_misaligned_ptr", "want0", "want4", "null_mesh"])
def test_nn_query_rejects(h, case):
    want = nn.WANT_BOTH
    m = uniform(nn.TRI, 100, 10)
    if case == "type":
        m.type = 7
    elif case == "neg_nodes":
        m.n_nodes = -1
    elif case == "nodes_2_31":
        m.n_nodes = 1 << 31
    elif case == "elems_2_31":
        m = uniform(nn.TRI, 100, 1 << 31)
    elif case == "conn_mismatch":
        m.n_conn = 31
    elif case == "null_conn":
        m.conn = None
    elif case == "misaligned_conn":
        m.conn = FAKE + 4
    elif case == "mixed_no_ptr":
        m = nn.NNMesh(nn.MIXED, 100, 10, 40, FAKE, None, FAKE)
    elif case == "mixed_no_types":
        m = nn.NNMesh(nn.MIXED, 100, 10, 40, FAKE, FAKE, None)
    elif case == "mixed_misaligned_ptr":
        m = nn.NNMesh(nn.MIXED, 100, 10, 40, FAKE, FAKE + 4, FAKE)
    elif case == "want0":
        want = 0
    elif case == "want4":
        want = 4
    if case == "null_mesh":
        assert nn.lib().nn_query(h, None, want, None, None, None) == ARG
    else:
        assert query_status(h, m, want) == ARG


def test_mixed_conn_need_not_be_16_byte_aligned(h):
    """Only uniform meshes are read as 16-byte vectors; a mixed mesh's conn
    is read element by element through elem_ptr."""
    m = nn.NNMesh(nn.MIXED, 100, 10, 40, FAKE + 4, FAKE, FAKE)
    assert query_status(h, m) == 0


def test_null_handle_is_an_argument_error():
    m = uniform(nn.TRI, 100, 10)
    assert nn.lib().nn_query(None, C.byref(m), nn.WANT_BOTH, None, None, None) == ARG


# ------------------------------------------------------------ tuning

@pytest.mark.parametrize("tuning,ok", [
    ({"sb": 4}, True), ({"sb": 11}, True), ({"sb": 3}, False), ({"sb": 12}, False),
    ({"bucket_threads": 128}, True), ({"bucket_threads": 256}, True), ({"bucket_threads": 512}, False),
    ({"bucket_threads": 64}, False), ({"bucket_ctas_per_sm": 8}, True), ({"bucket_ctas_per_sm": 9}, False),
    ({"bucket_ctas_per_sm": -1}, False), ({}, True)])
def test_tuning_limits(tuning, ok):
    hh = nn.nn_create_offline()
    try:
        if ok:
            nn.nn_set_tuning(hh, tuning)
        else:
            with pytest.raises(nn.NNError) as e:
                nn.nn_set_tuning(hh, tuning)
            assert e.value.code == ARG
        nn.nn_set_tuning(hh, None)
    finally:
        nn.nn_destroy(hh)


def test_tuning_changes_the_plan_not_the_bounds():
    """A forced bucket width shows in the plan; the result bounds stay the same."""
    hh = nn.nn_create_offline()
    try:
        m = uniform(nn.TET, 200_000, 1_000_000)
        base = nn.nn_query(hh, m, nn.WANT_BOTH)
        for sb in (5, 9):
            nn.nn_set_tuning(hh, {"sb": sb})
            assert nn.nn_plan_info(hh, m, nn.WANT_BOTH)["sb"] == sb
            assert nn.nn_query(hh, m, nn.WANT_BOTH)[1:] == base[1:]
    finally:
        nn.nn_destroy(hh)


# ------------------------------------------------------------ offline handle refuses compute

def test_compute_calls_refuse_the_offline_handle(h):
    L = nn.lib()
    m = uniform(nn.TRI, 100, 10)
    out = nn.NNCSR(FAKE, FAKE, 1000)
    out2 = nn.NNCSR(FAKE, FAKE, 1000)
    ws, st = FAKE, FAKE
    assert L.nn_neighbor_nodes(h, C.byref(m), C.byref(out), ws, 1 << 30, st, None) == ARG
    assert L.nn_neighbor_elements(h, C.byref(m), C.byref(out), ws, 1 << 30, st, None) == ARG
    assert L.nn_neighbors_both(h, C.byref(m), C.byref(out), C.byref(out2), ws, 1 << 30, st, None) == ARG
    assert L.nn_element_neighbors(h, C.byref(m), C.byref(out), C.byref(out2), ws, 1 << 30, st, None) == ARG
    assert L.nn_chunk_count(h, C.byref(m), FAKE, st, None) == ARG
    chunk = nn.NNChunk(0, 100, 30)
    assert L.nn_neighbors_chunked(h, C.byref(m), nn.WANT_BOTH, C.byref(chunk), 1, C.byref(out), C.byref(out2),
                                  ws, 1 << 30, st, None) == ARG
    assert L.nn_profile_enable(h, 1) == ARG
    caps = nn.NNBatchCaps(4, nn.WANT_BOTH, 1000, 1000, 4000, 0)
    assert L.nn_batch_launch(h, C.byref(caps), FAKE, ws, 1 << 30, None) == ARG


def test_offline_handle_limits_are_checked():
    hh = C.c_void_p()
    assert nn.lib().nn_create_offline(C.byref(hh), 0, 232448, 233472) == ARG
    assert nn.lib().nn_create_offline(C.byref(hh), 152, 1024, 233472) == ARG
    assert nn.lib().nn_create_offline(C.byref(hh), 152, 232448, 1024) == ARG


# ------------------------------------------------------------ batches, adjacency, generator sizes

def test_batch_query_grows_with_capacity(h):
    small = nn.nn_batch_query(h, nn.NNBatchCaps(8, nn.WANT_BOTH, 10_000, 10_000, 40_000, 0))
    large = nn.nn_batch_query(h, nn.NNBatchCaps(8, nn.WANT_BOTH, 1_000_000, 1_000_000, 4_000_000, 0))
    assert all(x > 0 for x in small) and large[0] > small[0]


def test_batch_query_rejects_bad_caps(h):
    for caps in (nn.NNBatchCaps(8, nn.WANT_BOTH, 1 << 31, 1000, 4000, 0),
                 nn.NNBatchCaps(8, nn.WANT_BOTH, 1000, 1000, 1 << 31, 0),
                 nn.NNBatchCaps(8, nn.WANT_BOTH, 1000, 1000, 4000, 3),
                 nn.NNBatchCaps(8, nn.WANT_BOTH, 1000, 1000, 4000, 12)):
        with pytest.raises(nn.NNError) as e:
            nn.nn_batch_query(h, caps)
        assert e.value.code == ARG


@pytest.mark.parametrize("etype,faces", [(nn.TRI, 3), (nn.QUAD, 4), (nn.TET, 4), (nn.HEX, 6)])
def test_element_adjacency_bound(h, etype, faces):
    """Two entries per face of every element: each face borders at most two
    elements on the far side when a split face meets two triangles."""
    T = 777
    _, cap = nn.nn_element_neighbors_query(h, uniform(etype, 5000, T))
    assert cap == 2 * faces * T


@pytest.mark.parametrize("etype", [nn.TRI, nn.QUAD, nn.TET, nn.HEX])
@pytest.mark.parametrize("n", [2, 3, 17])
def test_generator_size_query_matches_host_generator(etype, n):
    """nn_generate_grid with conn == NULL only reports sizes (no device work);
    they equal the host generator's meshes."""
    nn_, ne = C.c_int64(), C.c_int64()
    st = nn.lib().nn_generate_grid(etype, n, 1, 1, 1, None, 0, C.byref(nn_), C.byref(ne), None)
    assert st == 0
    host = {nn.TRI: mg.tri_grid, nn.QUAD: mg.quad_grid, nn.TET: mg.tet_grid, nn.HEX: mg.hex_grid}[etype](n, 1)
    assert (nn_.value, ne.value) == (host.n_nodes, host.n_elems)


@pytest.mark.parametrize("etype,n", [(7, 10), (nn.TRI, 1), (nn.TRI, (1 << 20) + 1), (nn.HEX, 1291)])
def test_generator_rejects(etype, n):
    nn_, ne = C.c_int64(), C.c_int64()
    assert nn.lib().nn_generate_grid(etype, n, 1, 1, 1, None, 0, C.byref(nn_), C.byref(ne), None) == ARG


def test_generator_capacity_error_before_any_launch():
    nn_, ne = C.c_int64(), C.c_int64()
    st = nn.lib().nn_generate_grid(nn.TET, 5, 1, 1, 1, FAKE, 10, C.byref(nn_), C.byref(ne), None)
    assert st == CAP


# ------------------------------------------------------------ statuses, no fallback

def test_every_status_has_its_own_text():
    texts = [nn.lib().nn_status_str(s) for s in range(10)]
    assert len(set(texts)) == 10 and all(texts)
    assert nn.lib().nn_status_str(99) == b"unknown status"


def test_missing_library_raises(monkeypatch, tmp_path):
    """The binding loads libnn.so or raises; there is no CPU path to fall back on."""
    monkeypatch.setattr(nn, "LIB_PATH", str(tmp_path / "libnn.so"))
    monkeypatch.setattr(nn, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        nn.lib()
    with pytest.raises(RuntimeError, match="not built"):
        nn.nn_create_offline()


# ------------------------------------------------------------ build plan (host planner)

PLAN_MESHES = {
    "tri64": (nn.TRI, 4096, 7938),
    "tri2048": (nn.TRI, 4_194_304, 8_380_418),
    "tet161": (nn.TET, 4_173_281, 24_576_000),
    "hex257": (nn.HEX, 16_974_593, 16_777_216),
    "quad300": (nn.QUAD, 90_000, 89_401),
}


@pytest.mark.parametrize("name", sorted(PLAN_MESHES))
@pytest.mark.parametrize("want", [nn.WANT_NODES, nn.WANT_ELEMS, nn.WANT_BOTH])
def test_plan_covers_the_nodes_and_holds_the_records(h, name, want):
    etype, N, T = PLAN_MESHES[name]
    m = uniform(etype, N, T)
    p = nn.nn_plan_info(h, m, want)
    ws, _, _ = nn.nn_query(h, m, want)
    n_conn = nn.NPE[etype] * T
    # the buckets tile [0, N): 2^sb consecutive ids each, the last one partial
    assert 4 <= p["sb"] <= 11
    assert (p["n_buckets"] - 1) << p["sb"] < N <= p["n_buckets"] << p["sb"]
    # one packed record per incidence, 8 or 16 bytes, in the minimum workspace
    assert p["record_bytes"] in (8, 16)
    assert p["ws_min"] >= n_conn * p["record_bytes"]
    # the recommended workspace adds a spill area of 16 MiB + 8 B per incidence
    assert ws == p["ws_min"] + (16 << 20) + 8 * n_conn
    # tile-sorted partition: one pass up to 256 buckets, else coarse regions of
    # 2^k buckets, at most 256 of them and at most 4096 buckets each
    if p["n_buckets"] <= 256:
        assert p["partition"] == 0
    else:
        k = p["partition"]
        assert 0 < k <= 12 and (p["n_buckets"] + (1 << k) - 1) >> k <= 256
    assert p["bucket_threads"] in (128, 256)
    assert 1 <= p["bucket_ctas"] <= p["n_buckets"]
    assert p["bucket_smem"] <= 233472


def test_record_width_follows_the_fields(h):
    """Small meshes pack a record in 64 bits; the 2048^2 triangle grid (23-bit
    element ids and two 23-bit neighbour fields) needs 128, unless only the
    element rows are wanted (no neighbour fields)."""
    assert nn.nn_plan_info(h, uniform(*PLAN_MESHES["tri64"]), nn.WANT_BOTH)["record_bytes"] == 8
    assert nn.nn_plan_info(h, uniform(*PLAN_MESHES["tri2048"]), nn.WANT_BOTH)["record_bytes"] == 16
    assert nn.nn_plan_info(h, uniform(*PLAN_MESHES["tri2048"]), nn.WANT_ELEMS)["record_bytes"] == 8


def test_workspace_grows_with_the_mesh(h):
    sizes = [nn.nn_query(h, uniform(nn.TET, 6 * n * n * n // 5, 6 * n * n * n), nn.WANT_BOTH)[0]
             for n in (10, 40, 160)]
    assert sizes[0] < sizes[1] < sizes[2]


def test_wait_probe_checks_its_pointers_on_the_host():
    """The bounded-wait diagnostic rejects null and misaligned pointers before
    touching the device."""
    L = nn.lib()
    assert L.nn_diag_wait_timeout(None, FAKE, None) == ARG
    assert L.nn_diag_wait_timeout(FAKE, None, None) == ARG
    assert L.nn_diag_wait_timeout(FAKE + 4, FAKE, None) == ARG
    assert L.nn_diag_wait_timeout(FAKE, FAKE + 2, None) == ARG


def test_batch_submit_host_rules(h):
    """The one-call batch sizes its workspace as the three-step batch does for
    the meshes' totals, and refuses bad requests before touching the device."""
    L = nn.lib()
    ms = [uniform(nn.TRI, 100, 150), uniform(nn.HEX, 64, 27), uniform(nn.TET, 50, 120)]
    arr = (nn.NNMesh * 3)(*ms)
    ws = nn.nn_batch_submit_query(h, arr, 3, nn.WANT_BOTH)
    caps = nn.NNBatchCaps(3, nn.WANT_BOTH, sum(m.n_elems for m in ms), sum(m.n_nodes for m in ms),
                          sum(m.n_conn for m in ms), 0)
    assert ws == nn.nn_batch_query(h, caps)[0]
    outs = (nn.NNCSR * 3)(*[nn.NNCSR(FAKE, FAKE, 10_000) for _ in ms])
    assert L.nn_batch_submit(h, arr, None, None, 3, FAKE, ws, FAKE, None) == ARG       # no output wanted
    assert L.nn_batch_submit(h, arr, outs, outs, 3, FAKE, ws, FAKE, None) == ARG       # offline handle
    assert L.nn_batch_submit(h, arr, outs, outs, 0, FAKE, ws, FAKE, None) == 0         # nothing to do
    assert L.nn_batch_submit(h, None, outs, outs, 2, FAKE, ws, FAKE, None) == ARG
    bad = (nn.NNMesh * 1)(uniform(nn.TRI, -1, 2))
    with pytest.raises(nn.NNError):
        nn.nn_batch_submit_query(h, bad, 1, nn.WANT_BOTH)
