"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit for
bit (integer output), on meshes the oracle finishes in seconds that span many
buckets and a ragged last bucket, on every element type, every result
selection, forced bucket widths and the spill path, and on edge cases."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn
from tests.gpu_util import assert_same, check_against_oracle, env, gpu_build

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "small_meshes.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def builder():
    return nn.Builder()


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("fx", golden(), ids=lambda f: f["name"])
def test_golden_fixtures(fx, builder):
    ep = np.array(fx["elem_ptr"], dtype=np.int64) if "elem_ptr" in fx else None
    et = np.array(fx["elem_type"], dtype=np.uint8) if "elem_type" in fx else None
    mesh = mg.Mesh(fx["type"], fx["n_nodes"], np.array(fx["conn"], dtype=np.int32), ep, et)
    res = gpu_build(mesh, nn.WANT_BOTH, builder)
    assert res["status"] == fx["status"]
    if fx["status"] == 0:
        for k in ("nodes", "elems"):
            rp, col = res[k]
            assert [col[rp[v]:rp[v + 1]].tolist() for v in range(mesh.n_nodes)] == fx[k]


MESHES = {
    "tri300": lambda: mg.tri_grid(300, 11),
    "tri300_holes": lambda: mg.tri_grid(300, 12, holes=0.05),
    "quad257": lambda: mg.quad_grid(257, 13),
    "tet41": lambda: mg.tet_grid(41, 14),
    "hex61": lambda: mg.hex_grid(61, 15),
    "hex37_elem_perm": lambda: mg.hex_grid(37, 16, permute_elems=True),
    "mixed41": lambda: mg.mixed_grid(41, 17),
    "tri64": lambda: mg.workload_mesh("tri64"),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("want", [nn.WANT_BOTH, nn.WANT_NODES, nn.WANT_ELEMS])
def test_parity_mid_size(name, want, builder):
    check_against_oracle(MESHES[name](), want, builder)


@pytest.mark.parametrize("sb", [4, 7, 11])
@pytest.mark.parametrize("name", ["tri300_holes", "tet41", "mixed41"])
def test_parity_forced_bucket_width(sb, name):
    with env(NN_SB=sb):
        b = nn.Builder()
    m = MESHES[name]()
    check_against_oracle(m, nn.WANT_BOTH, b, ws_extra=64 * m.n_conn)   # room for every bucket to spill


@pytest.mark.parametrize("name", ["tri300", "tet41", "hex61", "mixed41"])
def test_parity_spill_path(name):
    """Shared memory cut down so most buckets keep their tables in the spill area."""
    with env(NN_BUCKET_SMEM_KB=40, NN_SB=11):
        b = nn.Builder()
    m = MESHES[name]()
    check_against_oracle(m, nn.WANT_BOTH, b, ws_extra=64 * m.n_conn)


@pytest.mark.parametrize("name", ["tri300_holes", "tet41", "hex61", "mixed41"])
def test_parity_scattered_partition(name):
    """The one-pass partition with one scattered store per record (the fallback
    when the fine-digit field does not fit the record)."""
    with env(NN_PART="scatter"):
        b = nn.Builder()
    check_against_oracle(MESHES[name](), nn.WANT_BOTH, b)


@pytest.mark.parametrize("sb", [4, 6])
def test_parity_two_level_partition_many_buckets(sb):
    """Narrow buckets: thousands of buckets, coarse regions of up to 2^cshift buckets."""
    with env(NN_SB=sb):
        b = nn.Builder()
    m = mg.tet_grid(61, 31)
    check_against_oracle(m, nn.WANT_BOTH, b, ws_extra=64 * m.n_conn)


@pytest.mark.parametrize("chunk", [1, 37, 100, 600])
def test_parity_histogram_in_chunks(chunk):
    """More buckets than shared counters: the histogram walks the elements once per chunk
    (chunk 600: at most twice as many buckets as counters, one walk with 16-bit counters)."""
    with env(NN_HIST_CHUNK=chunk, NN_SB=6):
        b = nn.Builder()
    check_against_oracle(MESHES["mixed41"](), nn.WANT_BOTH, b, ws_extra=64 * MESHES["mixed41"]().n_conn)


def test_histogram_16_bit_count_wraps_and_is_counted_again():
    """One element-walk CTA over a fan of 300k triangles with 16-bit histogram
    counters: the hub's bucket passes 65535 records, the CTA sees the wrap
    and counts its slice again with 32-bit counters."""
    f = fan(300000)
    n_buckets = -(-f.n_nodes // 64)
    with env(NN_HIST_CHUNK=n_buckets // 2 + 1, NN_SB=6, NN_EMIT_CTAS=1):
        b = nn.Builder()
    check_against_oracle(f, nn.WANT_BOTH, b)


def fan(n_tri, hub=0, extra_nodes=3):
    """A closed fan of n_tri triangles around the hub (valence n_tri) plus isolated nodes."""
    el = [(mg.TRI, (hub, 1 + k, 1 + (k + 1) % n_tri)) for k in range(n_tri)]
    return mg.from_elements(el, n_tri + 1 + extra_nodes, f"fan{n_tri}")


@pytest.mark.parametrize("n_tri", [3, 33, 47, 48, 49, 100, 1000, 20000])
def test_high_valence_rows(n_tri, builder):
    check_against_oracle(fan(n_tri), nn.WANT_BOTH, builder)


def test_giant_row_spill():
    """A hub of valence 300k does not fit shared memory: spill tables + block sort."""
    check_against_oracle(fan(300000), nn.WANT_BOTH, nn.Builder())


def test_many_hubs_and_grid():
    """Several high-valence hubs inside one mesh, with a permuted triangle grid."""
    g = mg.tri_grid(120, 3)
    el = g.elements()
    base = g.n_nodes
    for h in range(5):
        hub = base + h * 2001
        el += [(mg.TRI, (hub, hub + 1 + k, hub + 1 + (k + 1) % 2000)) for k in range(2000)]
    m = mg.from_elements(el, base + 5 * 2001 + 7)
    check_against_oracle(m, nn.WANT_BOTH, nn.Builder())


def test_degenerate_elements(builder):
    rng = np.random.default_rng(5)
    for t, k in ((mg.TRI, 3), (mg.TET, 4), (mg.HEX, 8), (mg.QUAD, 4)):
        conn = rng.integers(0, 40, size=(3000, k)).astype(np.int32)   # many repeated nodes
        check_against_oracle(mg.Mesh(t, 45, conn.ravel()), nn.WANT_BOTH, builder)


@pytest.mark.parametrize("sb", [None, 4])
def test_degenerate_elements_many_buckets(sb):
    """Repeated nodes scattered over many buckets: element-CSR offsets of every
    bucket discount the repeated-node records of all buckets before it."""
    rng = np.random.default_rng(12)
    for m in (mg.tri_grid(200, 3), mg.tet_grid(25, 4), mg.hex_grid(30, 5)):
        conn = m.conn.reshape(m.n_elems, -1).copy()
        hit = rng.random(m.n_elems) < 0.05
        conn[hit, 1] = conn[hit, 0]                      # collapse one edge
        dm = mg.Mesh(m.etype, m.n_nodes, conn.ravel())
        with env(**({"NN_SB": sb} if sb else {})):
            b = nn.Builder()
        check_against_oracle(dm, nn.WANT_BOTH, b, ws_extra=64 * dm.n_conn)
        check_against_oracle(dm, nn.WANT_ELEMS, b, ws_extra=64 * dm.n_conn)


def test_random_mixed_soup(builder):
    rng = np.random.default_rng(9)
    el = []
    for e in range(20000):
        t = int(rng.integers(0, 4))
        el.append((t, tuple(int(x) for x in rng.integers(0, 5000, size=mg.NPE[t]))))
    check_against_oracle(mg.from_elements(el, 5003), nn.WANT_BOTH, builder)


def test_ragged_tri_counts(builder):
    """Triangle counts that are not a multiple of the 4-triangle load unit."""
    base = mg.tri_grid(40, 2)
    for drop in (1, 2, 3, 5):
        m = mg.Mesh(mg.TRI, base.n_nodes, base.conn[: base.conn.size - 3 * drop].copy())
        check_against_oracle(m, nn.WANT_BOTH, builder)


def test_empty_and_tiny(builder):
    for m in (mg.Mesh(mg.TRI, 7, np.zeros(0, np.int32)), mg.Mesh(mg.TET, 1, np.zeros(0, np.int32)),
              mg.Mesh(mg.HEX, 0, np.zeros(0, np.int32)), mg.tri_grid(2, 1), mg.tet_grid(2, 1),
              mg.Mesh(mg.QUAD, 4, np.array([0, 1, 2, 3], np.int32))):
        res = gpu_build(m, nn.WANT_BOTH, builder)
        ref = oracle.neighbors(m)
        assert_same(res, ref)


def test_node_range_error(builder):
    m = mg.tri_grid(50, 1)
    bad = m.conn.copy()
    bad[100] = m.n_nodes
    res = gpu_build(mg.Mesh(mg.TRI, m.n_nodes, bad), nn.WANT_BOTH, builder)
    assert res["status"] == 4
    bad[100] = -5
    assert gpu_build(mg.Mesh(mg.TRI, m.n_nodes, bad), nn.WANT_NODES, builder)["status"] == 4


def test_elem_ptr_error(builder):
    mx = mg.mixed_grid(8, 1)
    ep = mx.elem_ptr.copy()
    ep[5] += 1
    assert gpu_build(mg.Mesh(mg.MIXED, mx.n_nodes, mx.conn, ep, mx.elem_type), nn.WANT_BOTH, builder)["status"] == 5
    et = mx.elem_type.copy()
    et[3] = 7
    assert gpu_build(mg.Mesh(mg.MIXED, mx.n_nodes, mx.conn, mx.elem_ptr, et), nn.WANT_BOTH, builder)["status"] == 5


def test_capacity_error(builder):
    m = mg.tet_grid(12, 1)
    ref = oracle.neighbors(m)
    res = gpu_build(m, nn.WANT_NODES, builder, node_cap=int(ref["nodes"][0][-1]) - 1)
    assert res["status"] == 3
    res = gpu_build(m, nn.WANT_ELEMS, builder, elem_cap=int(ref["elems"][0][-1]) - 1)
    assert res["status"] == 3
    # exactly enough is fine
    res = gpu_build(m, nn.WANT_BOTH, builder, node_cap=int(ref["nodes"][0][-1]),
                    elem_cap=int(ref["elems"][0][-1]))
    assert_same(res, ref)


def test_workspace_errors():
    import torch
    b = nn.Builder()
    m = mg.tri_grid(50, 1)
    dm = nn.DeviceMesh.from_host(m)
    out = b.alloc_outputs(dm, nn.WANT_BOTH)
    need, _, _ = b.query(dm, nn.WANT_BOTH)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    assert b.launch(dm, nn.WANT_BOTH, out, ws=ws, ws_bytes=16) == 2          # host: below minimum
    # spill exhausted on the device: a giant hub with no spill space at all
    with env(NN_BUCKET_SMEM_KB=40):
        b2 = nn.Builder()
    f = fan(200000)
    dm = nn.DeviceMesh.from_host(f)
    out = b2.alloc_outputs(dm, nn.WANT_BOTH)
    need, _, _ = b2.query(dm, nn.WANT_BOTH)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    ws_min = nn.nn_plan_info(b2.h, dm.struct(), nn.WANT_BOTH)["ws_min"]          # no spill area at all
    st = b2.launch(dm, nn.WANT_BOTH, out, ws=ws, ws_bytes=ws_min)
    assert st == 0
    torch.cuda.synchronize()
    assert int(b2.status.item()) == 2


def test_bad_arguments(builder):
    import torch
    m = mg.tri_grid(10, 1)
    dm = nn.DeviceMesh.from_host(m)
    out = builder.alloc_outputs(dm, nn.WANT_BOTH)
    need, _, _ = builder.query(dm, nn.WANT_BOTH)
    ws = builder.workspace(need)
    mis = nn.DeviceMesh(dm.etype, dm.n_nodes, torch.zeros(dm.n_conn + 1, dtype=torch.int32, device="cuda")[1:])
    assert builder.launch(mis, nn.WANT_BOTH, out, ws=ws, ws_bytes=need) == 1    # conn not 16-byte aligned
    with pytest.raises(nn.NNError):
        builder.query(mis, nn.WANT_BOTH)
    bad = dm.struct()
    bad.type = 7                                                                # unknown element type
    with pytest.raises(nn.NNError):
        nn.nn_query(builder.h, bad, nn.WANT_BOTH)
    with pytest.raises(nn.NNError):
        nn.nn_query(builder.h, dm.struct(), 0)                                  # nothing wanted


def test_repeatable(builder):
    m = MESHES["mixed41"]()
    a = gpu_build(m, nn.WANT_BOTH, builder)
    b = gpu_build(m, nn.WANT_BOTH, builder)
    for k in ("nodes", "elems"):
        np.testing.assert_array_equal(a[k][0], b[k][0])
        np.testing.assert_array_equal(a[k][1], b[k][1])


def test_nonzero_stream(builder):
    import torch
    m = MESHES["tet41"]()
    ref = oracle.neighbors(m)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        res = gpu_build(m, nn.WANT_BOTH, builder)
    assert_same(res, ref)
