"""GPU parity of the chunked build: the nodes are cut into chunks of
consecutive ids, each built in turn into its rows of the same CSRs, within
a bounded workspace.  Bit for bit against the oracle and the single build,
with planner-made and hand-made chunk boundaries, a host-resident mesh and
outputs (out of core), full size, and the error statuses."""
import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn
from tests.gpu_util import assert_same, gpu_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def builder():
    return nn.Builder()


def slab_counts(b, dm):
    """Per-slab incidence counts from the device kernel."""
    import torch
    s = dm.struct()
    shift, ns = nn.nn_chunk_slabs(s)
    counts = torch.zeros(max(ns, 1), dtype=torch.int32, device="cuda")
    assert nn.nn_chunk_count(b.h, s, counts.data_ptr(), b.status.data_ptr(), 0) == 0
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    return shift, [c & 0xFFFFFFFF for c in counts[:ns].cpu().tolist()]


def plan_at(b, dm, want, frac):
    """Chunks for a workspace `frac` of the way from the planner's minimum
    to the whole-mesh workspace; returns (chunks, ws_bytes)."""
    _, counts = slab_counts(b, dm)
    st, _, need = nn.nn_chunk_plan(b.h, dm.struct(), want, counts, 1 << 45)
    assert st == 0
    whole = b.query(dm, want)[0] + 256
    ws = int(need + frac * max(0, whole - need))
    st, chunks, _ = nn.nn_chunk_plan(b.h, dm.struct(), want, counts, ws)
    assert st == 0
    return chunks, ws


def run_chunked(b, dm, want, chunks, ws_bytes=None, out=None):
    import torch
    if ws_bytes is None:
        ws_bytes = max(nn.nn_chunk_query(b.h, dm.struct(), want, c) for c in chunks) if chunks else 256
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device="cuda")
    out = out if out is not None else b.alloc_outputs(dm, want)
    st = b.launch_chunked(dm, want, out, chunks, ws, ws_bytes)
    assert st == 0, nn.STATUS.get(st, st)
    torch.cuda.synchronize()
    status = int(b.status.item())
    res = {"status": status}
    for k, (rp, col) in out.items():
        rp = rp.cpu().numpy()
        res[k] = (rp, col.cpu().numpy()[: rp[-1]] if status == 0 else col.cpu().numpy())
    return res


MESHES = {
    "tri300": lambda: mg.tri_grid(300, 11),
    "tri300_holes": lambda: mg.tri_grid(300, 12, holes=0.05),
    "quad257": lambda: mg.quad_grid(257, 13),
    "tet41": lambda: mg.tet_grid(41, 14),
    "hex61": lambda: mg.hex_grid(61, 15),
    "mixed41": lambda: mg.mixed_grid(41, 17),
}


def test_slab_counts_are_incidences(builder):
    for name in ("tri300_holes", "mixed41", "hex61"):
        m = MESHES[name]()
        dm = nn.DeviceMesh.from_host(m)
        shift, counts = slab_counts(builder, dm)
        ref = np.bincount(m.conn.astype(np.int64) >> shift, minlength=len(counts))
        np.testing.assert_array_equal(np.array(counts), ref)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("want", [nn.WANT_BOTH, nn.WANT_NODES, nn.WANT_ELEMS])
def test_chunked_matches_oracle(name, want, builder):
    m = MESHES[name]()
    dm = nn.DeviceMesh.from_host(m)
    chunks, ws = plan_at(builder, dm, want, 0.3)
    assert len(chunks) >= 2
    res = run_chunked(builder, dm, want, chunks, ws)
    assert_same(res, oracle.neighbors(m, want), want)


@pytest.mark.parametrize("name", ["tri300", "tet41"])
def test_chunked_at_the_smallest_workspace(name, builder):
    """The planner's minimum: many small chunks."""
    m = MESHES[name]()
    dm = nn.DeviceMesh.from_host(m)
    chunks, ws = plan_at(builder, dm, nn.WANT_BOTH, 0.0)
    assert len(chunks) >= 8
    assert_same(run_chunked(builder, dm, nn.WANT_BOTH, chunks, ws), gpu_build(m, nn.WANT_BOTH, builder))


def records_of(m, lo, hi):
    return int(np.count_nonzero((m.conn >= lo) & (m.conn < hi)))


@pytest.mark.parametrize("name", ["tri300_holes", "tet41", "mixed41"])
def test_hand_made_chunks(name, builder):
    """Boundaries off the slabs and off any power of two, single-node chunks,
    and a chunk of nodes that no element touches."""
    m = MESHES[name]()
    n = m.n_nodes
    cuts = sorted({0, 1, 37, 38, 1001, n // 3, n // 3 + 5, n - 2, n})
    chunks = [(a, b, records_of(m, a, b)) for a, b in zip(cuts, cuts[1:]) if b > a]
    dm = nn.DeviceMesh.from_host(m)
    for want in (nn.WANT_BOTH, nn.WANT_NODES, nn.WANT_ELEMS):
        assert_same(run_chunked(builder, dm, want, chunks), oracle.neighbors(m, want), want)
    iso = mg.Mesh(m.etype, n + 500, m.conn, m.elem_ptr, m.elem_type)   # 500 trailing isolated nodes
    chunks = [(0, n // 2, records_of(iso, 0, n // 2)), (n // 2, n, records_of(iso, n // 2, n)), (n, n + 500, 0)]
    assert_same(run_chunked(builder, nn.DeviceMesh.from_host(iso), nn.WANT_BOTH, chunks), oracle.neighbors(iso))


def test_degenerate_elements_chunked(builder):
    """Repeated nodes: element-CSR offsets across chunk boundaries."""
    rng = np.random.default_rng(3)
    for m in (mg.tri_grid(200, 3), mg.tet_grid(25, 4), mg.hex_grid(30, 5)):
        conn = m.conn.reshape(m.n_elems, -1).copy()
        hit = rng.random(m.n_elems) < 0.05
        conn[hit, 1] = conn[hit, 0]
        d = mg.Mesh(m.etype, m.n_nodes, conn.ravel())
        n = d.n_nodes
        cuts = [0, n // 5, n // 2, n // 2 + 1, n]
        chunks = [(a, b, records_of(d, a, b)) for a, b in zip(cuts, cuts[1:])]
        assert_same(run_chunked(builder, nn.DeviceMesh.from_host(d), nn.WANT_BOTH, chunks), oracle.neighbors(d))


def test_empty_meshes_chunked(builder):
    import torch
    m0 = mg.Mesh(mg.TRI, 0, np.zeros(0, np.int32))
    r = run_chunked(builder, nn.DeviceMesh.from_host(m0), nn.WANT_BOTH, [], 256)
    assert r["status"] == 0 and r["nodes"][0].tolist() == [0] and r["elems"][0].tolist() == [0]
    m1 = mg.Mesh(mg.TET, 3000, np.zeros(0, np.int32))
    dm = nn.DeviceMesh.from_host(m1)
    chunks = builder.plan_chunks(dm, nn.WANT_BOTH, 1 << 26)
    assert chunks == [(0, 3000, 0)]
    assert_same(run_chunked(builder, dm, nn.WANT_BOTH, chunks), oracle.neighbors(m1))
    torch.cuda.synchronize()


def test_build_chunked_helper(builder):
    m = MESHES["hex61"]()
    dm = nn.DeviceMesh.from_host(m)
    whole = builder.query(dm, nn.WANT_BOTH)[0]
    res = builder.build_chunked(dm, nn.WANT_BOTH, ws_bytes=whole // 2)
    assert len(res["chunks"]) >= 2 and res["status"] == 0
    ref = oracle.neighbors(m)
    for k in ("nodes", "elems"):
        np.testing.assert_array_equal(res[k][0].cpu().numpy(), ref[k][0])
        np.testing.assert_array_equal(res[k][1].cpu().numpy(), ref[k][1])


def test_out_of_core_host_mesh_and_outputs(builder):
    """Connectivity and both CSRs in pinned host memory, only the workspace
    and the status word on the device."""
    import torch
    m = mg.tet_grid(30, 21)
    conn = torch.from_numpy(m.conn).pin_memory()
    dm = nn.DeviceMesh(m.etype, m.n_nodes, conn)
    _, nc, ec = builder.query(dm, nn.WANT_BOTH)
    out = {"nodes": (torch.empty(m.n_nodes + 1, dtype=torch.int64, pin_memory=True),
                     torch.empty(nc, dtype=torch.int32, pin_memory=True)),
           "elems": (torch.empty(m.n_nodes + 1, dtype=torch.int64, pin_memory=True),
                     torch.empty(ec, dtype=torch.int32, pin_memory=True))}
    n = m.n_nodes
    chunks = [(a, b, records_of(m, a, b)) for a, b in ((0, n // 3), (n // 3, 2 * n // 3), (2 * n // 3, n))]
    res = run_chunked(builder, dm, nn.WANT_BOTH, chunks, out=out)
    assert_same(res, oracle.neighbors(m))


def test_chunked_errors(builder):
    import torch
    m = MESHES["tet41"]()
    dm = nn.DeviceMesh.from_host(m)
    n = m.n_nodes
    good = [(0, n // 2, records_of(m, 0, n // 2)), (n // 2, n, records_of(m, n // 2, n))]
    ws_bytes = max(nn.nn_chunk_query(builder.h, dm.struct(), nn.WANT_BOTH, c) for c in good)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = builder.alloc_outputs(dm, nn.WANT_BOTH)
    L = builder.launch_chunked
    assert L(dm, nn.WANT_BOTH, out, [good[0]], ws, ws_bytes) == 1                     # does not reach n
    assert L(dm, nn.WANT_BOTH, out, [good[1], good[0]], ws, ws_bytes) == 1            # out of order
    assert L(dm, nn.WANT_BOTH, out, good, ws, 4096) == 2                              # workspace too small
    host_ws = torch.empty(ws_bytes, dtype=torch.uint8, pin_memory=True)
    assert L(dm, nn.WANT_BOTH, out, good, host_ws, ws_bytes) == 1                     # workspace not on the device
    # records below the true count: a device status, not a stray write
    stale = [(0, n // 2, good[0][2] - 100), good[1]]
    assert run_chunked(builder, dm, nn.WANT_BOTH, stale, ws_bytes)["status"] == 2
    # output capacity
    ref = oracle.neighbors(m)
    small = builder.alloc_outputs(dm, nn.WANT_BOTH, node_cap=int(ref["nodes"][0][-1]) - 1)
    assert run_chunked(builder, dm, nn.WANT_BOTH, good, ws_bytes, out=small)["status"] == 3
    # a bad node id is reported by the count pass
    bad = m.conn.copy()
    bad[77] = n + 3
    bdm = nn.DeviceMesh.from_host(mg.Mesh(m.etype, n, bad))
    with pytest.raises(nn.NNError) as e:
        builder.plan_chunks(bdm, nn.WANT_BOTH, 1 << 30)
    assert e.value.code == 4
    # and the chunked build itself
    assert run_chunked(builder, bdm, nn.WANT_BOTH, good, ws_bytes)["status"] == 4
    # after all that, a good build still matches
    assert_same(run_chunked(builder, dm, nn.WANT_BOTH, good, ws_bytes), ref)
