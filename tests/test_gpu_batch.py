"""Batched builds (one launch sequence for many meshes) against the oracle and
against single-mesh builds, bit for bit, including CUDA-graph replay of one
captured launch for different batches, per-mesh error isolation and the
capacity check."""
import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn
from tests.gpu_util import gpu_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


def batch_meshes(seed):
    rng = np.random.default_rng(seed)
    out = [mg.Mesh(mg.TRI, 0, np.zeros(0, np.int32)),            # no nodes at all
           mg.Mesh(mg.HEX, 9, np.zeros(0, np.int32)),            # nodes, no elements
           mg.tri_grid(2, 1), mg.tri_grid(3, 2)]
    for i in range(30):
        kind = int(rng.integers(0, 6))
        n = int(rng.integers(3, 40))
        if kind == 0:
            out.append(mg.tri_grid(n * 3, int(rng.integers(1 << 30))))
        elif kind == 1:
            out.append(mg.tet_grid(max(2, n // 2), int(rng.integers(1 << 30))))
        elif kind == 2:
            out.append(mg.hex_grid(max(2, n // 2), int(rng.integers(1 << 30)), permute_elems=bool(i & 1)))
        elif kind == 3:
            out.append(mg.mixed_grid(max(2, n // 2), int(rng.integers(1 << 30))))
        elif kind == 4:
            out.append(mg.tri_grid(n * 2, int(rng.integers(1 << 30)), holes=0.1))
        else:
            out.append(mg.quad_grid(n * 2, int(rng.integers(1 << 30))))
    # a fan with a high-valence hub
    out.append(mg.from_elements([(mg.TRI, (0, 1 + k, 1 + (k + 1) % 700)) for k in range(700)], 705))
    return out


def caps_for(meshes, slack=1.0):
    return dict(max_meshes=len(meshes) + 4,
                max_elems=int(sum(m.n_elems for m in meshes) * slack) + 16,
                max_nodes=int(sum(m.n_nodes for m in meshes) * slack) + 16,
                max_conn=int(sum(m.n_conn for m in meshes) * slack) + 64)


def check(res, mesh):
    ref = oracle.neighbors(mesh)
    assert res["status"] == 0 == ref["status"]
    for k in ("nodes", "elems"):
        np.testing.assert_array_equal(res[k][0].cpu().numpy(), ref[k][0], err_msg=f"{mesh.name} {k} row_ptr")
        np.testing.assert_array_equal(res[k][1].cpu().numpy(), ref[k][1], err_msg=f"{mesh.name} {k} col")


@pytest.mark.parametrize("sb", [0, 5, 9])
def test_batch_matches_oracle(sb):
    meshes = batch_meshes(1)
    caps = caps_for(meshes)
    bb = nn.BatchBuilder(**caps, sb=sb, extra_ws=64 * caps["max_conn"])   # wide buckets spill
    res = bb.run([nn.DeviceMesh.from_host(m) for m in meshes])
    for r, m in zip(res, meshes):
        check(r, m)


def test_batch_equals_single_builds():
    meshes = batch_meshes(2)
    bb = nn.BatchBuilder(**caps_for(meshes))
    res = bb.run([nn.DeviceMesh.from_host(m) for m in meshes])
    b = nn.Builder()
    for r, m in zip(res, meshes):
        single = gpu_build(m, nn.WANT_BOTH, b)
        for k in ("nodes", "elems"):
            np.testing.assert_array_equal(r[k][0].cpu().numpy(), single[k][0])
            np.testing.assert_array_equal(r[k][1].cpu().numpy(), single[k][1])


def test_graph_replay_of_one_capture_serves_different_batches():
    import torch
    a, b2 = batch_meshes(3), batch_meshes(4)
    caps = caps_for(a + b2)
    bb = nn.BatchBuilder(**caps)
    da = [nn.DeviceMesh.from_host(m) for m in a]
    db = [nn.DeviceMesh.from_host(m) for m in b2]
    outs_a = [bb.alloc_outputs(d) for d in da]
    outs_b = [bb.alloc_outputs(d) for d in db]
    assert bb.prepare(da, outs_a) == 0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        assert bb.launch(s) == 0          # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert bb.launch(s) == 0
    for meshes, dms, outs in ((a, da, outs_a), (b2, db, outs_b), (a, da, outs_a)):
        for o in outs:
            for rp, col in o.values():
                rp.fill_(-3)
        assert bb.prepare(dms, outs) == 0
        g.replay()
        torch.cuda.synchronize()
        stat = bb.status[: len(dms)].cpu().tolist()
        for st, o, m in zip(stat, outs, meshes):
            r = {"status": st}
            for k, (rp, col) in o.items():
                r[k] = (rp, col[: int(rp[-1].item())])
            check(r, m)


def test_errors_stay_with_their_mesh():
    meshes = batch_meshes(5)[:12]
    bad = meshes[6]
    conn = bad.conn.copy()
    conn[0] = bad.n_nodes + 5
    meshes[6] = mg.Mesh(bad.etype, bad.n_nodes, conn, bad.elem_ptr, bad.elem_type, "bad")
    bb = nn.BatchBuilder(**caps_for(meshes))
    res = bb.run([nn.DeviceMesh.from_host(m) for m in meshes])
    for i, (r, m) in enumerate(zip(res, meshes)):
        if i == 6:
            assert r["status"] == 4
        else:
            check(r, m)


def test_capacity_is_checked_on_the_host():
    meshes = batch_meshes(6)[:8]
    caps = caps_for(meshes)
    caps["max_conn"] = sum(m.n_conn for m in meshes) - 1
    bb = nn.BatchBuilder(**caps)
    dms = [nn.DeviceMesh.from_host(m) for m in meshes]
    assert bb.prepare(dms, [bb.alloc_outputs(d) for d in dms]) == 7     # NN_ERR_BUDGET
    small = nn.BatchBuilder(max_meshes=2, max_elems=10**6, max_nodes=10**6, max_conn=10**6)
    assert small.prepare(dms, [small.alloc_outputs(d) for d in dms]) == 1   # more meshes than slots


@pytest.mark.parametrize("want", [nn.WANT_BOTH, nn.WANT_NODES, nn.WANT_ELEMS])
def test_one_call_submit_equals_the_oracle(want):
    """nn_batch_submit: two batches enqueued back to back on one stream (the
    first one's staging is still in use when the second is prepared), each
    mesh's CSRs equal to the oracle's."""
    import torch
    h = nn.nn_create()
    try:
        stream = torch.cuda.current_stream().cuda_stream
        runs = []
        for meshes in (batch_meshes(7)[:14], batch_meshes(8)[2:12]):
            dms = [nn.DeviceMesh.from_host(m) for m in meshes]
            n = len(dms)
            arr = (nn.NNMesh * n)(*[d.struct() for d in dms])
            ws_bytes = nn.nn_batch_submit_query(h, arr, n, want)
            ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
            status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            outs = []
            for d in dms:
                o = {}
                if want & nn.WANT_NODES:
                    k = 2 if d.etype in (nn.TRI, nn.QUAD) else 3
                    o["nodes"] = (torch.empty(d.n_nodes + 1, dtype=torch.int64, device="cuda"),
                                  torch.empty(max(k * d.n_conn, 1), dtype=torch.int32, device="cuda"))
                if want & nn.WANT_ELEMS:
                    o["elems"] = (torch.empty(d.n_nodes + 1, dtype=torch.int64, device="cuda"),
                                  torch.empty(max(d.n_conn, 1), dtype=torch.int32, device="cuda"))
                outs.append(o)

            def csrs(key):
                if key not in outs[0]:
                    return None
                return (nn.NNCSR * n)(*[nn.NNCSR(o[key][0].data_ptr(), o[key][1].data_ptr(), o[key][1].numel())
                                        for o in outs])
            node_arr, elem_arr = csrs("nodes"), csrs("elems")
            st = nn.nn_batch_submit(h, arr, node_arr, elem_arr, n, ws.data_ptr(), ws_bytes, status.data_ptr(),
                                    stream)
            assert st == 0, nn.STATUS.get(st, st)
            runs.append((meshes, dms, outs, status, ws, arr, node_arr, elem_arr))
        torch.cuda.synchronize()
        for meshes, _, outs, status, *_ in runs:
            assert status.cpu().tolist() == [0] * len(meshes)
            for m, o in zip(meshes, outs):
                ref = oracle.neighbors(m, want)
                for key, (rp, col) in o.items():
                    rp = rp.cpu().numpy()
                    np.testing.assert_array_equal(rp, ref[key][0], err_msg=f"{m.name} {key} row_ptr")
                    np.testing.assert_array_equal(col.cpu().numpy()[: rp[-1]], ref[key][1],
                                                  err_msg=f"{m.name} {key} col")
    finally:
        nn.nn_destroy(h)


def test_one_call_submit_refuses_a_capturing_stream():
    """nn_batch_submit frees its host staging from the stream; captured into a
    graph that would run on every replay, so a capturing stream is refused
    with NN_ERR_ARG and nothing is enqueued (the captured graph stays empty)."""
    import torch
    h = nn.nn_create()
    try:
        meshes = batch_meshes(9)[:3]
        dms = [nn.DeviceMesh.from_host(m) for m in meshes]
        n = len(dms)
        arr = (nn.NNMesh * n)(*[d.struct() for d in dms])
        ws_bytes = nn.nn_batch_submit_query(h, arr, n, nn.WANT_ELEMS)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        status = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        outs = [(torch.full((d.n_nodes + 1,), -3, dtype=torch.int64, device="cuda"),
                 torch.empty(max(d.n_conn, 1), dtype=torch.int32, device="cuda")) for d in dms]
        elem_arr = (nn.NNCSR * n)(*[nn.NNCSR(rp.data_ptr(), col.data_ptr(), col.numel()) for rp, col in outs])
        side = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            st = nn.nn_batch_submit(h, arr, None, elem_arr, n, ws.data_ptr(), ws_bytes, status.data_ptr(),
                                    side.cuda_stream)
        assert st == 1                               # NN_ERR_ARG
        g.replay()                                   # the empty graph: nothing was captured
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [-5] * n
        assert all(int(rp[0].item()) == -3 for rp, _ in outs)
    finally:
        nn.nn_destroy(h)
