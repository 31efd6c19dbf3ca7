"""Serving loop on the GPU: every request's CSRs are the same alone (plain
server, one build per mesh), in a continuous batch, and in the oracle."""
import copy

import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn
from paper_1604_04689_gb300.serve import BatchServer, LaneCaps, PlainServer, Request

pytestmark = pytest.mark.gpu

GEN = {mg.TRI: mg.tri_grid, mg.QUAD: mg.quad_grid, mg.TET: mg.tet_grid, mg.HEX: mg.hex_grid}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


def small_requests(n, seed, spacing=2e-4):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        t = int(rng.choice([mg.TRI, mg.TET, mg.HEX, mg.QUAD]))
        side = int(rng.integers(3, 60 if t in (mg.TRI, mg.QUAD) else 18))
        out.append(Request(i, t, side, int(rng.integers(1 << 40)), i * spacing))
    return out


def test_device_generator_matches_host_generator():
    import torch
    for t, n, seed in ((mg.TRI, 37, 5), (mg.TRI, 2, 1), (mg.QUAD, 20, 9), (mg.TET, 9, 2), (mg.HEX, 11, 3),
                       (mg.TET, 2, 7), (mg.HEX, 2, 1 << 50)):
        dm = nn.generate_grid(t, n, seed)
        host = GEN[t](n, seed)
        torch.cuda.synchronize()
        assert dm.n_nodes == host.n_nodes
        np.testing.assert_array_equal(dm.conn.cpu().numpy(), host.conn)


def test_batched_equals_plain_equals_oracle():
    reqs_b = small_requests(80, 1)
    reqs_p = copy.deepcopy(reqs_b)
    caps = LaneCaps(max_meshes=8, max_elems=60000, max_nodes=60000, max_conn=400000)
    bs = BatchServer(budget_bytes=2 << 30, lanes=2, caps=caps, keep_results=True)
    sb = bs.run(reqs_b)
    assert sb["failed"] == 0 and sb["rejected"] == 0 and sb["batches"] > 5
    big = max(reqs_p, key=lambda r: r.n_conn)
    ps = PlainServer(big, keep_results=True)
    sp = ps.run(reqs_p)
    assert sp["failed"] == 0
    for rb, rp in zip(reqs_b, reqs_p):
        for k in ("nodes", "elems"):
            a_rp, a_col = rb.result[k]
            b_rp, b_col = rp.result[k]
            nnz = int(b_rp[-1].item())
            assert int(a_rp[-1].item()) == nnz
            assert bool((a_rp == b_rp).all()) and bool((a_col[:nnz] == b_col[:nnz]).all()), (rb.rid, k)
    for r in reqs_b[::9]:
        ref = oracle.neighbors(GEN[r.etype](r.n, r.seed))
        for k in ("nodes", "elems"):
            rp, col = r.result[k]
            np.testing.assert_array_equal(rp.cpu().numpy(), ref[k][0])
            np.testing.assert_array_equal(col[: int(rp[-1].item())].cpu().numpy(), ref[k][1])


def test_oversize_request_is_rejected_and_others_served():
    reqs = small_requests(10, 2)
    reqs.append(Request(10, mg.TRI, 300, 1, 0.0005))               # 178,802 tris: larger than a lane
    caps = LaneCaps(max_meshes=4, max_elems=50000, max_nodes=50000, max_conn=300000)
    bs = BatchServer(budget_bytes=1 << 30, lanes=2, caps=caps)
    st = bs.run(reqs)
    assert st["rejected"] == 1 and reqs[-1].status == 7
    assert all(r.status == 0 for r in reqs[:-1])
