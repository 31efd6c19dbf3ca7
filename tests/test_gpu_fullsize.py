"""Full-size workloads in the benchmark's launch configuration.

The oracle cannot build these meshes whole in seconds, so each check uses what
holds at any size: rows of a seeded sample of nodes against the oracle's
sample-only walk (bit for bit), the closed-form sizes of the structured grids,
the sum of element rows (one entry per incidence), per-node element counts,
sorted rows without self entries, and symmetry of the node relation."""
import os

import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn
from tests import pins
from tests.gpu_util import env

pytestmark = pytest.mark.gpu

WORKLOADS = {
    "tri2048": (lambda: mg.workload_mesh("tri2048"), 2 * pins.tri_grid_edges(2047)),
    "tri2048_holes": (lambda: mg.workload_mesh("tri2048_holes"), None),
    "tet161": (lambda: mg.workload_mesh("tet161"), 2 * pins.kuhn_grid_edges(160)),
    "hex257": (lambda: mg.workload_mesh("hex257"), 2 * pins.hex_grid_edges(256)),
    "mixed257": (lambda: mg.workload_mesh("mixed257"), None),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


def build_on_gpu(mesh, builder, tune=True):
    """Build in the launch configuration the benchmark times: the autotuner's
    choice for this mesh class (timed afresh into a scratch cache)."""
    import tempfile
    import torch
    from paper_1604_04689_gb300 import autotune
    dm = nn.DeviceMesh.from_host(mesh)
    if tune:
        with tempfile.TemporaryDirectory() as d:
            autotune.tuned(builder, dm, nn.WANT_BOTH, path=os.path.join(d, "tune.json"))
    out = builder.alloc_outputs(dm, nn.WANT_BOTH)
    assert builder.launch(dm, nn.WANT_BOTH, out) == 0
    torch.cuda.synchronize()
    assert int(builder.status.item()) == 0
    return dm, {k: (rp, col[: int(rp[-1].item())]) for k, (rp, col) in out.items()}


def check_properties(mesh, dm, res, node_nnz):
    import torch
    N = mesh.n_nodes
    for k in ("nodes", "elems"):
        rp, col = res[k]
        assert int(rp[0].item()) == 0 and bool((rp[1:] >= rp[:-1]).all())
        lens = rp[1:] - rp[:-1]
        first = torch.zeros(col.numel(), dtype=torch.bool, device=col.device)
        first[rp[:-1][lens > 0]] = True
        d = col[1:].to(torch.int64) - col[:-1].to(torch.int64)
        assert bool((d[~first[1:]] > 0).all()), f"{k}: rows not strictly ascending"
    rp, col = res["nodes"]
    if node_nnz is not None:
        assert int(rp[-1].item()) == node_nnz
    src = torch.repeat_interleave(torch.arange(N, device=col.device), rp[1:] - rp[:-1])
    assert not bool((src == col).any())
    a = torch.sort(src * N + col.to(torch.int64)).values
    b = torch.sort(col.to(torch.int64) * N + src).values
    assert torch.equal(a, b), "node relation not symmetric"
    del src, a, b
    erp, ecol = res["elems"]
    assert int(erp[-1].item()) == mesh.n_conn            # no repeated node in any element
    inc = torch.bincount(dm.conn.to(torch.int64), minlength=N)
    assert torch.equal(erp[1:] - erp[:-1], inc)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_full_size_workload(name):
    mesh_fn, node_nnz = WORKLOADS[name]
    mesh = mesh_fn()
    b = nn.Builder()
    dm, res = build_on_gpu(mesh, b)
    rng = np.random.default_rng(17)
    sample = np.unique(np.concatenate([rng.integers(0, mesh.n_nodes, 3000), [0, mesh.n_nodes - 1]]))
    ref = oracle.rows(mesh, sample)
    assert ref["status"] == 0
    for k in ("nodes", "elems"):
        rp, col = (t.cpu().numpy() for t in res[k])
        got = np.concatenate([col[rp[v]:rp[v + 1]] for v in sample])
        got_len = np.array([rp[v + 1] - rp[v] for v in sample])
        np.testing.assert_array_equal(got_len, np.diff(ref[k][0]), err_msg=f"{name} {k} row lengths")
        np.testing.assert_array_equal(got, ref[k][1], err_msg=f"{name} {k} rows")
    check_properties(mesh, dm, res, node_nnz)


def test_more_than_65536_buckets():
    """Narrow buckets on a 1.2M-node mesh: 75K buckets, 512 buckets per coarse region."""
    mesh = mg.tri_grid(1100, 5, holes=0.02)
    with env(NN_SB=4):
        b = nn.Builder()
    plan = nn.nn_plan_info(b.h, nn.DeviceMesh.from_host(mesh).struct(), nn.WANT_BOTH)
    assert plan["n_buckets"] > 65536
    dm = nn.DeviceMesh.from_host(mesh)
    need = b.query(dm, nn.WANT_BOTH)[0] + 64 * mesh.n_conn
    ws = b.workspace(need)
    import torch
    out = b.alloc_outputs(dm, nn.WANT_BOTH)
    assert b.launch(dm, nn.WANT_BOTH, out, ws=ws, ws_bytes=need) == 0
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    res = {k: (rp, col[: int(rp[-1].item())]) for k, (rp, col) in out.items()}
    sample = np.random.default_rng(3).integers(0, mesh.n_nodes, 4000)
    ref = oracle.rows(mesh, sample)
    for k in ("nodes", "elems"):
        rp, col = (t.cpu().numpy() for t in res[k])
        got = np.concatenate([col[rp[v]:rp[v + 1]] for v in sample])
        np.testing.assert_array_equal(got, ref[k][1])
    check_properties(mesh, dm, res, None)
