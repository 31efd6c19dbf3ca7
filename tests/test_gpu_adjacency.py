"""GPU element face adjacency through the C ABI against the oracle, bit for
bit, on every element type, mixed and degenerate meshes and a hand-built
hex next to a split cell; at full size, sampled rows plus the closed form and
symmetry."""
import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


def gpu_adjacency(mesh, b):
    dm = nn.DeviceMesh.from_host(mesh)
    res = b.build(dm, nn.WANT_ELEMS)
    assert res["status"] == 0
    return b.element_neighbors(dm, res["elems"])


def split_cell_pair():
    def node(i, j, k):
        return i + 3 * j + 6 * k
    hexc = [node(0, 0, 0), node(1, 0, 0), node(1, 1, 0), node(0, 1, 0),
            node(0, 0, 1), node(1, 0, 1), node(1, 1, 1), node(0, 1, 1)]
    cell = [node(1, 0, 0), node(2, 0, 0), node(2, 1, 0), node(1, 1, 0),
            node(1, 0, 1), node(2, 0, 1), node(2, 1, 1), node(1, 1, 1)]
    kuhn = [(0, 1, 2, 6), (0, 1, 5, 6), (0, 3, 2, 6), (0, 3, 7, 6), (0, 4, 5, 6), (0, 4, 7, 6)]
    return mg.from_elements([(mg.HEX, tuple(hexc))] + [(mg.TET, tuple(cell[q] for q in t)) for t in kuhn], 12)


def soup(seed, n_el, n_nodes):
    rng = np.random.default_rng(seed)
    el = []
    for _ in range(n_el):
        t = int(rng.integers(0, 4))
        el.append((t, tuple(int(x) for x in rng.integers(0, n_nodes, size=mg.NPE[t]))))
    return mg.from_elements(el, n_nodes)


MESHES = {
    "tri60_holes": lambda: mg.tri_grid(60, 3, holes=0.1),
    "quad40": lambda: mg.quad_grid(40, 4),
    "tet12": lambda: mg.tet_grid(12, 5),
    "hex14": lambda: mg.hex_grid(14, 6),
    "hex10_elem_perm": lambda: mg.hex_grid(10, 7, permute_elems=True),
    "mixed10": lambda: mg.mixed_grid(10, 8),
    "split_cell_pair": split_cell_pair,
    "soup_dense": lambda: soup(9, 3000, 60),        # many repeated nodes and shared faces
    "soup_sparse": lambda: soup(10, 5000, 4000),
    "fan": lambda: mg.from_elements([(mg.TRI, (0, 1 + k, 1 + (k + 1) % 500)) for k in range(500)], 501),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_adjacency_matches_oracle(name):
    mesh = MESHES[name]()
    rp, col = gpu_adjacency(mesh, nn.Builder())
    ref = oracle.element_adjacency(mesh)
    assert ref["status"] == 0
    np.testing.assert_array_equal(rp.cpu().numpy(), ref["adj"][0])
    np.testing.assert_array_equal(col.cpu().numpy(), ref["adj"][1])


def test_capacity_error_reported():
    import torch
    mesh = mg.tri_grid(20, 1)
    b = nn.Builder()
    dm = nn.DeviceMesh.from_host(mesh)
    res = b.build(dm, nn.WANT_ELEMS)
    ne_rp, ne_col = res["elems"]
    ws_bytes, cap = nn.nn_element_neighbors_query(b.h, dm.struct())
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    rp = torch.empty(mesh.n_elems + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(10, dtype=torch.int32, device="cuda")
    st = nn.nn_element_neighbors(b.h, dm.struct(), nn.NNCSR(ne_rp.data_ptr(), ne_col.data_ptr(), ne_col.numel()),
                                 nn.NNCSR(rp.data_ptr(), col.data_ptr(), 10), ws.data_ptr(), ws_bytes,
                                 b.status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert int(b.status.item()) == 3   # NN_ERR_CAPACITY
    assert nn.nn_element_neighbors(b.h, dm.struct(), nn.NNCSR(ne_rp.data_ptr(), ne_col.data_ptr(), 0),
                                   nn.NNCSR(rp.data_ptr(), col.data_ptr(), 10), ws.data_ptr(), 16,
                                   b.status.data_ptr(), 0) == 2   # workspace below the minimum


def test_full_size_tri2048():
    import torch
    mesh = mg.workload_mesh("tri2048")
    rp, col = gpu_adjacency(mesh, nn.Builder())
    m = 2047
    assert int(rp[-1].item()) == 2 * ((2 * m * 2048 + m * m) - 4 * m)    # twice the interior edges
    T = mesh.n_elems
    src = torch.repeat_interleave(torch.arange(T, device=col.device), rp[1:] - rp[:-1])
    assert not bool((src == col).any())
    a = torch.sort(src * T + col.to(torch.int64)).values
    b = torch.sort(col.to(torch.int64) * T + src).values
    assert torch.equal(a, b), "adjacency not symmetric"
    sample = np.unique(np.random.default_rng(4).integers(0, T, 2000)).astype(np.int32)
    ref = oracle.element_adjacency(mesh, sample)
    rp_h, col_h = rp.cpu().numpy(), col.cpu().numpy()
    got = np.concatenate([col_h[rp_h[e]:rp_h[e + 1]] for e in sample])
    np.testing.assert_array_equal(got, ref["adj"][1])
