"""Seeded synthetic mesh generators (host side)."""
import numpy as np
import pytest

from paper_1604_04689_gb300 import meshgen as mg


@pytest.mark.parametrize("n", [1, 2, 3, 5, 100, 4097, 65536])
def test_feistel_is_bijection(n):
    p = mg.feistel_perm(n, mg.stream_key(7, mg.STREAM_NODE_PERM))
    assert sorted(p.tolist()) == list(range(n))


def test_feistel_depends_on_key_and_is_deterministic():
    a = mg.feistel_perm(1000, 1)
    assert (a == mg.feistel_perm(1000, 1)).all()
    assert (a != mg.feistel_perm(1000, 2)).any()
    # pointwise evaluation agrees with the whole-range table
    idx = np.array([0, 17, 999], dtype=np.uint64)
    assert (mg.feistel_perm(1000, 1, idx) == a[[0, 17, 999]]).all()


def test_splitmix64_reference_values():
    # first outputs of splitmix64 seeded with 0 (state advanced by the golden gamma each call)
    assert mg.splitmix64(0) == 0xE220A8397B1DCDAF
    assert mg.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    v = mg.splitmix64(np.array([0, 0x9E3779B97F4A7C15], dtype=np.uint64))
    assert v.tolist() == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_tri64_sizes():
    m = mg.workload_mesh("tri64")
    assert m.n_nodes == 4096 and m.n_elems == 7938 and m.conn.dtype == np.int32
    assert m.conn.min() == 0 and m.conn.max() == 4095


def test_sizes_of_grid_families():
    assert mg.tet_grid(5, 1).n_elems == 6 * 4 ** 3
    assert mg.hex_grid(5, 1).n_elems == 4 ** 3 and mg.hex_grid(5, 1).n_nodes == 125
    assert mg.quad_grid(5, 1).n_elems == 16


def test_permutations_are_relabelings():
    a = mg.tet_grid(6, 3, permute_nodes=False, permute_elems=False)
    b = mg.tet_grid(6, 3)
    pi = mg.feistel_perm(a.n_nodes, mg.stream_key(3, mg.STREAM_NODE_PERM))
    pos = mg.feistel_perm(a.n_elems, mg.stream_key(3, mg.STREAM_ELEM_PERM))
    assert (b.conn.reshape(-1, 4)[pos] == pi[a.conn.reshape(-1, 4)]).all()


def test_hole_fraction():
    m = mg.tri_grid(257, 100, holes=0.05)
    full = 2 * 256 * 256
    frac = 1 - m.n_elems / full
    assert abs(frac - 0.05) < 4 * np.sqrt(0.05 * 0.95 / full)


def test_mixed_fraction_and_layout():
    m = mg.mixed_grid(33, 103)
    cells = 32 ** 3
    frac = m.meta["n_split"] / cells
    assert abs(frac - 0.30) < 4 * np.sqrt(0.3 * 0.7 / cells)
    assert m.n_elems == m.meta["n_hex"] + 6 * m.meta["n_split"]
    npe = np.where(m.elem_type == mg.HEX, 8, 4)
    assert (np.diff(m.elem_ptr) == npe).all() and m.elem_ptr[-1] == m.n_conn


def test_kuhn_tets_tile_the_cube():
    xyz = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)], float)
    vols = []
    for t in mg.KUHN_TETS:
        p = xyz[t]
        vols.append(abs(np.linalg.det(p[1:] - p[0])) / 6)
    assert np.allclose(vols, 1 / 6) and abs(sum(vols) - 1) < 1e-12


def test_request_specs_cover_range():
    specs = [mg.request_spec(i) for i in range(2000)]
    types = {t for t, _, _ in specs}
    assert types == {mg.TRI, mg.TET, mg.HEX}
    counts = []
    for t, n, _ in specs:
        m = n - 1
        counts.append({mg.TRI: 2 * m * m, mg.TET: 6 * m ** 3, mg.HEX: m ** 3}[t])
    counts = np.array(counts)
    assert counts.min() >= 500 and counts.max() <= 2.5e6
    assert 2e4 < np.median(counts) < 1e5


def test_poisson_arrivals():
    t = mg.poisson_arrivals(20000, rate=100.0)
    assert (np.diff(t) > 0).all()
    assert abs(t[-1] / 20000 - 0.01) < 0.0005
