"""Host logic of the chunked build (no GPU): node slabs, the greedy chunk
plan and its error codes, on an offline handle sized like a GB300.  The
mesh's pointers are never dereferenced on the host, so a fake aligned
address stands in for device memory here."""
import numpy as np
import pytest

from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn

FAKE = 1 << 20  # 16-byte aligned, never read


@pytest.fixture(scope="module")
def h():
    from paper_1604_04689_gb300 import build
    build.build()
    handle = nn.nn_create_offline()
    yield handle
    nn.nn_destroy(handle)


def struct(m):
    return nn.NNMesh(int(m.etype), m.n_nodes, m.n_elems, int(m.conn.size), FAKE if m.conn.size else None,
                     FAKE if m.elem_ptr is not None else None, FAKE if m.elem_type is not None else None)


def slab_counts(m, shift, ns):
    """Incidences per slab of 2^shift node ids: every connectivity entry of
    a valid mesh is one incidence."""
    return np.bincount(m.conn.astype(np.int64) >> shift, minlength=ns).astype(np.int64)


@pytest.mark.parametrize("n,shift,ns", [(0, 0, 0), (1, 0, 1), (4096, 0, 4096), (4097, 1, 2049),
                                        (1 << 22, 10, 4096), ((1 << 22) + 1, 11, 2049)])
def test_slabs(n, shift, ns):
    m = nn.NNMesh(nn.TRI, n, 0, 0, None, None, None)
    assert nn.nn_chunk_slabs(m) == (shift, ns)


MESHES = {
    "tri300": lambda: mg.tri_grid(300, 3),
    "tet40": lambda: mg.tet_grid(40, 2),
    "hex33": lambda: mg.hex_grid(33, 4),
    "mixed21": lambda: mg.mixed_grid(21, 5),
}


def plan(h, m, want, ws):
    s = struct(m)
    shift, ns = nn.nn_chunk_slabs(s)
    counts = slab_counts(m, shift, ns)
    st, chunks, need = nn.nn_chunk_plan(h, s, want, counts, ws)
    return st, chunks, need, counts, shift


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("want", [nn.WANT_NODES, nn.WANT_ELEMS, nn.WANT_BOTH])
def test_plan_tiles_and_fits(h, name, want):
    m = MESHES[name]()
    s = struct(m)
    whole, _, _ = nn.nn_query(h, s, want)
    st, chunks, need, counts, shift = plan(h, m, want, 1 << 40)
    assert st == 0 and len(chunks) == 1
    assert chunks[0] == (0, m.n_nodes, m.conn.size)
    # the whole-mesh workspace (plus the running offsets) holds the whole mesh as one chunk
    st, chunks, _, _, _ = plan(h, m, want, whole + 256)
    assert st == 0 and chunks == [(0, m.n_nodes, m.conn.size)]
    # a quarter of it: several chunks, each fitting, each maximal
    for ws in (max(need, whole // 4), need):
        st, chunks, _, counts, shift = plan(h, m, want, ws)
        assert st == 0 and len(chunks) > 1
        assert chunks[0][0] == 0 and chunks[-1][1] == m.n_nodes
        for a, b in zip(chunks, chunks[1:]):
            assert a[1] == b[0]
        for lo, hi, rec in chunks:
            assert hi > lo and lo % (1 << shift) == 0
            assert rec == int(counts[lo >> shift: (hi + (1 << shift) - 1) >> shift].sum())
            assert nn.nn_chunk_query(h, s, want, (lo, hi, rec)) <= ws
            if hi < m.n_nodes:           # greedy: one more slab would not fit
                nxt = min(m.n_nodes, hi + (1 << shift))
                grown = (lo, nxt, rec + int(counts[hi >> shift]))
                assert nn.nn_chunk_query(h, s, want, grown) > ws
        assert sum(c[2] for c in chunks) == m.conn.size


def test_plan_errors(h):
    m = MESHES["tri300"]()
    s = struct(m)
    shift, ns = nn.nn_chunk_slabs(s)
    counts = slab_counts(m, shift, ns)
    st, chunks, need = nn.nn_chunk_plan(h, s, nn.WANT_BOTH, counts, 1 << 40)
    assert st == 0
    st, chunks, need2 = nn.nn_chunk_plan(h, s, nn.WANT_BOTH, counts, need - 1)
    assert st == 2 and chunks == [] and need2 == need             # below the largest single slab
    st, chunks, _ = nn.nn_chunk_plan(h, s, nn.WANT_BOTH, counts, need, max_chunks=2)
    assert st == 3 and len(chunks) == 2                           # more chunks than room for
    bad = counts.copy()
    bad[0] += m.conn.size
    st, _, _ = nn.nn_chunk_plan(h, s, nn.WANT_BOTH, bad, 1 << 40)
    assert st == 1                                                # not this mesh's counts
    with pytest.raises(nn.NNError):
        nn.nn_chunk_query(h, s, nn.WANT_BOTH, (5, 5, 0))           # empty chunk
    with pytest.raises(nn.NNError):
        nn.nn_chunk_query(h, s, nn.WANT_BOTH, (0, m.n_nodes + 1, 0))  # past the last node


def test_smaller_workspace_more_chunks(h):
    m = MESHES["tet40"]()
    s = struct(m)
    whole, _, _ = nn.nn_query(h, s, nn.WANT_BOTH)
    need = plan(h, m, nn.WANT_BOTH, 1 << 40)[2]
    # every chunk also keeps nn_query's fixed 16 MiB spill reserve, so the
    # smallest workspace that plans is a little above 16 MiB
    assert 16 << 20 < need < whole
    sizes = [len(plan(h, m, nn.WANT_BOTH, int(need + f * (whole - need)))[1]) for f in (1.0, 0.5, 0.25, 0.0)]
    assert sizes == sorted(sizes) and sizes[1] >= 2


def test_offline_handle_refuses_compute(h):
    m = MESHES["tri300"]()
    s = struct(m)
    csr = nn.NNCSR(FAKE, FAKE, 10)
    assert nn.nn_neighbors_both(h, s, csr, csr, FAKE, 1 << 30, FAKE, 0) == 1
    assert nn.nn_chunk_count(h, s, FAKE, FAKE, 0) == 1
    assert nn.nn_neighbors_chunked(h, s, nn.WANT_BOTH, [(0, m.n_nodes, m.conn.size)], csr, csr, FAKE, 1 << 30,
                                   FAKE, 0) == 1
    with pytest.raises(nn.NNError):
        nn.nn_create_offline(0, 1 << 17, 1 << 17)


def random_counts(seed, ns):
    """Slab-count profiles a grid never gives: empty slabs, one hub slab
    holding a large share, heavy tails."""
    rng = np.random.default_rng(seed)
    kind = seed % 3
    if kind == 0:
        c = rng.integers(0, 5000, ns)
        c[rng.random(ns) < 0.3] = 0
    elif kind == 1:
        c = rng.integers(0, 200, ns)
        c[int(rng.integers(ns))] = 400_000
    else:
        c = (rng.pareto(1.2, ns) * 300).astype(np.int64)
    return c.astype(np.int64)


@pytest.mark.parametrize("seed", range(12))
def test_plan_on_random_slab_profiles(h, seed):
    N = int(np.random.default_rng(100 + seed).integers(5_000, 3_000_000))
    probe = nn.NNMesh(nn.TRI, N, 0, 0, None, None, None)
    shift, ns = nn.nn_chunk_slabs(probe)
    counts = random_counts(seed, ns)
    total = int(counts.sum())
    T = (total + 2) // 3
    s = nn.NNMesh(nn.TRI, N, T, 3 * T, FAKE if T else None, None, None)
    st, one, need = nn.nn_chunk_plan(h, s, nn.WANT_BOTH, counts, 1 << 42)
    assert st == 0 and one == [(0, N, total)]
    assert nn.nn_chunk_plan(h, s, nn.WANT_BOTH, counts, need - 1)[0] == 2     # below the largest slab
    prev = None
    for ws in (need, need + (need >> 1), 2 * need, 4 * need):
        st, chunks, _ = nn.nn_chunk_plan(h, s, nn.WANT_BOTH, counts, ws)
        assert st == 0
        assert chunks[0][0] == 0 and chunks[-1][1] == N
        assert all(a[1] == b[0] for a, b in zip(chunks, chunks[1:]))
        for lo, hi, rec in chunks:
            assert lo % (1 << shift) == 0
            assert rec == int(counts[lo >> shift: (hi + (1 << shift) - 1) >> shift].sum())
            assert nn.nn_chunk_query(h, s, nn.WANT_BOTH, (lo, hi, rec)) <= ws
            if hi < N:
                grown = (lo, min(N, hi + (1 << shift)), rec + int(counts[hi >> shift]))
                assert nn.nn_chunk_query(h, s, nn.WANT_BOTH, grown) > ws
        assert prev is None or len(chunks) <= prev
        prev = len(chunks)
