"""Host logic of the serving loop (no GPU): request stream and admission."""
from collections import deque

from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300.serve import Admission, LaneCaps, Request, make_requests


def test_request_sizes_match_the_generator():
    for t, n in ((mg.TRI, 5), (mg.TET, 4), (mg.HEX, 6), (mg.QUAD, 3)):
        r = Request(0, t, n, 1, 0.0)
        m = {mg.TRI: mg.tri_grid, mg.TET: mg.tet_grid, mg.HEX: mg.hex_grid, mg.QUAD: mg.quad_grid}[t](n, 1)
        assert (r.n_nodes, r.n_elems, r.n_conn) == (m.n_nodes, m.n_elems, m.n_conn)


def test_request_stream_is_seeded():
    a, b = make_requests(50, 100.0), make_requests(50, 100.0)
    assert [(r.etype, r.n, r.seed, r.arrival) for r in a] == [(r.etype, r.n, r.seed, r.arrival) for r in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))
    assert all(1e3 * 0.5 <= r.n_elems <= 2e6 * 1.3 for r in a)


def test_admission_fifo_caps_and_budget():
    caps = LaneCaps(max_meshes=3, max_elems=10**9, max_nodes=10**9, max_conn=10**9)
    reqs = [Request(i, mg.TRI, 10 + i, i, 0.0) for i in range(6)]
    q = deque(reqs)
    adm = Admission(caps)
    b = adm.form(q, 1 << 40)
    assert [r.rid for r in b] == [0, 1, 2] and len(q) == 3           # slot limit, arrival order
    budget = reqs[3].device_bytes() + reqs[4].device_bytes() + 1
    b = adm.form(q, budget)
    assert [r.rid for r in b] == [3, 4] and [r.rid for r in q] == [5]  # memory budget
    assert adm.form(q, 0) == [] and len(q) == 1                        # nothing fits: nothing taken


def test_admission_stops_at_first_misfit_and_rejects_oversize():
    caps = LaneCaps(max_meshes=100, max_elems=3000, max_nodes=10**9, max_conn=10**9)
    small, big = Request(0, mg.TRI, 20, 1, 0.0), Request(1, mg.TRI, 60, 1, 0.0)   # 722 and 6962 tris
    adm = Admission(caps)
    assert adm.fits_alone(small) and not adm.fits_alone(big)
    mid = Request(2, mg.TRI, 30, 1, 0.0)                                            # 1682 tris
    q = deque([small, mid, Request(3, mg.TRI, 20, 2, 0.0), small])
    b = adm.form(q, 1 << 40)
    assert [r.rid for r in b] == [0, 2] and [r.rid for r in q] == [3, 0]              # 722+1682+722 > 3000


def test_request_bytes_cover_the_library_bounds():
    """What admission counts per request is the connectivity plus both CSRs at
    the library's own capacity bounds (nn_query on an offline handle), so a
    batch admitted under the budget can always hold its results."""
    from paper_1604_04689_gb300 import build, nn
    build.build()
    h = nn.nn_create_offline()
    try:
        for t, n in ((mg.TRI, 40), (mg.QUAD, 17), (mg.TET, 9), (mg.HEX, 11)):
            r = Request(0, t, n, 1, 0.0)
            s = nn.NNMesh(t, r.n_nodes, r.n_elems, r.n_conn, 1 << 20, None, None)
            _, node_cap, elem_cap = nn.nn_query(h, s, nn.WANT_BOTH)
            assert r.device_bytes() == 4 * r.n_conn + 2 * 8 * (r.n_nodes + 1) + 4 * (node_cap + elem_cap)
    finally:
        nn.nn_destroy(h)


def test_capacity_classes_pick_the_smallest_that_holds_the_batch():
    from paper_1604_04689_gb300.serve import SMALL_CAPS, LaneCaps, Request
    full = LaneCaps()
    assert SMALL_CAPS.holds_caps(full) and not full.holds_caps(full)
    assert not SMALL_CAPS.holds_caps(LaneCaps(max_meshes=8))  # a lane smaller in any capacity gets no small class
    small = [Request(i, 0, 100, i, 0.0) for i in range(3)]        # 3 triangle grids of 19,602 triangles
    assert SMALL_CAPS.holds(small) and full.holds(small)
    big = [Request(0, 3, 121, 0, 0.0)]                            # a hex grid of 1,728,000 hexes: 13.8 M entries
    assert not SMALL_CAPS.holds(big) and full.holds(big)
    many = [Request(i, 0, 10, i, 0.0) for i in range(SMALL_CAPS.max_meshes + 1)]
    assert not SMALL_CAPS.holds(many) and full.holds(many)
