"""Pins of the CPU oracle (no GPU): golden fixtures, brute force, the paper's
sort recipe restated with numpy, closed forms, invariants, metamorphic checks
and mutants of the oracle source that the pins must catch."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "small_meshes.json")


def load_golden():
    with open(GOLDEN) as f:
        return json.load(f)


def golden_mesh(fx):
    ep = np.array(fx["elem_ptr"], dtype=np.int64) if "elem_ptr" in fx else None
    et = np.array(fx["elem_type"], dtype=np.uint8) if "elem_type" in fx else None
    return mg.Mesh(fx["type"], fx["n_nodes"], np.array(fx["conn"], dtype=np.int32), ep, et, fx["name"])


def small_meshes():
    """Tiny meshes of every kind, including holes, mixed types and permutations."""
    out = [
        mg.tri_grid(5, 7), mg.tri_grid(6, 8, diag=0), mg.tri_grid(7, 9, holes=0.2),
        mg.quad_grid(5, 3), mg.tet_grid(3, 4), mg.tet_grid(4, 5, permute_nodes=False),
        mg.hex_grid(4, 6), mg.hex_grid(3, 2, permute_elems=True), mg.mixed_grid(4, 11, frac_tet=0.5),
        mg.tri_grid(2, 1), mg.tri_grid(1, 1),
    ]
    # a fan of 40 triangles (one high-valence node) plus an isolated node
    fan = [(mg.TRI, (0, 1 + k, 1 + (k + 1) % 40)) for k in range(40)]
    out.append(mg.from_elements(fan, 42, "fan40"))
    return out


# ------------------------------------------------------------------ golden

@pytest.mark.parametrize("fx", load_golden(), ids=lambda f: f["name"])
def test_golden(fx):
    r = oracle.neighbors(golden_mesh(fx))
    assert r["status"] == fx["status"]
    if fx["status"] == 0:
        assert pins.rows_of(*r["nodes"]) == fx["nodes"]
        assert pins.rows_of(*r["elems"]) == fx["elems"]


@pytest.mark.parametrize("fx", [f for f in load_golden() if f["status"] == 0], ids=lambda f: f["name"])
def test_golden_agrees_with_brute_force(fx):
    """The hand-derived fixtures and the geometric brute force agree."""
    m = golden_mesh(fx)
    bn, be = pins.brute_force(m.elements(), m.n_nodes)
    assert bn == fx["nodes"] and be == fx["elems"]


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("mesh", small_meshes(), ids=lambda m: m.name)
def test_brute_force(mesh):
    r = oracle.neighbors(mesh)
    assert r["status"] == 0
    bn, be = pins.brute_force(mesh.elements(), mesh.n_nodes)
    assert pins.rows_of(*r["nodes"]) == bn
    assert pins.rows_of(*r["elems"]) == be


@pytest.mark.parametrize("mesh", small_meshes() + [mg.tri_grid(40, 3, holes=0.05), mg.tet_grid(9, 1),
                                                   mg.mixed_grid(9, 13)], ids=lambda m: m.name)
def test_sort_restatement(mesh):
    """The paper's pair-sort recipe (numpy) gives the same CSR arrays."""
    r = oracle.neighbors(mesh)
    (nrp, ncol), (erp, ecol) = pins.sort_restatement(mesh.elements(), mesh.n_nodes)
    np.testing.assert_array_equal(r["nodes"][0], nrp)
    np.testing.assert_array_equal(r["nodes"][1], ncol)
    np.testing.assert_array_equal(r["elems"][0], erp)
    np.testing.assert_array_equal(r["elems"][1], ecol)


def random_soup(seed):
    """Arbitrary connectivity: random element types, node ids drawn from a
    small range so that elements repeat nodes (degenerate edges), share
    nodes in no grid pattern, and leave some nodes untouched."""
    rng = np.random.default_rng(seed)
    n_nodes = int(rng.integers(1, 40))
    elems = []
    for _ in range(int(rng.integers(0, 30))):
        t = int(rng.choice([mg.TRI, mg.QUAD, mg.TET, mg.HEX]))
        elems.append((t, tuple(int(x) for x in rng.integers(0, n_nodes, mg.NPE[t]))))
    if seed % 3 == 0 and elems:            # uniform type: the same element list, one type
        t = elems[0][0]
        elems = [(t, tuple(int(x) for x in rng.integers(0, n_nodes, mg.NPE[t]))) for _ in elems]
    return mg.from_elements(elems, n_nodes, f"soup{seed}") if elems else \
        mg.Mesh(mg.TRI, n_nodes, np.zeros(0, np.int32), name=f"soup{seed}")


@pytest.mark.parametrize("seed", range(40))
def test_random_soup_brute_force_and_sort(seed):
    """Element soups with repeated and isolated nodes: the oracle equals the
    geometric brute force and the paper's pair-sort recipe."""
    mesh = random_soup(seed)
    r = oracle.neighbors(mesh)
    assert r["status"] == 0
    bn, be = pins.brute_force(mesh.elements(), mesh.n_nodes)
    assert pins.rows_of(*r["nodes"]) == bn
    assert pins.rows_of(*r["elems"]) == be
    (nrp, ncol), (erp, ecol) = pins.sort_restatement(mesh.elements(), mesh.n_nodes)
    np.testing.assert_array_equal(r["nodes"][0], nrp)
    np.testing.assert_array_equal(r["nodes"][1], ncol)
    np.testing.assert_array_equal(r["elems"][0], erp)
    np.testing.assert_array_equal(r["elems"][1], ecol)


# ----------------------------------------------------------- closed forms

def _coords2(n):
    i = np.arange(n * n) % n
    j = np.arange(n * n) // n
    return i, j


@pytest.mark.parametrize("n", [2, 3, 17, 64])
def test_tri_grid_closed_forms(n):
    m = n - 1
    mesh = mg.tri_grid(n, 5)
    r = oracle.neighbors(mesh)
    rp, col = r["nodes"]
    assert rp[-1] == 2 * pins.tri_grid_edges(m)
    assert r["elems"][0][-1] == 3 * mesh.n_elems == 6 * m * m
    # Euler characteristic of a triangulated disk
    assert n * n - rp[-1] // 2 + 2 * m * m == 1


def test_tri_grid_fixed_diagonal_interior_valence():
    n = 12
    mesh = mg.tri_grid(n, 0, diag=0, permute_nodes=False, permute_elems=False)
    r = oracle.neighbors(mesh)
    deg = np.diff(r["nodes"][0])
    edeg = np.diff(r["elems"][0])
    i, j = _coords2(n)
    interior = (i > 0) & (i < n - 1) & (j > 0) & (j < n - 1)
    assert (deg[interior] == 6).all() and (edeg[interior] == 6).all()
    # corners (0,0) and (n-1,n-1) touch the diagonal; the other two do not
    assert deg[0] == 3 and deg[n * n - 1] == 3 and deg[n - 1] == 2 and deg[n * (n - 1)] == 2


def test_tri_grid_random_diagonal_valence():
    """interior degree = element count = 4 + number of diagonals at the node."""
    n = 30
    m = n - 1
    seed = 17
    mesh = mg.tri_grid(n, seed, permute_nodes=False, permute_elems=False)
    q = np.arange(m * m, dtype=np.uint64)
    bit = (mg.hash_u64(mg.stream_key(seed, mg.STREAM_DIAG), q) & np.uint64(1)).astype(int).reshape(m, m)  # [j, i]
    r = oracle.neighbors(mesh)
    deg = np.diff(r["nodes"][0])
    edeg = np.diff(r["elems"][0])
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            # quads around (i,j): (i,j) corner a, (i-1,j) corner b, (i-1,j-1) corner c, (i,j-1) corner d
            d = int(bit[j, i] == 0) + int(bit[j, i - 1] == 1) + int(bit[j - 1, i - 1] == 0) + int(bit[j - 1, i] == 1)
            v = i + n * j
            assert deg[v] == 4 + d and edeg[v] == 4 + d


@pytest.mark.parametrize("n", [2, 5, 20])
def test_quad_grid_closed_forms(n):
    m = n - 1
    mesh = mg.quad_grid(n, 2, permute_nodes=False)
    r = oracle.neighbors(mesh)
    rp = r["nodes"][0]
    assert rp[-1] == 2 * pins.quad_grid_edges(m)
    i, j = _coords2(n)
    interior = (i > 0) & (i < n - 1) & (j > 0) & (j < n - 1)
    assert (np.diff(rp)[interior] == 4).all() and (np.diff(r["elems"][0])[interior] == 4).all()


def _coords3(n):
    v = np.arange(n ** 3)
    return v % n, (v // n) % n, v // (n * n)


@pytest.mark.parametrize("n", [2, 3, 6, 11])
def test_kuhn_grid_closed_forms(n):
    m = n - 1
    mesh = mg.tet_grid(n, 3)
    r = oracle.neighbors(mesh)
    E = r["nodes"][0][-1] // 2
    assert E == pins.kuhn_grid_edges(m)
    assert r["elems"][0][-1] == 4 * 6 * m ** 3
    assert n ** 3 - E + pins.kuhn_grid_faces(m) - 6 * m ** 3 == 1       # Euler of a ball


def test_kuhn_grid_interior_neighbourhood():
    n = 6
    mesh = mg.tet_grid(n, 3, permute_nodes=False, permute_elems=False)
    r = oracle.neighbors(mesh)
    rp, col = r["nodes"]
    x, y, z = _coords3(n)
    for v in range(n ** 3):
        if 0 < x[v] < n - 1 and 0 < y[v] < n - 1 and 0 < z[v] < n - 1:
            nb = col[rp[v]:rp[v + 1]]
            offs = sorted((int(x[u] - x[v]), int(y[u] - y[v]), int(z[u] - z[v])) for u in nb)
            assert offs == pins.KUHN_OFFSETS
            assert r["elems"][0][v + 1] - r["elems"][0][v] == 24


@pytest.mark.parametrize("n", [2, 3, 7])
def test_hex_grid_closed_forms(n):
    m = n - 1
    mesh = mg.hex_grid(n, 9, permute_nodes=False)
    r = oracle.neighbors(mesh)
    rp, col = r["nodes"]
    E = rp[-1] // 2
    assert E == pins.hex_grid_edges(m)
    assert n ** 3 - E + pins.hex_grid_faces(m) - m ** 3 == 1
    x, y, z = _coords3(n)
    for v in range(n ** 3):
        if 0 < x[v] < n - 1 and 0 < y[v] < n - 1 and 0 < z[v] < n - 1:
            nb = col[rp[v]:rp[v + 1]]
            offs = sorted((int(x[u] - x[v]), int(y[u] - y[v]), int(z[u] - z[v])) for u in nb)
            assert offs == pins.HEX_OFFSETS
            assert r["elems"][0][v + 1] - r["elems"][0][v] == 8


# -------------------------------------------------------------- invariants

def _check_invariants(mesh, r):
    rp, col = r["nodes"]
    erp, ecol = r["elems"]
    # rows sorted strictly ascending (sets), ids in range, no self loops
    for a, b, c, hi in ((rp[:-1], rp[1:], col, mesh.n_nodes), (erp[:-1], erp[1:], ecol, mesh.n_elems)):
        if c.size:
            inner = np.ones(c.size, dtype=bool)
            inner[b[b < c.size]] = False           # first entry of each next row
            d = np.diff(c.astype(np.int64))
            assert (d[inner[1:]] > 0).all()
            assert c.min() >= 0 and c.max() < hi
    src = np.repeat(np.arange(mesh.n_nodes), np.diff(rp))
    assert not (src == col).any()
    # symmetry: u in N(v) <=> v in N(u)
    fwd = src.astype(np.int64) * mesh.n_nodes + col
    bwd = col.astype(np.int64) * mesh.n_nodes + src
    np.testing.assert_array_equal(np.sort(fwd), np.sort(bwd))
    # sum of node rows = twice the unique edge count (hash set of (min,max))
    assert rp[-1] == 2 * len(pins.unique_edges(mesh.elements()))


@pytest.mark.parametrize("mesh", [mg.tri_grid(25, 4, holes=0.15), mg.mixed_grid(6, 5), mg.hex_grid(5, 1),
                                  mg.tet_grid(5, 8)], ids=lambda m: m.name)
def test_invariants(mesh):
    r = oracle.neighbors(mesh)
    _check_invariants(mesh, r)
    if mesh.etype == mg.MIXED:
        assert r["elems"][0][-1] == mesh.n_conn      # no repeated nodes: sum of npe


def test_triangle_identity_with_holes():
    """deg(v) = tris(v) + b(v)/2, b = incident edges with one triangle (<= 2 per edge)."""
    mesh = mg.tri_grid(48, 100, holes=0.05)
    r = oracle.neighbors(mesh)
    deg = np.diff(r["nodes"][0])
    tris = np.diff(r["elems"][0])
    uk, cnt, base = pins.tri_edge_triangle_counts(mesh.conn)
    assert cnt.max() <= 2
    bound = uk[cnt == 1]
    b = np.bincount(np.concatenate([bound // base, bound % base]), minlength=mesh.n_nodes)
    assert ((2 * tris + b) % 2 == 0).all()
    np.testing.assert_array_equal(deg, tris + b // 2)
    assert (deg == 0).sum() > 0 or True       # holes may isolate nodes: empty rows allowed


# ------------------------------------------------------------- metamorphic

def test_node_relabel_and_element_reorder():
    base = mg.tet_grid(5, 2)
    r0 = oracle.neighbors(base)
    rng = np.random.default_rng(0)
    sigma = rng.permutation(base.n_nodes)
    tau = rng.permutation(base.n_elems)
    c = sigma[base.conn.reshape(-1, 4)]
    c2 = np.empty_like(c)
    c2[tau] = c
    m2 = mg.Mesh(mg.TET, base.n_nodes, c2.ravel().astype(np.int32))
    r2 = oracle.neighbors(m2)
    n0 = pins.rows_of(*r0["nodes"])
    n2 = pins.rows_of(*r2["nodes"])
    e0 = pins.rows_of(*r0["elems"])
    e2 = pins.rows_of(*r2["elems"])
    for v in range(base.n_nodes):
        assert n2[sigma[v]] == sorted(sigma[u] for u in n0[v])
        assert e2[sigma[v]] == sorted(tau[e] for e in e0[v])


def test_local_rotations_do_not_change_output():
    tri = mg.tri_grid(9, 4)
    t = tri.conn.reshape(-1, 3)
    tri2 = mg.Mesh(mg.TRI, tri.n_nodes, t[:, [1, 2, 0]].ravel().copy())
    tri3 = mg.Mesh(mg.TRI, tri.n_nodes, t[:, [2, 1, 0]].ravel().copy())        # orientation flip
    tet = mg.tet_grid(4, 4)
    tt = tet.conn.reshape(-1, 4)
    tet2 = mg.Mesh(mg.TET, tet.n_nodes, tt[:, [2, 0, 3, 1]].ravel().copy())
    hx = mg.hex_grid(4, 4)
    h = hx.conn.reshape(-1, 8)
    # rotate the cube a quarter turn about z, and swap bottom/top (both keep VTK edges)
    hx2 = mg.Mesh(mg.HEX, hx.n_nodes, h[:, [1, 2, 3, 0, 5, 6, 7, 4]].ravel().copy())
    hx3 = mg.Mesh(mg.HEX, hx.n_nodes, h[:, [4, 5, 6, 7, 0, 1, 2, 3]].ravel().copy())
    for a, b in ((tri, tri2), (tri, tri3), (tet, tet2), (hx, hx2), (hx, hx3)):
        ra, rb = oracle.neighbors(a), oracle.neighbors(b)
        for k in ("nodes", "elems"):
            np.testing.assert_array_equal(ra[k][0], rb[k][0])
            np.testing.assert_array_equal(ra[k][1], rb[k][1])


def test_disjoint_union_equals_parts():
    a, b = mg.tri_grid(6, 1), mg.hex_grid(4, 2)
    c = mg.from_elements(a.elements() + [(t, tuple(x + a.n_nodes for x in nd)) for t, nd in b.elements()],
                         a.n_nodes + b.n_nodes)
    ra, rb, rc = oracle.neighbors(a), oracle.neighbors(b), oracle.neighbors(c)
    na, nb, nc = (pins.rows_of(*r["nodes"]) for r in (ra, rb, rc))
    ea, eb, ec = (pins.rows_of(*r["elems"]) for r in (ra, rb, rc))
    assert nc == na + [[u + a.n_nodes for u in row] for row in nb]
    assert ec == ea + [[e + a.n_elems for e in row] for row in eb]


# ------------------------------------------------------------ sampled rows

@pytest.mark.parametrize("mesh", [mg.tri_grid(20, 3, holes=0.1), mg.mixed_grid(5, 3)], ids=lambda m: m.name)
def test_rows_matches_full_build(mesh):
    full = oracle.neighbors(mesh)
    sample = np.array([0, 5, 5, mesh.n_nodes - 1, 17, 3], dtype=np.int32)
    part = oracle.rows(mesh, sample)
    for k in ("nodes", "elems"):
        fr = pins.rows_of(*full[k])
        pr = pins.rows_of(*part[k])
        assert pr == [fr[v] for v in sample]


# ------------------------------------------------------------------ errors

def test_error_status_codes():
    m = mg.tri_grid(6, 2)
    bad = m.conn.copy()
    bad[7] = m.n_nodes
    assert oracle.neighbors(mg.Mesh(mg.TRI, m.n_nodes, bad))["status"] == 4
    bad[7] = -1
    assert oracle.neighbors(mg.Mesh(mg.TRI, m.n_nodes, bad))["status"] == 4
    mx = mg.mixed_grid(4, 1)
    ep = mx.elem_ptr.copy()
    ep[3] += 1
    assert oracle.neighbors(mg.Mesh(mg.MIXED, mx.n_nodes, mx.conn, ep, mx.elem_type))["status"] == 5
    et = mx.elem_type.copy()
    et[2] = 9
    assert oracle.neighbors(mg.Mesh(mg.MIXED, mx.n_nodes, mx.conn, mx.elem_ptr, et))["status"] == 5


def test_empty_meshes():
    r = oracle.neighbors(mg.Mesh(mg.TRI, 5, np.zeros(0, dtype=np.int32)))
    assert r["status"] == 0
    assert r["nodes"][0].tolist() == [0] * 6 and r["elems"][0].tolist() == [0] * 6
    r = oracle.neighbors(mg.Mesh(mg.HEX, 0, np.zeros(0, dtype=np.int32)))
    assert r["nodes"][0].tolist() == [0] and r["nodes"][1].size == 0


# ------------------------------------------------------------------ mutants

MUTANTS = {
    "drop_reverse_direction": ("nn[b].insert(a);", ""),
    "hex_edge_wrong_corner": ("{0, 4}, {1, 5}", "{0, 5}, {1, 5}"),
    "tet_edge_missing": ("{1, 3}, {2, 3}}}", "{1, 3}, {1, 3}}}"),
    "quad_diagonal": ("{2, 3}, {3, 0}}}", "{2, 3}, {3, 1}}}"),
    "keep_self_pairs": ("if (a == b) continue;\n                nn[a]", "nn[a]"),
    "range_off_by_one": ("nodes[i] >= m.n_nodes", "nodes[i] > m.n_nodes"),
    "elem_id_shift": ("ne[nodes[i]].insert((int32_t)e);", "ne[nodes[i]].insert((int32_t)e + 1);"),
}


def _pin_failures(lib):
    """Run a compact set of pins against an oracle build; return the names that fail."""
    failed = []
    for fx in load_golden():
        try:
            r = oracle.neighbors(golden_mesh(fx), lib=lib)
            ok = r["status"] == fx["status"] and (fx["status"] != 0 or (
                pins.rows_of(*r["nodes"]) == fx["nodes"] and pins.rows_of(*r["elems"]) == fx["elems"]))
        except Exception:
            ok = False
        if not ok:
            failed.append("golden:" + fx["name"])
    for mesh in (mg.tri_grid(5, 7), mg.tet_grid(3, 4), mg.hex_grid(3, 6), mg.quad_grid(4, 3)):
        r = oracle.neighbors(mesh, lib=lib)
        bn, be = pins.brute_force(mesh.elements(), mesh.n_nodes)
        if pins.rows_of(*r["nodes"]) != bn or pins.rows_of(*r["elems"]) != be:
            failed.append("brute:" + mesh.name)
    return failed


def test_pins_catch_oracle_mutants():
    """Each planted mistake in a copy of the oracle source fails at least one pin.

    Mutants run in a child process each, so one that crashes or hangs counts
    as caught without taking the test run down.  A mutant that indexes out of
    bounds writes past a vector of sets: depending on the memory layout it
    faults, or corrupts a set so that a later walk never ends; the child is
    then stopped after a time limit far above the real oracle's run time."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp")).read()
    assert _pin_failures(None) == []
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as td:
        for name, (a, b) in MUTANTS.items():
            assert a in src, name
            path = os.path.join(td, name + ".cpp")
            with open(path, "w") as f:
                f.write(src.replace(a, b, 1))
            so = os.path.join(td, name + ".so")
            subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", path, "-o", so])
            code = ("import sys, oracle; from tests.test_oracle import _pin_failures; "
                    f"sys.exit(0 if not _pin_failures(oracle.load_library({so!r})) else 3)")
            try:
                rc = subprocess.run([sys.executable, "-c", code], cwd=root, stdout=subprocess.DEVNULL,
                                    stderr=subprocess.DEVNULL, timeout=20).returncode
            except subprocess.TimeoutExpired:   # run() has killed the child
                rc = "hung"
            assert rc != 0, f"mutant {name} survived the pins"


def test_non_manifold_book_and_bowtie():
    """Hand-derived rows (Sec. 2.1.1 / 2.1.2 read as sets) for inputs a grid
    never has.  Book: three triangles on one edge 0-1, pages 2, 3, 4.
    Bowtie: two triangles meeting only at node 2."""
    book = mg.from_elements([(mg.TRI, (0, 1, 2)), (mg.TRI, (1, 0, 3)), (mg.TRI, (0, 4, 1))], 5, "book")
    r = oracle.neighbors(book)
    assert pins.rows_of(*r["nodes"]) == [[1, 2, 3, 4], [0, 2, 3, 4], [0, 1], [0, 1], [0, 1]]
    assert pins.rows_of(*r["elems"]) == [[0, 1, 2], [0, 1, 2], [0], [1], [2]]
    bowtie = mg.from_elements([(mg.TRI, (0, 1, 2)), (mg.TRI, (2, 3, 4))], 5, "bowtie")
    r = oracle.neighbors(bowtie)
    assert pins.rows_of(*r["nodes"]) == [[1, 2], [0, 2], [0, 1, 3, 4], [2, 4], [2, 3]]
    assert pins.rows_of(*r["elems"]) == [[0], [0], [0, 1], [1], [1]]
