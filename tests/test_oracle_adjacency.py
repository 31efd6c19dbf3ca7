"""Pins of the oracle's element face adjacency, each independent of its face
tables: closed-form interior-face counts of the structured grids, interior
element degrees, neighbours from cell coordinates (quad and hex grids), the
shared-vertex rule for conforming simplices, a hand-derived mixed fixture (a
hex next to a cell split into Kuhn tets), degenerate elements, a pairwise
brute force with geometrically derived faces on grids and random element
soups, and mutants of the oracle source that these pins must catch."""
import os
import subprocess
import sys
import tempfile
from itertools import combinations

import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from tests import pins
from tests.test_oracle import random_soup


_LIB = [None]   # oracle build the pins run against (a mutant's, in the mutant test)


def adj_rows(mesh, lib=None):
    r = oracle.element_adjacency(mesh, lib=lib or _LIB[0])
    assert r["status"] == 0
    rp, col = r["adj"]
    return [col[rp[e]:rp[e + 1]].tolist() for e in range(mesh.n_elems)]


# interior (shared) faces of the structured grids, m cells per side:
#   triangle grid: interior edges = (2mn + m^2) - 4m  (any diagonals)
#   quad grid: 2m(m-1);  hex grid: 3 m^2 (m-1)
#   Kuhn tets: all faces 12m^3 + 6m^2 minus 2 boundary triangles per boundary square (12 m^2)
def interior_faces(kind, n):
    m = n - 1
    return {"tri": (2 * m * n + m * m) - 4 * m, "quad": 2 * m * (m - 1),
            "tet": 12 * m ** 3 + 6 * m ** 2 - 12 * m ** 2, "hex": 3 * m * m * (m - 1)}[kind]


@pytest.mark.parametrize("kind,n", [("tri", 2), ("tri", 7), ("quad", 6), ("tet", 2), ("tet", 4), ("hex", 2), ("hex", 5)])
def test_sum_of_rows_is_twice_the_interior_faces(kind, n):
    mesh = {"tri": lambda: mg.tri_grid(n, 3), "quad": lambda: mg.quad_grid(n, 3),
            "tet": lambda: mg.tet_grid(n, 3), "hex": lambda: mg.hex_grid(n, 3)}[kind]()
    rows = adj_rows(mesh)
    assert sum(len(r) for r in rows) == 2 * interior_faces(kind, n)


def test_rows_symmetric_sorted_no_self():
    for mesh in (mg.tri_grid(6, 1, holes=0.2), mg.mixed_grid(4, 2), mg.tet_grid(3, 5)):
        rows = adj_rows(mesh)
        for e, r in enumerate(rows):
            assert r == sorted(set(r)) and e not in r
            for f in r:
                assert e in rows[f]


def test_neighbours_from_cell_coordinates():
    """Quad and hex grids with cells in natural order: face neighbours are the
    cells one step away along one axis."""
    n = 5
    m = n - 1
    rows = adj_rows(mg.quad_grid(n, 2, permute_elems=False))
    for j in range(m):
        for i in range(m):
            exp = sorted(c for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1))
                         if 0 <= i + di < m and 0 <= j + dj < m for c in [(i + di) + m * (j + dj)])
            assert rows[i + m * j] == exp
    rows = adj_rows(mg.hex_grid(n, 2, permute_elems=False))
    for k in range(m):
        for j in range(m):
            for i in range(m):
                exp = []
                for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    a, b, c = i + d[0], j + d[1], k + d[2]
                    if 0 <= a < m and 0 <= b < m and 0 <= c < m:
                        exp.append(a + m * b + m * m * c)
                assert rows[i + m * j + m * m * k] == sorted(exp)


def test_conforming_simplices_share_d_vertices():
    """In a conforming triangle (tet) mesh two elements are face neighbours
    exactly when they share 2 (3) vertices: brute force over all pairs."""
    for mesh, d in ((mg.tri_grid(6, 4), 2), (mg.tet_grid(3, 6), 3)):
        el = [set(x) for _, x in mesh.elements()]
        exp = [[] for _ in el]
        for a, b in combinations(range(len(el)), 2):
            if len(el[a] & el[b]) >= d:
                exp[a].append(b)
                exp[b].append(a)
        assert adj_rows(mesh) == [sorted(x) for x in exp]


def test_interior_degrees():
    """Elements away from the boundary: 3 (tri), 4 (quad), 4 (tet), 6 (hex) neighbours."""
    want = {mg.TRI: 3, mg.QUAD: 4, mg.TET: 4, mg.HEX: 6}
    for mesh in (mg.tri_grid(8, 5), mg.quad_grid(8, 5), mg.tet_grid(5, 5), mg.hex_grid(5, 5)):
        rows = adj_rows(mesh)
        bnd = set()
        deg_node = np.zeros(mesh.n_nodes, dtype=np.int64)
        for t, x in mesh.elements():
            for v in x:
                deg_node[v] += 1
        # boundary nodes: those in fewer elements than the interior maximum
        full = deg_node.max()
        for e, (t, x) in enumerate(mesh.elements()):
            if all(deg_node[v] == full for v in x) and mesh.etype != mg.TRI:
                assert len(rows[e]) == want[t]
        if mesh.etype == mg.TRI:   # valence varies with random diagonals: use the closed form instead
            assert sum(len(r) for r in rows) == 2 * interior_faces("tri", 8)


def test_hex_next_to_split_cell():
    """A hex and the next cell along x split into its 6 Kuhn tets (hand-derived):
    the shared square x = 1 is covered by the two tets with a triangle in it,
    (0,3,7,6) and (0,4,7,6) in the split cell's local VTK corners, so those two
    are the hex's only neighbours; every tet has its in-cell neighbours too."""
    def node(i, j, k):
        return i + 3 * j + 6 * k   # 3 x 2 x 2 nodes
    hexc = [node(0, 0, 0), node(1, 0, 0), node(1, 1, 0), node(0, 1, 0),
            node(0, 0, 1), node(1, 0, 1), node(1, 1, 1), node(0, 1, 1)]
    cell = [node(1, 0, 0), node(2, 0, 0), node(2, 1, 0), node(1, 1, 0),
            node(1, 0, 1), node(2, 0, 1), node(2, 1, 1), node(1, 1, 1)]
    kuhn = [(0, 1, 2, 6), (0, 1, 5, 6), (0, 3, 2, 6), (0, 3, 7, 6), (0, 4, 5, 6), (0, 4, 7, 6)]
    el = [(mg.HEX, tuple(hexc))] + [(mg.TET, tuple(cell[q] for q in t)) for t in kuhn]
    rows = adj_rows(mg.from_elements(el, 12))
    assert rows[0] == [1 + 3, 1 + 5]
    # inside the split cell: consecutive Kuhn tets of one axis order share a face
    for a in range(6):
        inner = sorted(b + 1 for b in range(6) if b != a and len(set(kuhn[a]) & set(kuhn[b])) == 3)
        assert [f for f in rows[a + 1] if f != 0] == inner


def test_degenerate_elements():
    """A triangle with a repeated node has one face; a collapsed tet face is no face."""
    el = [(mg.TRI, (0, 1, 2)), (mg.TRI, (1, 1, 2)), (mg.TRI, (0, 2, 3)), (mg.TRI, (3, 3, 3))]
    rows = adj_rows(mg.from_elements(el, 4))
    assert rows == [[1, 2], [0], [0], []]
    el = [(mg.TET, (0, 1, 2, 3)), (mg.TET, (0, 1, 2, 4)), (mg.TET, (0, 0, 1, 5))]
    rows = adj_rows(mg.from_elements(el, 6))
    # tet 2's faces: {0,1,5} only (the others repeat node 0); tets 0 and 1 share {0,1,2}
    assert rows == [[1], [0], []]


def test_sample_rows_equal_full_rows():
    mesh = mg.mixed_grid(5, 8)
    full = adj_rows(mesh)
    sample = np.array([0, 5, 17, 5, mesh.n_elems - 1], dtype=np.int32)
    r = oracle.element_adjacency(mesh, sample)
    rp, col = r["adj"]
    assert [col[rp[i]:rp[i + 1]].tolist() for i in range(len(sample))] == [full[e] for e in sample]


@pytest.mark.parametrize("seed", range(40))
def test_random_soup_brute_force(seed):
    """Element soups (random types, repeated and shared nodes in no grid
    pattern): the oracle equals the pairwise brute force with geometric faces."""
    mesh = random_soup(seed)
    assert adj_rows(mesh) == pins.brute_force_faces(mesh.elements())


@pytest.mark.parametrize("mesh", [mg.mixed_grid(4, 11, frac_tet=0.5), mg.tri_grid(7, 9, holes=0.2),
                                  mg.hex_grid(4, 6), mg.quad_grid(5, 3), mg.tet_grid(3, 4)],
                         ids=lambda m: m.name)
def test_grid_brute_force(mesh):
    assert adj_rows(mesh) == pins.brute_force_faces(mesh.elements())


MUTANTS = {
    # both y-faces (one hex's y = 0 face is its neighbour's y = 1 face, and the
    # test runs both ways, so one wrong face alone changes nothing)
    "hex_y_faces_wrong": ("{0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}", "{0, 1, 6, 4}, {1, 2, 6, 5}, {2, 3, 4, 6}"),
    "tet_face_missing": ("{{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}}", "{{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 3}}"),
    "one_direction_only": ("(face_in(e, f) || face_in(f, e))", "face_in(e, f)"),
    "keep_degenerate_faces": ("if ((int)face.size() < FS[t]) continue;", ""),
    "keep_self": ("if (f != e && (", "if (("),
}


def _adj_pin_failures(lib):
    failed = []
    for kind, n in (("tri", 7), ("quad", 6), ("tet", 4), ("hex", 5)):
        mesh = {"tri": lambda: mg.tri_grid(n, 3), "quad": lambda: mg.quad_grid(n, 3),
                "tet": lambda: mg.tet_grid(n, 3), "hex": lambda: mg.hex_grid(n, 3)}[kind]()
        try:
            if sum(len(r) for r in adj_rows(mesh, lib)) != 2 * interior_faces(kind, n):
                failed.append("closed:" + kind)
        except Exception:
            failed.append("closed:" + kind)
    for seed in range(20):
        mesh = random_soup(seed)
        try:
            if adj_rows(mesh, lib) != pins.brute_force_faces(mesh.elements()):
                failed.append(f"soup:{seed}")
        except Exception:
            failed.append(f"soup:{seed}")
    for name, fn in (("split", test_hex_next_to_split_cell), ("degenerate", test_degenerate_elements)):
        _LIB[0] = lib
        try:
            fn()
        except Exception:
            failed.append(name)
        finally:
            _LIB[0] = None
    return failed


def test_pins_catch_adjacency_mutants():
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp")).read()
    assert _adj_pin_failures(None) == []
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as td:
        for name, (a, b) in MUTANTS.items():
            assert a in src, name
            path = os.path.join(td, name + ".cpp")
            with open(path, "w") as f:
                f.write(src.replace(a, b, 1))
            so = os.path.join(td, name + ".so")
            subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", path, "-o", so])
            code = ("import sys, oracle; from tests.test_oracle_adjacency import _adj_pin_failures; "
                    f"sys.exit(0 if not _adj_pin_failures(oracle.load_library({so!r})) else 3)")
            try:   # a mutant that crashes or never ends counts as caught
                rc = subprocess.run([sys.executable, "-c", code], cwd=root, stdout=subprocess.DEVNULL,
                                    stderr=subprocess.DEVNULL, timeout=20).returncode
            except subprocess.TimeoutExpired:
                rc = "hung"
            assert rc != 0, f"mutant {name} survived the pins"
