"""Independent checks ("pins") of the CPU oracle, written from the definitions.

Nothing here calls the oracle's C++ code or the CUDA library: these are
separate restatements used to pin the oracle down.

* ``brute_force``: O(N^2 T) test of every node pair against every element
  (Sec. 2.1.1: u and v are neighbors iff some element has an edge {u, v};
  Sec. 2.1.2: e is a neighbor element of v iff v is a node of e).  Element
  edges are derived geometrically, not from a table: every node pair of a
  simplex, cyclically adjacent corners of a quad, and hex corners whose unit
  cube coordinates differ in exactly one axis.
* ``sort_restatement``: the paper's own GPU recipe run with numpy on the CPU
  (Sec. 2.2: emit integer pairs, sort by key, segment by key), plus removal
  of repeated pairs so rows are sets.
* ``brute_force_faces``: element face adjacency over all element pairs,
  with faces derived geometrically too: edges of a triangle or quad (the
  sides), 3-subsets of a tet, and hex corners sharing one unit-cube
  coordinate value.
* closed forms for structured grids and the per-node triangle identity.
"""
from __future__ import annotations

import itertools

import numpy as np

# unit-cube coordinates of the VTK hex corners 0..7
HEX_XYZ = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]


def local_edges(etype: int):
    """Local edges derived from the element's shape (not copied from a table)."""
    if etype == 0:        # triangle: a simplex, every pair
        return list(itertools.combinations(range(3), 2))
    if etype == 2:        # tetrahedron: a simplex, every pair
        return list(itertools.combinations(range(4), 2))
    if etype == 1:        # quad: corners adjacent around the boundary cycle
        return [(i, (i + 1) % 4) for i in range(4)]
    if etype == 3:        # hex: corners one unit apart
        return [(i, j) for i, j in itertools.combinations(range(8), 2)
                if sum(abs(a - b) for a, b in zip(HEX_XYZ[i], HEX_XYZ[j])) == 1]
    raise ValueError(etype)


def local_faces(etype: int):
    """Local faces derived from the element's shape (not copied from a table):
    the sides of a polygon, the vertex triples of a tet, the six sets of hex
    corners that agree in one unit-cube coordinate."""
    if etype in (0, 1):   # polygon: its sides are its edges
        return local_edges(etype)
    if etype == 2:
        return list(itertools.combinations(range(4), 3))
    if etype == 3:
        return [tuple(i for i in range(8) if HEX_XYZ[i][d] == c) for d in range(3) for c in (0, 1)]
    raise ValueError(etype)


def brute_force_faces(elements):
    """Rows of element face neighbours: e != f are neighbours iff every node of
    some face of one of them (a face whose nodes are all distinct) is a node
    of the other."""
    faces = [[frozenset(nd[i] for i in fc) for fc in local_faces(t) if len({nd[i] for i in fc}) == len(fc)]
             for t, nd in elements]
    nodes = [set(nd) for _, nd in elements]
    rows = [[] for _ in elements]
    for e, f in itertools.combinations(range(len(elements)), 2):
        if any(fc <= nodes[f] for fc in faces[e]) or any(fc <= nodes[e] for fc in faces[f]):
            rows[e].append(f)
            rows[f].append(e)
    return rows


def brute_force(elements, n_nodes):
    """Rows (lists) of neighbor nodes and neighbor elements for tiny meshes."""
    edge_sets = [set(frozenset((nd[a], nd[b])) for a, b in local_edges(t) if nd[a] != nd[b])
                 for t, nd in elements]
    nodes, elems = [], []
    for v in range(n_nodes):
        nodes.append([u for u in range(n_nodes)
                      if u != v and any(frozenset((u, v)) in es for es in edge_sets)])
        elems.append([e for e, (t, nd) in enumerate(elements) if v in nd])
    return nodes, elems


def sort_restatement(elements, n_nodes):
    """CSR (row_ptr, col) for nodes and elements via pair emission + sort + unique."""
    ka, va, ke, ve = [], [], [], []
    for e, (t, nd) in enumerate(elements):
        for a, b in local_edges(t):
            if nd[a] != nd[b]:
                ka += [nd[a], nd[b]]
                va += [nd[b], nd[a]]
        for x in nd:
            ke.append(x)
            ve.append(e)

    def csr(keys, vals):
        keys = np.asarray(keys, dtype=np.int64)
        vals = np.asarray(vals, dtype=np.int64)
        order = np.lexsort((vals, keys))           # by key, then value
        k, v = keys[order], vals[order]
        if k.size:
            keep = np.ones(k.size, dtype=bool)
            keep[1:] = (k[1:] != k[:-1]) | (v[1:] != v[:-1])
            k, v = k[keep], v[keep]
        counts = np.bincount(k, minlength=n_nodes) if k.size else np.zeros(n_nodes, dtype=np.int64)
        rp = np.zeros(n_nodes + 1, dtype=np.int64)
        np.cumsum(counts, out=rp[1:])
        return rp, v.astype(np.int32)

    return csr(ka, va), csr(ke, ve)


def rows_of(rp, col):
    return [col[rp[v]:rp[v + 1]].tolist() for v in range(len(rp) - 1)]


def unique_edges(elements):
    """Set of undirected edges (min, max), by hashing."""
    s = set()
    for t, nd in elements:
        for a, b in local_edges(t):
            x, y = nd[a], nd[b]
            if x != y:
                s.add((min(x, y), max(x, y)))
    return s


def tri_edge_triangle_counts(conn):
    """{(min,max): number of triangles containing the edge} for a triangle mesh."""
    c = np.asarray(conn, dtype=np.int64).reshape(-1, 3)
    e = np.concatenate([c[:, [0, 1]], c[:, [1, 2]], c[:, [2, 0]]])
    e.sort(axis=1)
    key = e[:, 0] * (int(c.max(initial=0)) + 1) + e[:, 1]
    uk, cnt = np.unique(key, return_counts=True)
    return uk, cnt, int(c.max(initial=0)) + 1


# ---- closed forms (m cells per side, n = m + 1 nodes per side)

def tri_grid_edges(m):          # horizontal + vertical + one diagonal per quad
    n = m + 1
    return 2 * m * n + m * m


def quad_grid_edges(m):
    n = m + 1
    return 2 * m * n


def kuhn_grid_edges(m):         # axis edges + face diagonals + cell diagonals
    n = m + 1
    return 3 * m * n * n + 3 * m * m * n + m ** 3


def kuhn_grid_faces(m):         # triangles: 2 per grid square + 6 interior per cell
    n = m + 1
    return 6 * m * m * n + 6 * m ** 3


def hex_grid_edges(m):
    n = m + 1
    return 3 * m * n * n


def hex_grid_faces(m):
    n = m + 1
    return 3 * m * m * n


KUHN_OFFSETS = sorted([tuple(s * x for x in o) for s in (1, -1) for o in
                       [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]])
HEX_OFFSETS = sorted([tuple(s * x for x in o) for s in (1, -1) for o in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]])
