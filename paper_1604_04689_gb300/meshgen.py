"""Seeded synthetic mesh generators (host side, numpy).

This module is input generation only: it builds element-to-node connectivity
arrays and holds none of the neighbor-finding arithmetic.  Both the CUDA path
and the CPU oracle consume what it produces; neither is imported here.

Meshes (all connectivity int32, element id = position in the returned array):

* ``tri_grid(n, seed)``   n x n node grid, every one of the (n-1)^2 quads cut
  into two triangles along a seeded random diagonal.
* ``quad_grid(n, seed)``  n x n node grid of quads.
* ``tet_grid(n, seed)``   n^3 node grid, every cube cell split into the six
  tetrahedra of the Kuhn (Freudenthal) subdivision along its main diagonal.
* ``hex_grid(n, seed)``   n^3 node grid of hexahedra in VTK local order.
* ``mixed_grid(n, seed)`` hex grid in which a seeded 30% of the cells are
  replaced by their six Kuhn tetrahedra (type-tagged, per-element offsets).

Randomness is counter based so that a device generator can reproduce it
bit for bit: ``splitmix64`` (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as published by
Vigna) drives every choice, and node/element relabelings are a 4-round
Feistel network over the next even power of two with cycle walking, which is a
bijection on [0, N).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

TRI, QUAD, TET, HEX, MIXED = 0, 1, 2, 3, 255
NPE = {TRI: 3, QUAD: 4, TET: 4, HEX: 8}
TYPE_NAMES = {TRI: "tri", QUAD: "quad", TET: "tet", HEX: "hex", MIXED: "mixed"}

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15

# stream tags, so that independent choices drawn from one seed never collide
STREAM_NODE_PERM = 1
STREAM_ELEM_PERM = 2
STREAM_DIAG = 3
STREAM_HOLE = 4
STREAM_MIXED = 5
STREAM_REQUEST = 6

# Kuhn split of a VTK-ordered hex (0=(0,0,0) 1=(1,0,0) 2=(1,1,0) 3=(0,1,0)
# 4=(0,0,1) 5=(1,0,1) 6=(1,1,1) 7=(0,1,1)): one tet per axis order, all
# sharing the 0-6 diagonal, so neighbouring cells stay conforming.
KUHN_TETS = np.array([[0, 1, 2, 6], [0, 1, 5, 6], [0, 3, 2, 6],
                      [0, 3, 7, 6], [0, 4, 5, 6], [0, 4, 7, 6]], dtype=np.int64)


def splitmix64(x):
    """splitmix64 output function on uint64 numpy arrays or Python ints."""
    if isinstance(x, (int, np.integer)):
        z = (int(x) + _GOLDEN) & _M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)
    z = np.asarray(x, dtype=np.uint64) + np.uint64(_GOLDEN)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of one independent random stream of a seed."""
    return splitmix64((splitmix64(seed) ^ (stream * _GOLDEN)) & _M64)


def hash_u64(key: int, idx):
    """Counter-based draw number ``idx`` of the stream with key ``key``."""
    return splitmix64(np.asarray(idx, dtype=np.uint64) ^ np.uint64(key))


def feistel_perm(n: int, key: int, idx=None) -> np.ndarray:
    """pi(idx) for the seeded bijection pi on [0, n) (all of [0, n) if idx is None).

    4 balanced Feistel rounds on 2h bits (2^(2h) >= n, h >= 1), round function
    the low h bits of splitmix64(round_key ^ R); values >= n are walked through
    the cipher again until they land inside [0, n).
    """
    if n <= 0:
        return np.zeros(0, dtype=np.int64)
    if idx is None:
        idx = np.arange(n, dtype=np.uint64)
    x = np.asarray(idx, dtype=np.uint64).copy()
    bits = max(2, (n - 1).bit_length())
    h = (bits + 1) // 2
    mask = np.uint64((1 << h) - 1)
    sh = np.uint64(h)
    rk = [np.uint64(splitmix64((key + r * 0xD1B54A32D192ED03) & _M64)) for r in range(4)]

    def enc(v):
        L = v >> sh
        R = v & mask
        for r in range(4):
            f = splitmix64(R ^ rk[r]) & mask
            L, R = R, L ^ f
        return (L << sh) | R

    out = enc(x)
    bad = out >= np.uint64(n)
    while bad.any():
        out[bad] = enc(out[bad])
        bad = out >= np.uint64(n)
    return out.astype(np.int64)


@dataclass
class Mesh:
    """A mesh as plain arrays; ``etype`` is TRI/QUAD/TET/HEX or MIXED."""
    etype: int
    n_nodes: int
    conn: np.ndarray                      # int32, flat
    elem_ptr: Optional[np.ndarray] = None  # int64 [n_elems+1], MIXED only
    elem_type: Optional[np.ndarray] = None  # uint8 [n_elems], MIXED only
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_elems(self) -> int:
        if self.etype == MIXED:
            return int(self.elem_type.shape[0])
        return int(self.conn.shape[0] // NPE[self.etype])

    @property
    def n_conn(self) -> int:
        return int(self.conn.shape[0])

    def elements(self):
        """List of (type, node tuple) per element, for small meshes only."""
        out = []
        if self.etype == MIXED:
            for e in range(self.n_elems):
                a, b = int(self.elem_ptr[e]), int(self.elem_ptr[e + 1])
                out.append((int(self.elem_type[e]), tuple(int(x) for x in self.conn[a:b])))
        else:
            k = NPE[self.etype]
            c = self.conn.reshape(-1, k)
            for e in range(c.shape[0]):
                out.append((self.etype, tuple(int(x) for x in c[e])))
        return out


def _relabel(nat_conn: np.ndarray, n_nodes: int, seed: int, permute_nodes: bool) -> np.ndarray:
    if not permute_nodes:
        return nat_conn.astype(np.int32)
    pi = feistel_perm(n_nodes, stream_key(seed, STREAM_NODE_PERM))
    return pi[nat_conn].astype(np.int32)


def _reorder(elems: np.ndarray, seed: int, permute_elems: bool) -> np.ndarray:
    """Element at natural index t moves to position pi'(t)."""
    if not permute_elems or elems.shape[0] == 0:
        return elems
    t = elems.shape[0]
    pos = feistel_perm(t, stream_key(seed, STREAM_ELEM_PERM))
    out = np.empty_like(elems)
    out[pos] = elems
    return out


def tri_grid_natural(n: int, seed: int, diag: Optional[int] = None) -> np.ndarray:
    """(2(n-1)^2, 3) natural-order triangles; node (i, j) has id i + n*j.

    Quad (i, j) with corners a=(i,j) b=(i+1,j) c=(i+1,j+1) d=(i,j+1) becomes
    (a,b,c),(a,c,d) when its diagonal bit is 0 and (a,b,d),(b,c,d) when it is 1.
    The bit is the low bit of the quad's draw, or ``diag`` for every quad.
    """
    m = n - 1
    if m <= 0:
        return np.zeros((0, 3), dtype=np.int64)
    i, j = np.meshgrid(np.arange(m, dtype=np.int64), np.arange(m, dtype=np.int64), indexing="xy")
    i = i.ravel(); j = j.ravel()            # quad index q = i + m*j
    a = i + n * j; b = a + 1; c = a + 1 + n; d = a + n
    if diag is None:
        q = np.arange(m * m, dtype=np.uint64)
        bit = (hash_u64(stream_key(seed, STREAM_DIAG), q) & np.uint64(1)).astype(bool)
    else:
        bit = np.full(m * m, bool(diag))
    t = np.empty((m * m, 2, 3), dtype=np.int64)
    t[:, 0, 0] = a; t[:, 0, 1] = b; t[:, 0, 2] = np.where(bit, d, c)
    t[:, 1, 0] = np.where(bit, b, a); t[:, 1, 1] = c; t[:, 1, 2] = d
    return t.reshape(-1, 3)


def tri_grid(n: int, seed: int, holes: float = 0.0, diag: Optional[int] = None,
             permute_nodes: bool = True, permute_elems: bool = True) -> Mesh:
    tris = tri_grid_natural(n, seed, diag)
    if holes > 0.0 and tris.shape[0]:
        thr = np.uint64(min(int(holes * 2.0 ** 64), _M64))
        keep = hash_u64(stream_key(seed, STREAM_HOLE), np.arange(tris.shape[0], dtype=np.uint64)) >= thr
        tris = tris[keep]
    tris = _reorder(tris, seed, permute_elems)
    conn = _relabel(tris.ravel(), n * n, seed, permute_nodes)
    return Mesh(TRI, n * n, conn, name=f"tri{n}x{n}" + (f"-holes{holes:g}" if holes else ""),
                meta=dict(n=n, seed=seed, holes=holes))


def quad_grid(n: int, seed: int, permute_nodes: bool = True, permute_elems: bool = True) -> Mesh:
    m = n - 1
    i, j = np.meshgrid(np.arange(max(m, 0), dtype=np.int64), np.arange(max(m, 0), dtype=np.int64), indexing="xy")
    a = (i + n * j).ravel()
    q = np.stack([a, a + 1, a + 1 + n, a + n], axis=1)
    q = _reorder(q, seed, permute_elems)
    conn = _relabel(q.ravel(), n * n, seed, permute_nodes)
    return Mesh(QUAD, n * n, conn, name=f"quad{n}x{n}", meta=dict(n=n, seed=seed))


def _hex_cells(n: int) -> np.ndarray:
    """(m^3, 8) VTK-ordered hex cells of an n^3 grid; node (i,j,k) = i + n*j + n*n*k."""
    m = n - 1
    if m <= 0:
        return np.zeros((0, 8), dtype=np.int64)
    r = np.arange(m, dtype=np.int64)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")   # cell index i + m*j + m*m*k
    base = (i + n * j + n * n * k).ravel()
    off = np.array([0, 1, 1 + n, n, n * n, n * n + 1, n * n + 1 + n, n * n + n], dtype=np.int64)
    return base[:, None] + off[None, :]


def tet_grid(n: int, seed: int, permute_nodes: bool = True, permute_elems: bool = True) -> Mesh:
    hexes = _hex_cells(n)
    tets = hexes[:, KUHN_TETS].reshape(-1, 4)      # 6 per cell, consecutive
    tets = _reorder(tets, seed, permute_elems)
    conn = _relabel(tets.ravel(), n ** 3, seed, permute_nodes)
    return Mesh(TET, n ** 3, conn, name=f"tet{n}^3", meta=dict(n=n, seed=seed))


def hex_grid(n: int, seed: int, permute_nodes: bool = True, permute_elems: bool = False) -> Mesh:
    hexes = _reorder(_hex_cells(n), seed, permute_elems)
    conn = _relabel(hexes.ravel(), n ** 3, seed, permute_nodes)
    return Mesh(HEX, n ** 3, conn, name=f"hex{n}^3", meta=dict(n=n, seed=seed))


def mixed_grid(n: int, seed: int, frac_tet: float = 0.30, permute_nodes: bool = True) -> Mesh:
    """Hex grid with a seeded fraction of cells replaced by their 6 Kuhn tets.

    The replacement tets sit consecutively where the hex was (cell order kept).
    """
    hexes = _hex_cells(n)
    c = hexes.shape[0]
    thr = np.uint64(min(int(frac_tet * 2.0 ** 64), _M64))
    split = hash_u64(stream_key(seed, STREAM_MIXED), np.arange(c, dtype=np.uint64)) < thr
    n_per = np.where(split, 6, 1)
    ebase = np.zeros(c + 1, dtype=np.int64)
    np.cumsum(n_per, out=ebase[1:])
    t = int(ebase[-1])
    etype = np.full(t, HEX, dtype=np.uint8)
    npe = np.full(t, 8, dtype=np.int64)
    sidx = np.nonzero(split)[0]
    tet_pos = (ebase[sidx][:, None] + np.arange(6)[None, :]).ravel()
    etype[tet_pos] = TET
    npe[tet_pos] = 4
    elem_ptr = np.zeros(t + 1, dtype=np.int64)
    np.cumsum(npe, out=elem_ptr[1:])
    conn = np.empty(int(elem_ptr[-1]), dtype=np.int64)
    hidx = np.nonzero(~split)[0]
    hpos = elem_ptr[ebase[hidx]]
    conn[(hpos[:, None] + np.arange(8)[None, :]).ravel()] = hexes[hidx].ravel()
    tets = hexes[sidx][:, KUHN_TETS]               # (s, 6, 4)
    tpos = elem_ptr[tet_pos]
    conn[(tpos[:, None] + np.arange(4)[None, :]).ravel()] = tets.reshape(-1, 4).ravel()
    conn32 = _relabel(conn, n ** 3, seed, permute_nodes)
    return Mesh(MIXED, n ** 3, conn32, elem_ptr=elem_ptr, elem_type=etype,
                name=f"mixed{n}^3", meta=dict(n=n, seed=seed, frac_tet=frac_tet,
                                              n_hex=int((~split).sum()), n_split=int(split.sum())))


def from_elements(elems, n_nodes: int, name: str = "") -> Mesh:
    """Mesh from a list of (type, nodes); uniform type if all types agree."""
    types = {t for t, _ in elems}
    if len(types) == 1:
        t = types.pop()
        conn = np.array([x for _, nd in elems for x in nd], dtype=np.int32)
        return Mesh(t, n_nodes, conn, name=name)
    et = np.array([t for t, _ in elems], dtype=np.uint8)
    ptr = np.zeros(len(elems) + 1, dtype=np.int64)
    np.cumsum([len(nd) for _, nd in elems], out=ptr[1:])
    conn = np.array([x for _, nd in elems for x in nd], dtype=np.int32)
    return Mesh(MIXED, n_nodes, conn, elem_ptr=ptr, elem_type=et, name=name)


# ---------------------------------------------------------------- workloads

WORKLOAD_NAMES = ("tri64", "tri2048", "tri2048_holes", "tet161", "hex257", "mixed257")


def workload_mesh(name: str) -> Mesh:
    """The seeded synthetic workloads, by name.

    tri64: triangle grid 64x64 (seed 0); tri2048: triangle grid 2048x2048
    (seed 1); tri2048_holes: the same grid with 5% of triangles deleted
    (seed 100); tet161: Kuhn tet grid 161^3 (seed 2); hex257: hex grid 257^3
    (seed 3); mixed257: hex257 with 30% of cells split into 6 tets (seed 103).
    """
    if name == "tri64":
        return tri_grid(64, 0)
    if name == "tri2048":
        return tri_grid(2048, 1)
    if name == "tri2048_holes":
        return tri_grid(2048, 100, holes=0.05)
    if name == "tet161":
        return tet_grid(161, 2)
    if name == "hex257":
        return hex_grid(257, 3)
    if name == "mixed257":
        return mixed_grid(257, 103)
    raise ValueError(f"unknown workload {name!r}; known: {', '.join(WORKLOAD_NAMES)}")


def request_spec(i: int, base_seed: int = 4, lo: float = 1e3, hi: float = 2e6):
    """(type, n, seed) of serving request i: log-uniform element count in [lo, hi],
    type uniform over {tri grid, Kuhn tet grid, hex grid}, grid side chosen so the
    element count is closest to the draw."""
    rs = splitmix64(((base_seed << 32) + i) & _M64)
    u = splitmix64(rs ^ 0x1) / 2.0 ** 64
    target = math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    t = (TRI, TET, HEX)[splitmix64(rs ^ 0x2) % 3]
    if t == TRI:
        f = lambda m: 2 * m * m
    elif t == TET:
        f = lambda m: 6 * m ** 3
    else:
        f = lambda m: m ** 3
    m = 1
    while f(m + 1) <= target:
        m += 1
    if abs(f(m + 1) - target) < abs(f(m) - target):
        m += 1
    return t, m + 1, rs


def request_mesh(i: int, base_seed: int = 4) -> Mesh:
    t, n, s = request_spec(i, base_seed)
    if t == TRI:
        return tri_grid(n, s)
    if t == TET:
        return tet_grid(n, s)
    return hex_grid(n, s)


def poisson_arrivals(n: int, rate: float, seed: int = 4) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate, from the seed."""
    u = (hash_u64(stream_key(seed, STREAM_REQUEST), np.arange(n, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64)
    u = (u + 0.5) / 2.0 ** 53
    return np.cumsum(-np.log(u) / rate)
