"""Surface-mesh files in, connectivity out: PLY (ascii, binary little and big
endian) and Wavefront OBJ readers that turn a polygon mesh into the
library's mesh form (int32 connectivity, 0-based node ids), plus writers used
by the tests to round-trip generated meshes.

The paper measures scanned triangle surfaces distributed as PLY files
(Sec. 3.1, Table 1).  Only the topology matters to the build: vertex
positions and any other vertex or face properties are skipped.  Faces with
three corners become triangles and faces with four become quads; a file with
both becomes a mixed mesh (per-element type and offsets).  Larger polygons
are refused (their edges are not in the element tables).
"""
from __future__ import annotations

import os
import re
from typing import List, Tuple

import numpy as np

from .meshgen import MIXED, QUAD, TRI, Mesh

# PLY scalar types and their numpy codes
_PLY_TYPES = {
    "char": "i1", "int8": "i1", "uchar": "u1", "uint8": "u1",
    "short": "i2", "int16": "i2", "ushort": "u2", "uint16": "u2",
    "int": "i4", "int32": "i4", "uint": "u4", "uint32": "u4",
    "float": "f4", "float32": "f4", "double": "f8", "float64": "f8",
}
_FACE_TYPE = {3: TRI, 4: QUAD}


def from_faces(faces: List[Tuple[int, ...]] | np.ndarray, n_nodes: int, name: str = "") -> Mesh:
    """Mesh from polygon faces (0-based corner lists) over n_nodes vertices."""
    if isinstance(faces, np.ndarray) and faces.ndim == 2:
        k = faces.shape[1] if faces.size else 3
        if k not in _FACE_TYPE:
            raise ValueError(f"faces with {k} corners are not supported (triangles and quads only)")
        if faces.size and (faces.min() < 0 or faces.max() >= n_nodes):
            raise ValueError("a face refers to a vertex that does not exist")
        return Mesh(_FACE_TYPE[k], n_nodes, np.ascontiguousarray(faces, dtype=np.int32).reshape(-1), name=name)
    sizes = np.array([len(f) for f in faces], dtype=np.int64)
    bad = sizes[(sizes != 3) & (sizes != 4)]
    if bad.size:
        raise ValueError(f"a face with {int(bad[0])} corners: triangles and quads only")
    conn = np.fromiter((v for f in faces for v in f), dtype=np.int64, count=int(sizes.sum()))
    if conn.size and (conn.min() < 0 or conn.max() >= n_nodes):
        raise ValueError("a face refers to a vertex that does not exist")
    conn = conn.astype(np.int32)
    kinds = set(sizes.tolist())
    if len(kinds) <= 1:
        return Mesh(_FACE_TYPE[kinds.pop()] if kinds else TRI, n_nodes, conn, name=name)
    ptr = np.zeros(len(faces) + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    et = np.where(sizes == 3, TRI, QUAD).astype(np.uint8)
    return Mesh(MIXED, n_nodes, conn, elem_ptr=ptr, elem_type=et, name=name)


# ------------------------------------------------------------------ PLY

def _ply_header(f):
    """(format, [(element, count, [(property, type or ('list', count type, item type))])]);
    the file is left at the first byte of the body."""
    if f.readline().strip() != b"ply":
        raise ValueError("not a PLY file")
    fmt, elems = None, []
    while True:
        line = f.readline()
        if not line:
            raise ValueError("PLY header has no end_header")
        words = line.decode("ascii", "replace").split()
        if not words or words[0] in ("comment", "obj_info"):
            continue
        if words[0] == "format":
            fmt = words[1]
        elif words[0] == "element":
            elems.append((words[1], int(words[2]), []))
        elif words[0] == "property":
            if not elems:
                raise ValueError("PLY property before any element")
            if words[1] == "list":
                elems[-1][2].append((words[4], ("list", _PLY_TYPES[words[2]], _PLY_TYPES[words[3]])))
            else:
                elems[-1][2].append((words[2], _PLY_TYPES[words[1]]))
        elif words[0] == "end_header":
            break
    if fmt not in ("ascii", "binary_little_endian", "binary_big_endian"):
        raise ValueError(f"unknown PLY format {fmt!r}")
    return fmt, elems


def _face_list_index(props):
    for i, (name, t) in enumerate(props):
        if isinstance(t, tuple) and name in ("vertex_indices", "vertex_index"):
            return i
    raise ValueError("PLY face element has no vertex_indices list")


def read_ply(path: str) -> Mesh:
    """The faces of a PLY file as a mesh over its vertices."""
    with open(path, "rb") as f:
        fmt, elems = _ply_header(f)
        body = f.read()
    name = os.path.basename(path)
    n_nodes, faces = 0, None
    if fmt == "ascii":
        tokens = body.split()
        pos = 0
        for ename, count, props in elems:
            if ename == "face":
                li = _face_list_index(props)
                out = []
                for _ in range(count):
                    corners = None
                    for i, (_, t) in enumerate(props):
                        if isinstance(t, tuple):
                            k = int(tokens[pos]); pos += 1
                            vals = tokens[pos:pos + k]; pos += k
                            if i == li:
                                corners = tuple(int(v) for v in vals)
                        else:
                            pos += 1
                    out.append(corners)
                faces = out
            else:
                if ename == "vertex":
                    n_nodes = count
                for _ in range(count):
                    for _, t in props:
                        if isinstance(t, tuple):
                            pos += 1 + int(tokens[pos])
                        else:
                            pos += 1
        return from_faces(faces or [], n_nodes, name)
    order = "<" if fmt == "binary_little_endian" else ">"
    off = 0
    for ename, count, props in elems:
        if ename == "face":
            faces, off = _ply_binary_faces(body, off, count, props, order)
            continue
        if any(isinstance(t, tuple) for _, t in props):
            raise ValueError(f"PLY element {ename!r} with list properties is not supported")
        if ename == "vertex":
            n_nodes = count
        off += count * sum(np.dtype(t).itemsize for _, t in props)
    if faces is None:
        faces = np.zeros((0, 3), dtype=np.int32)
    return from_faces(faces, n_nodes, name)


def _ply_binary_faces(body: bytes, off: int, count: int, props, order: str):
    li = _face_list_index(props)
    simple = len(props) == 1
    if simple and count:
        _, (_, ct, it) = props[0]
        cdt, idt = np.dtype(order + ct), np.dtype(order + it)
        k = int(np.frombuffer(body, dtype=cdt, count=1, offset=off)[0])
        rec = np.dtype([("n", cdt), ("v", idt, (k,))])
        if off + count * rec.itemsize <= len(body):
            arr = np.frombuffer(body, dtype=rec, count=count, offset=off)
            if (arr["n"] == k).all():           # every face has k corners: one vectorised read
                return arr["v"].astype(np.int64), off + count * rec.itemsize
    faces = []                                  # mixed corner counts or extra face properties
    for _ in range(count):
        corners = None
        for i, (_, t) in enumerate(props):
            if isinstance(t, tuple):
                cdt, idt = np.dtype(order + t[1]), np.dtype(order + t[2])
                k = int(np.frombuffer(body, dtype=cdt, count=1, offset=off)[0])
                off += cdt.itemsize
                vals = np.frombuffer(body, dtype=idt, count=k, offset=off)
                off += k * idt.itemsize
                if i == li:
                    corners = tuple(int(v) for v in vals)
            else:
                off += np.dtype(t).itemsize
        faces.append(corners)
    return faces, off


def write_ply(mesh: Mesh, path: str, binary: bool = True, big_endian: bool = False,
              vertex_extra: Tuple[str, ...] = ()) -> None:
    """Write a triangle, quad or mixed tri/quad mesh as PLY (vertex positions
    are placeholders; ``vertex_extra`` adds float properties per vertex)."""
    faces = [nd for _, nd in mesh.elements()]
    head = ["ply", "format " + ("ascii" if not binary else
                                "binary_big_endian" if big_endian else "binary_little_endian") + " 1.0",
            "comment written by paper_1604_04689_gb300.meshio",
            f"element vertex {mesh.n_nodes}", "property float x", "property float y", "property float z"]
    head += [f"property float {p}" for p in vertex_extra]
    head += [f"element face {len(faces)}", "property list uchar int vertex_indices", "end_header"]
    nv = 3 + len(vertex_extra)
    with open(path, "wb") as f:
        f.write(("\n".join(head) + "\n").encode("ascii"))
        if not binary:
            for v in range(mesh.n_nodes):
                f.write((" ".join(["0"] * nv) + "\n").encode("ascii"))
            for nd in faces:
                f.write((f"{len(nd)} " + " ".join(str(x) for x in nd) + "\n").encode("ascii"))
            return
        o = ">" if big_endian else "<"
        f.write(np.zeros(mesh.n_nodes * nv, dtype=o + "f4").tobytes())
        for nd in faces:
            f.write(np.array([len(nd)], dtype="u1").tobytes() + np.array(nd, dtype=o + "i4").tobytes())


# ------------------------------------------------------------------ OBJ

_SLASH = re.compile(rb"/.*")


def read_obj(path: str) -> Mesh:
    """The faces of a Wavefront OBJ file (``f`` lines; ``v/vt/vn`` corner forms
    and negative, relative indices allowed) as a mesh over its ``v`` vertices."""
    n_nodes, faces = 0, []
    with open(path, "rb") as f:
        for line in f:
            w = line.split()
            if not w:
                continue
            if w[0] == b"v":
                n_nodes += 1
            elif w[0] == b"f":
                corners = []
                for c in w[1:]:
                    i = int(_SLASH.sub(b"", c))
                    corners.append(i - 1 if i > 0 else n_nodes + i)
                faces.append(tuple(corners))
    return from_faces(faces, n_nodes, os.path.basename(path))


def write_obj(mesh: Mesh, path: str) -> None:
    with open(path, "w") as f:
        f.write("# written by paper_1604_04689_gb300.meshio\n")
        for _ in range(mesh.n_nodes):
            f.write("v 0 0 0\n")
        for _, nd in mesh.elements():
            f.write("f " + " ".join(str(x + 1) for x in nd) + "\n")


def read_mesh(path: str) -> Mesh:
    """Read a .ply or .obj surface mesh."""
    ext = os.path.splitext(path)[1].lower()
    if ext == ".ply":
        return read_ply(path)
    if ext == ".obj":
        return read_obj(path)
    raise ValueError(f"unknown mesh file type {ext!r} (.ply or .obj)")
