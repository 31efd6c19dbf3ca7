"""CPU oracle for one-ring neighbor finding -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never calls it.

``neighbors(mesh, want)`` runs the plain single-threaded C++ oracle
(``oracle.cpp``: a loop over all elements into one ordered set per node, the
serial method of Sec. 1 / Sec. 3.2.2 of the paper with set semantics) and
returns canonical CSR arrays.  ``rows(mesh, sample, want)`` returns the rows of
a sample of nodes only, for checking full-size builds.

The mesh argument is any object with ``etype``, ``n_nodes``, ``n_elems``,
``n_conn``, ``conn`` (int32), ``elem_ptr`` (int64 or None) and ``elem_type``
(uint8 or None) -- e.g. a ``meshgen.Mesh``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NODES, ELEMS, BOTH = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (g++ -O2, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """ctypes handle on an oracle shared library at ``path`` (signatures set)."""
    lib = C.CDLL(path)
    P, I64, I32, U8 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint8
    lib.oracle_build.restype = P
    lib.oracle_build.argtypes = [I32, I64, I64, I64, C.POINTER(I32), C.POINTER(I64),
                                 C.POINTER(U8), C.c_int]
    lib.oracle_rows.restype = P
    lib.oracle_rows.argtypes = [I32, I64, I64, I64, C.POINTER(I32), C.POINTER(I64),
                                C.POINTER(U8), C.c_int, C.POINTER(I32), I64]
    lib.oracle_status.restype = C.c_int
    lib.oracle_status.argtypes = [P]
    lib.oracle_nnz.restype = I64
    lib.oracle_nnz.argtypes = [P, C.c_int]
    lib.oracle_copy.restype = None
    lib.oracle_copy.argtypes = [P, C.c_int, C.POINTER(I64), C.POINTER(I32)]
    lib.oracle_elem_adjacency.restype = P
    lib.oracle_elem_adjacency.argtypes = [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int64), C.POINTER(C.c_uint8), C.POINTER(C.c_int32),
                                          C.c_int64]
    lib.oracle_free.restype = None
    lib.oracle_free.argtypes = [P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def _mesh_args(mesh):
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    ep = None if mesh.elem_ptr is None else np.ascontiguousarray(mesh.elem_ptr, dtype=np.int64)
    et = None if mesh.elem_type is None else np.ascontiguousarray(mesh.elem_type, dtype=np.uint8)
    keep = (conn, ep, et)
    args = (int(mesh.etype), int(mesh.n_nodes), int(mesh.n_elems), int(conn.shape[0]),
            _ptr(conn, C.c_int32), _ptr(ep, C.c_int64), _ptr(et, C.c_uint8))
    return args, keep


def _run(lib, h, want, n_rows):
    try:
        res = {"status": lib.oracle_status(h)}
        for which, key in ((NODES, "nodes"), (ELEMS, "elems")):
            if want & which:
                nnz = lib.oracle_nnz(h, which)
                rp = np.empty(n_rows + 1, dtype=np.int64)
                col = np.empty(nnz, dtype=np.int32)
                lib.oracle_copy(h, which, _ptr(rp, C.c_int64), _ptr(col, C.c_int32))
                res[key] = (rp, col)
        return res
    finally:
        lib.oracle_free(h)


def neighbors(mesh, want: int = BOTH, lib=None) -> dict:
    """{'status': int, 'nodes': (row_ptr, col), 'elems': (row_ptr, col)} for the whole mesh.

    ``lib`` selects another build of the oracle (see ``load_library``)."""
    lib = lib or _load()
    args, keep = _mesh_args(mesh)
    h = lib.oracle_build(*args, want)
    return _run(lib, h, want, int(mesh.n_nodes))


def rows(mesh, sample, want: int = BOTH, lib=None) -> dict:
    """Same as ``neighbors`` but only for the nodes in ``sample`` (CSR over the sample)."""
    lib = lib or _load()
    args, keep = _mesh_args(mesh)
    s = np.ascontiguousarray(sample, dtype=np.int32)
    h = lib.oracle_rows(*args, want, _ptr(s, C.c_int32), int(s.shape[0]))
    return _run(lib, h, want, int(s.shape[0]))


def element_adjacency(mesh, sample=None, lib=None) -> dict:
    """{'status': int, 'adj': (row_ptr, col)}: face neighbours of every element
    (or of the elements in ``sample``, CSR over the sample)."""
    lib = lib or _load()
    args, keep = _mesh_args(mesh)
    if sample is None:
        h = lib.oracle_elem_adjacency(*args, None, 0)
        n = int(mesh.n_elems)
    else:
        s = np.ascontiguousarray(sample, dtype=np.int32)
        h = lib.oracle_elem_adjacency(*args, _ptr(s, C.c_int32), int(s.shape[0]))
        n = int(s.shape[0])
    res = _run(lib, h, ELEMS, n)
    return {"status": res["status"], "adj": res["elems"]}
