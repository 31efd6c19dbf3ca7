"""ctypes binding of libnn.so (include/nn.h): argument marshalling only.

Every step of the build runs in the CUDA kernels behind the C ABI; this
module only turns torch device tensors into the C structs and calls it.
PyTorch provides device memory and the stream.

Low level (same names as the C ABI): ``nn_create``, ``nn_destroy``,
``nn_query``, ``nn_neighbor_nodes``, ``nn_neighbor_elements``,
``nn_neighbors_both``, ``nn_chunk_slabs``, ``nn_chunk_count``,
``nn_chunk_plan``, ``nn_neighbors_chunked``, ``nn_status_str`` and the rest
of include/nn.h.

High level: ``DeviceMesh`` (connectivity on the device) and ``Builder``,
which sizes and allocates workspace and outputs with torch and returns CSR
tensors.  If the library has not been built, loading raises RuntimeError --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnn.so")

TRI, QUAD, TET, HEX, MIXED = 0, 1, 2, 3, 255
WANT_NODES, WANT_ELEMS, WANT_BOTH = 1, 2, 3
STATUS = {0: "NN_OK", 1: "NN_ERR_ARG", 2: "NN_ERR_WORKSPACE", 3: "NN_ERR_CAPACITY", 4: "NN_ERR_NODE_RANGE",
          5: "NN_ERR_ELEM_PTR", 6: "NN_ERR_TIMEOUT", 7: "NN_ERR_BUDGET", 8: "NN_ERR_CUDA", 9: "NN_ERR_BOUNDS"}
NPE = {TRI: 3, QUAD: 4, TET: 4, HEX: 8}


class NNMesh(C.Structure):
    _fields_ = [("type", C.c_int32), ("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("n_conn", C.c_int64),
                ("conn", C.c_void_p), ("elem_ptr", C.c_void_p), ("elem_type", C.c_void_p)]


class NNCSR(C.Structure):
    _fields_ = [("row_ptr", C.c_void_p), ("col", C.c_void_p), ("col_capacity", C.c_int64)]


class NNBatchCaps(C.Structure):
    _fields_ = [("max_meshes", C.c_int32), ("want", C.c_int32), ("max_elems", C.c_int64),
                ("max_nodes", C.c_int64), ("max_conn", C.c_int64), ("sb", C.c_int32)]


class NNTuning(C.Structure):
    _fields_ = [("sb", C.c_int32), ("bucket_threads", C.c_int32), ("bucket_ctas_per_sm", C.c_int32)]


class NNChunk(C.Structure):
    _fields_ = [("node_lo", C.c_int64), ("node_hi", C.c_int64), ("records", C.c_int64)]


class NNError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libnn.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libnn.so not built ({LIB_PATH}); run __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            P = C.c_void_p
            L.nn_create.argtypes = [C.POINTER(P)]
            L.nn_create.restype = C.c_int
            L.nn_create_offline.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int32]
            L.nn_create_offline.restype = C.c_int
            L.nn_destroy.argtypes = [P]
            L.nn_destroy.restype = None
            L.nn_query.argtypes = [P, C.POINTER(NNMesh), C.c_int, C.POINTER(C.c_size_t),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.nn_query.restype = C.c_int
            for name in ("nn_neighbor_nodes", "nn_neighbor_elements"):
                f = getattr(L, name)
                f.argtypes = [P, C.POINTER(NNMesh), C.POINTER(NNCSR), P, C.c_size_t, P, P]
                f.restype = C.c_int
            L.nn_neighbors_both.argtypes = [P, C.POINTER(NNMesh), C.POINTER(NNCSR), C.POINTER(NNCSR), P,
                                            C.c_size_t, P, P]
            L.nn_neighbors_both.restype = C.c_int
            L.nn_profile_enable.argtypes = [P, C.c_int]
            L.nn_profile_enable.restype = C.c_int
            L.nn_profile_read.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]
            L.nn_profile_read.restype = C.c_int
            L.nn_element_neighbors_query.argtypes = [P, C.POINTER(NNMesh), C.POINTER(C.c_size_t),
                                                     C.POINTER(C.c_int64)]
            L.nn_element_neighbors_query.restype = C.c_int
            L.nn_element_neighbors.argtypes = [P, C.POINTER(NNMesh), C.POINTER(NNCSR), C.POINTER(NNCSR), P,
                                               C.c_size_t, P, P]
            L.nn_element_neighbors.restype = C.c_int
            L.nn_set_tuning.argtypes = [P, C.POINTER(NNTuning)]
            L.nn_set_tuning.restype = C.c_int
            L.nn_plan_info.argtypes = [P, C.POINTER(NNMesh), C.c_int, C.POINTER(C.c_int64), C.c_int]
            L.nn_plan_info.restype = C.c_int
            L.nn_neighbors_both_noalloc.argtypes = [C.POINTER(NNMesh), C.POINTER(NNCSR), C.POINTER(NNCSR), P, P]
            L.nn_neighbors_both_noalloc.restype = C.c_int
            L.nn_batch_query.argtypes = [P, C.POINTER(NNBatchCaps), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
            L.nn_batch_query.restype = C.c_int
            L.nn_batch_prepare.argtypes = [P, C.POINTER(NNBatchCaps), P, P, P, P, C.c_int, P, C.c_size_t]
            L.nn_batch_prepare.restype = C.c_int
            L.nn_batch_launch.argtypes = [P, C.POINTER(NNBatchCaps), P, P, C.c_size_t, P]
            L.nn_batch_launch.restype = C.c_int
            L.nn_generate_grid.argtypes = [C.c_int32, C.c_int64, C.c_uint64, C.c_int, C.c_int, P, C.c_int64,
                                           C.POINTER(C.c_int64), C.POINTER(C.c_int64), P]
            L.nn_generate_grid.restype = C.c_int
            L.nn_chunk_slabs.argtypes = [C.POINTER(NNMesh), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.nn_chunk_slabs.restype = C.c_int
            L.nn_chunk_count.argtypes = [P, C.POINTER(NNMesh), P, P, P]
            L.nn_chunk_count.restype = C.c_int
            L.nn_chunk_plan.argtypes = [P, C.POINTER(NNMesh), C.c_int, P, C.c_size_t, P, C.c_int,
                                        C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
            L.nn_chunk_plan.restype = C.c_int
            L.nn_chunk_query.argtypes = [P, C.POINTER(NNMesh), C.c_int, C.POINTER(NNChunk), C.POINTER(C.c_size_t)]
            L.nn_chunk_query.restype = C.c_int
            L.nn_neighbors_chunked.argtypes = [P, C.POINTER(NNMesh), C.c_int, P, C.c_int, C.POINTER(NNCSR),
                                               C.POINTER(NNCSR), P, C.c_size_t, P, P]
            L.nn_neighbors_chunked.restype = C.c_int
            L.nn_batch_submit_query.argtypes = [P, P, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
            L.nn_batch_submit_query.restype = C.c_int
            L.nn_batch_submit.argtypes = [P, P, P, P, C.c_int, P, C.c_size_t, P, P]
            L.nn_batch_submit.restype = C.c_int
            L.nn_diag_wait_timeout.argtypes = [P, P, P]
            L.nn_diag_wait_timeout.restype = C.c_int
            L.nn_status_str.argtypes = [C.c_int]
            L.nn_status_str.restype = C.c_char_p
            _lib = L
    return _lib


# ------------------------------------------------------------ C ABI mirrors

def nn_create() -> int:
    h = C.c_void_p()
    st = lib().nn_create(C.byref(h))
    if st:
        raise NNError(st, "nn_create")
    return h.value


GB300_LIMITS = (152, 232448, 233472)   # SMs, opt-in shared memory per block, shared memory per SM


def nn_create_offline(sms: int = GB300_LIMITS[0], smem_optin: int = GB300_LIMITS[1],
                      smem_per_sm: int = GB300_LIMITS[2]) -> int:
    """A sizing/planning-only handle for a described device (no GPU needed)."""
    h = C.c_void_p()
    st = lib().nn_create_offline(C.byref(h), sms, smem_optin, smem_per_sm)
    if st:
        raise NNError(st, "nn_create_offline")
    return h.value


def nn_destroy(h: int) -> None:
    lib().nn_destroy(h)


def nn_query(h: int, mesh: NNMesh, want: int):
    ws = C.c_size_t()
    nc = C.c_int64()
    ec = C.c_int64()
    st = lib().nn_query(h, C.byref(mesh), want, C.byref(ws), C.byref(nc), C.byref(ec))
    if st:
        raise NNError(st, "nn_query")
    return ws.value, nc.value, ec.value


PLAN_KEYS = ("sb", "n_buckets", "emit_ctas", "record_bytes", "ws_min", "bucket_ctas", "bucket_threads",
             "bucket_smem", "partition")


def nn_set_tuning(h: int, tuning: Optional[dict]) -> None:
    """Apply launch tuning {'sb', 'bucket_threads', 'bucket_ctas_per_sm'} (0 = automatic); None resets."""
    if tuning is None:
        st = lib().nn_set_tuning(h, None)
    else:
        t = NNTuning(int(tuning.get("sb", 0)), int(tuning.get("bucket_threads", 0)),
                     int(tuning.get("bucket_ctas_per_sm", 0)))
        st = lib().nn_set_tuning(h, C.byref(t))
    if st:
        raise NNError(st, "nn_set_tuning")


def nn_plan_info(h: int, mesh: NNMesh, want: int) -> dict:
    info = (C.c_int64 * 9)()
    st = lib().nn_plan_info(h, C.byref(mesh), want, info, 9)
    if st:
        raise NNError(st, "nn_plan_info")
    return dict(zip(PLAN_KEYS, list(info)))


def nn_neighbor_nodes(h, mesh: NNMesh, out: NNCSR, ws: int, ws_bytes: int, d_status: int, stream: int) -> int:
    return lib().nn_neighbor_nodes(h, C.byref(mesh), C.byref(out), ws, ws_bytes, d_status, stream)


def nn_neighbor_elements(h, mesh: NNMesh, out: NNCSR, ws: int, ws_bytes: int, d_status: int, stream: int) -> int:
    return lib().nn_neighbor_elements(h, C.byref(mesh), C.byref(out), ws, ws_bytes, d_status, stream)


def nn_neighbors_both(h, mesh: NNMesh, nodes: NNCSR, elems: NNCSR, ws: int, ws_bytes: int, d_status: int,
                      stream: int) -> int:
    return lib().nn_neighbors_both(h, C.byref(mesh), C.byref(nodes), C.byref(elems), ws, ws_bytes, d_status,
                                   stream)


def nn_element_neighbors_query(h: int, mesh: NNMesh):
    """(workspace bytes, col capacity bound) for element face adjacency."""
    ws = C.c_size_t()
    cap = C.c_int64()
    st = lib().nn_element_neighbors_query(h, C.byref(mesh), C.byref(ws), C.byref(cap))
    if st:
        raise NNError(st, "nn_element_neighbors_query")
    return ws.value, cap.value


def nn_element_neighbors(h, mesh: NNMesh, node_elems: NNCSR, out: NNCSR, ws: int, ws_bytes: int, d_status: int,
                         stream: int) -> int:
    return lib().nn_element_neighbors(h, C.byref(mesh), C.byref(node_elems), C.byref(out), ws, ws_bytes, d_status,
                                      stream)


CHUNK_SLABS_MAX = 4096


def nn_chunk_slabs(mesh: NNMesh):
    """(shift, n_slabs): node slabs of 2^shift ids for the chunked build (host only)."""
    sh = C.c_int()
    ns = C.c_int()
    st = lib().nn_chunk_slabs(C.byref(mesh), C.byref(sh), C.byref(ns))
    if st:
        raise NNError(st, "nn_chunk_slabs")
    return sh.value, ns.value


def nn_chunk_count(h: int, mesh: NNMesh, d_counts: int, d_status: int, stream: int) -> int:
    """Enqueue the per-slab incidence count into device uint32 d_counts[n_slabs]."""
    return lib().nn_chunk_count(h, C.byref(mesh), d_counts, d_status, stream)


def nn_chunk_plan(h: int, mesh: NNMesh, want: int, counts, ws_bytes: int, max_chunks: int = 4096):
    """Group slabs into chunks that fit ws_bytes (host only).  counts: sequence of
    per-slab incidence counts.  Returns (status, [(node_lo, node_hi, records)], ws_needed)."""
    arr = (C.c_uint32 * max(len(counts), 1))(*[int(c) for c in counts])
    out = (NNChunk * max(max_chunks, 1))()
    n = C.c_int()
    need = C.c_size_t()
    st = lib().nn_chunk_plan(h, C.byref(mesh), want, C.cast(arr, C.c_void_p), ws_bytes, C.cast(out, C.c_void_p),
                             max_chunks, C.byref(n), C.byref(need))
    chunks = [(out[i].node_lo, out[i].node_hi, out[i].records) for i in range(min(n.value, max_chunks))]
    return st, chunks, need.value


def nn_chunk_query(h: int, mesh: NNMesh, want: int, chunk) -> int:
    """Workspace bytes of one chunk (node_lo, node_hi, records) (host only)."""
    ws = C.c_size_t()
    st = lib().nn_chunk_query(h, C.byref(mesh), want, C.byref(NNChunk(*chunk)), C.byref(ws))
    if st:
        raise NNError(st, "nn_chunk_query")
    return ws.value


def nn_neighbors_chunked(h: int, mesh: NNMesh, want: int, chunks, nodes: Optional[NNCSR],
                         elems: Optional[NNCSR], ws: int, ws_bytes: int, d_status: int, stream: int) -> int:
    """Enqueue the chunked build; chunks: [(node_lo, node_hi, records)] tiling [0, n_nodes)."""
    arr = (NNChunk * max(len(chunks), 1))(*[NNChunk(*c) for c in chunks])
    return lib().nn_neighbors_chunked(h, C.byref(mesh), want, C.cast(arr, C.c_void_p), len(chunks),
                                      C.byref(nodes) if nodes is not None else None,
                                      C.byref(elems) if elems is not None else None, ws, ws_bytes, d_status,
                                      stream)


NOALLOC_SCRATCH_BYTES = 32 << 20


def nn_neighbors_both_noalloc(mesh: NNMesh, nodes: NNCSR, elems: NNCSR, d_status: int, stream: int) -> int:
    """Both CSRs with the library's fixed device scratch instead of a workspace (allocates nothing)."""
    return lib().nn_neighbors_both_noalloc(C.byref(mesh), C.byref(nodes), C.byref(elems), d_status, stream)


def nn_batch_submit_query(h: int, meshes, n: int, want: int) -> int:
    """Workspace bytes of a one-call batch of these meshes (an array of NNMesh)."""
    ws = C.c_size_t()
    st = lib().nn_batch_submit_query(h, meshes, n, want, C.byref(ws))
    if st:
        raise NNError(st, "nn_batch_submit_query")
    return ws.value


def nn_batch_submit(h: int, meshes, node_out, elem_out, n: int, ws: int, ws_bytes: int, d_status: int,
                    stream: int) -> int:
    """One-call batch: arrays of NNMesh and NNCSR (either output array may be None)."""
    return lib().nn_batch_submit(h, meshes, node_out, elem_out, n, ws, ws_bytes, d_status, stream)


def nn_diag_wait_timeout(d_state: int, d_status: int, stream: int) -> int:
    """Run one bounded lookback wait whose predecessor never publishes (see include/nn.h)."""
    return lib().nn_diag_wait_timeout(d_state, d_status, stream)


def nn_batch_query(h: int, caps: NNBatchCaps):
    ws = C.c_size_t()
    sg = C.c_size_t()
    st = lib().nn_batch_query(h, C.byref(caps), C.byref(ws), C.byref(sg))
    if st:
        raise NNError(st, "nn_batch_query")
    return ws.value, sg.value


def nn_batch_prepare(h: int, caps: NNBatchCaps, meshes, node_out, elem_out, d_status: int, n: int,
                     staging: int, staging_bytes: int) -> int:
    """meshes / node_out / elem_out: ctypes arrays of NNMesh / NNCSR (or None)."""
    return lib().nn_batch_prepare(h, C.byref(caps), C.cast(meshes, C.c_void_p) if meshes is not None else None,
                                  C.cast(node_out, C.c_void_p) if node_out is not None else None,
                                  C.cast(elem_out, C.c_void_p) if elem_out is not None else None,
                                  d_status, n, staging, staging_bytes)


def nn_batch_launch(h: int, caps: NNBatchCaps, staging: int, ws: int, ws_bytes: int, stream: int) -> int:
    return lib().nn_batch_launch(h, C.byref(caps), staging, ws, ws_bytes, stream)


def nn_generate_grid(etype: int, n: int, seed: int, permute_nodes: bool, permute_elems: bool, conn: int,
                     capacity: int, stream: int):
    """Generate a seeded grid mesh into device memory; returns (status, n_nodes, n_elems)."""
    nn_ = C.c_int64()
    ne = C.c_int64()
    st = lib().nn_generate_grid(etype, n, seed & ((1 << 64) - 1), int(permute_nodes), int(permute_elems), conn,
                                capacity, C.byref(nn_), C.byref(ne), stream)
    return st, nn_.value, ne.value


def generate_grid(etype: int, n: int, seed: int, permute_nodes: bool = True, permute_elems=None, device=None,
                  stream=None) -> "DeviceMesh":
    """A DeviceMesh generated on the device (same mesh as meshgen's tri/quad/tet/hex_grid)."""
    import torch
    if permute_elems is None:
        permute_elems = etype != HEX            # meshgen's defaults
    st, N, T = nn_generate_grid(etype, n, seed, permute_nodes, permute_elems, None, 0, 0)
    if st:
        raise NNError(st, "nn_generate_grid")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    conn = torch.empty(T * NPE[etype], dtype=torch.int32, device=dev)
    s = (stream or torch.cuda.current_stream(dev)).cuda_stream
    st, _, _ = nn_generate_grid(etype, n, seed, permute_nodes, permute_elems, conn.data_ptr() if T else None,
                                conn.numel(), s)
    if st:
        raise NNError(st, "nn_generate_grid")
    return DeviceMesh(etype, N, conn)


STAGES = ("init", "hist", "offsets", "part", "part_fine", "bucket", "place")


def nn_profile_enable(h: int, enable: bool) -> None:
    st = lib().nn_profile_enable(h, int(enable))
    if st:
        raise NNError(st, "nn_profile_enable")


def nn_profile_read(h: int):
    """({stage: summed ms}, calls) since profiling was enabled."""
    ms = (C.c_double * len(STAGES))()
    calls = C.c_int64()
    st = lib().nn_profile_read(h, ms, C.byref(calls), len(STAGES))
    if st:
        raise NNError(st, "nn_profile_read")
    return dict(zip(STAGES, list(ms))), calls.value


def nn_status_str(code: int) -> str:
    return lib().nn_status_str(code).decode()


# -------------------------------------------------------------- high level

@dataclass
class DeviceMesh:
    """Connectivity resident on the device (torch tensors)."""
    etype: int
    n_nodes: int
    conn: "torch.Tensor"                        # int32, 16-byte aligned
    elem_ptr: Optional["torch.Tensor"] = None   # int64, MIXED only
    elem_type: Optional["torch.Tensor"] = None  # uint8, MIXED only

    @property
    def n_conn(self) -> int:
        return int(self.conn.numel())

    @property
    def n_elems(self) -> int:
        if self.etype == MIXED:
            return int(self.elem_type.numel())
        return self.n_conn // NPE[self.etype]

    def struct(self) -> NNMesh:
        def ptr(t):
            return t.data_ptr() if t is not None and t.numel() else None
        return NNMesh(self.etype, self.n_nodes, self.n_elems, self.n_conn, ptr(self.conn), ptr(self.elem_ptr),
                      ptr(self.elem_type))

    @staticmethod
    def from_host(mesh, device="cuda", pin: bool = False) -> "DeviceMesh":
        """Copy a host mesh (e.g. meshgen.Mesh) to the device."""
        import torch

        def to(a):
            if a is None:
                return None
            t = torch.from_numpy(a)
            if pin:
                t = t.pin_memory()
            return t.to(device, non_blocking=pin)
        return DeviceMesh(int(mesh.etype), int(mesh.n_nodes), to(mesh.conn), to(mesh.elem_ptr), to(mesh.elem_type))


class Builder:
    """Owns a handle, a workspace and output buffers; rebuilds on demand."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.h = nn_create()
        self.ws = None
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def close(self):
        if self.h:
            nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, dm: DeviceMesh, want: int):
        return nn_query(self.h, dm.struct(), want)

    def workspace(self, nbytes: int):
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = self.torch.empty(max(nbytes, 256), dtype=self.torch.uint8, device=self.device)
        return self.ws

    def alloc_outputs(self, dm: DeviceMesh, want: int, node_cap=None, elem_cap=None):
        torch = self.torch
        _, nc, ec = self.query(dm, want)
        out = {}
        if want & WANT_NODES:
            out["nodes"] = (torch.empty(dm.n_nodes + 1, dtype=torch.int64, device=self.device),
                            torch.empty(max(nc if node_cap is None else node_cap, 1), dtype=torch.int32,
                                        device=self.device))
        if want & WANT_ELEMS:
            out["elems"] = (torch.empty(dm.n_nodes + 1, dtype=torch.int64, device=self.device),
                            torch.empty(max(ec if elem_cap is None else elem_cap, 1), dtype=torch.int32,
                                        device=self.device))
        return out

    def launch(self, dm: DeviceMesh, want: int, out: dict, ws=None, ws_bytes=None, stream=None, status=None) -> int:
        """Enqueue one build (no sync).  Returns the host status code.  ``status``: a device int32
        tensor to receive the device status instead of the builder's own."""
        torch = self.torch
        if ws is None:
            nbytes, _, _ = self.query(dm, want)
            ws = self.workspace(nbytes)
            ws_bytes = nbytes
        elif ws_bytes is None:   # a caller's workspace: all of it (one contiguous span from data_ptr())
            if not ws.is_contiguous():
                raise ValueError("a workspace given without ws_bytes must be contiguous")
            ws_bytes = ws.numel() * ws.element_size()
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        mesh = dm.struct()

        def csr(pair):
            rp, col = pair
            return NNCSR(rp.data_ptr(), col.data_ptr(), col.numel())
        sp = (status if status is not None else self.status).data_ptr()
        if want == WANT_NODES:
            return nn_neighbor_nodes(self.h, mesh, csr(out["nodes"]), ws.data_ptr(), ws_bytes, sp, s)
        if want == WANT_ELEMS:
            return nn_neighbor_elements(self.h, mesh, csr(out["elems"]), ws.data_ptr(), ws_bytes, sp, s)
        return nn_neighbors_both(self.h, mesh, csr(out["nodes"]), csr(out["elems"]), ws.data_ptr(), ws_bytes, sp, s)

    def element_neighbors(self, dm: DeviceMesh, node_elems, stream=None, sync: bool = True):
        """Face neighbours of every element: (row_ptr, col) on the device, from
        the mesh's node -> element CSR ``node_elems`` = (row_ptr, col).  With
        ``sync``, waits, checks the device status and trims col."""
        torch = self.torch
        ws_bytes, cap = nn_element_neighbors_query(self.h, dm.struct())
        ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=self.device)
        rp = torch.empty(dm.n_elems + 1, dtype=torch.int64, device=self.device)
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        ne_rp, ne_col = node_elems
        for attempt in range(2):
            col = torch.empty(max(cap, 1), dtype=torch.int32, device=self.device)
            st = nn_element_neighbors(self.h, dm.struct(),
                                      NNCSR(ne_rp.data_ptr(), ne_col.data_ptr(), ne_col.numel()),
                                      NNCSR(rp.data_ptr(), col.data_ptr(), col.numel()), ws.data_ptr(), ws_bytes,
                                      self.status.data_ptr(), s)
            if st:
                raise NNError(st, "nn_element_neighbors")
            self._adj_keep = ws
            if not sync:
                return rp, col
            torch.cuda.synchronize(self.device)
            status = int(self.status.item())
            if status == 3 and attempt == 0:   # faces shared by many elements: the exact size is in rp[-1]
                cap = int(rp[-1].item())
                continue
            if status:
                raise NNError(status, "nn_element_neighbors (device)")
            break
        return rp, col[: int(rp[-1].item())]

    def plan_chunks(self, dm: DeviceMesh, want: int, ws_bytes: int, stream=None):
        """Count incidences per node slab on the device, wait for them, and
        group the slabs into chunks whose workspace fits ws_bytes.  Returns
        the chunk list [(node_lo, node_hi, records)]."""
        torch = self.torch
        mesh = dm.struct()
        _, ns = nn_chunk_slabs(mesh)
        counts = torch.zeros(max(ns, 1), dtype=torch.int32, device=self.device)
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        st = nn_chunk_count(self.h, mesh, counts.data_ptr(), self.status.data_ptr(), s)
        if st:
            raise NNError(st, "nn_chunk_count")
        torch.cuda.synchronize(self.device)
        if int(self.status.item()):
            raise NNError(int(self.status.item()), "nn_chunk_count (device)")
        host = [c & 0xFFFFFFFF for c in counts[:ns].cpu().tolist()]
        st, chunks, need = nn_chunk_plan(self.h, mesh, want, host, ws_bytes)
        if st:
            raise NNError(st, f"nn_chunk_plan (smallest workspace {need} bytes)")
        return chunks

    def launch_chunked(self, dm: DeviceMesh, want: int, out: dict, chunks, ws, ws_bytes: int, stream=None,
                       status=None) -> int:
        """Enqueue a chunked build (no sync); returns the host status code."""
        torch = self.torch
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream

        def csr(key):
            if key not in out:
                return None
            rp, col = out[key]
            return NNCSR(rp.data_ptr(), col.data_ptr(), col.numel())
        sp = (status if status is not None else self.status).data_ptr()
        return nn_neighbors_chunked(self.h, dm.struct(), want, chunks, csr("nodes"), csr("elems"), ws.data_ptr(),
                                    ws_bytes, sp, s)

    def build_chunked(self, dm: DeviceMesh, want: int = WANT_BOTH, ws_bytes: int = 1 << 30):
        """Like build, with the workspace capped at ws_bytes: nodes are built in
        chunks of consecutive ids, each fitting the workspace."""
        chunks = self.plan_chunks(dm, want, ws_bytes)
        ws = self.torch.empty(max(ws_bytes, 256), dtype=self.torch.uint8, device=self.device)
        out = self.alloc_outputs(dm, want)
        st = self.launch_chunked(dm, want, out, chunks, ws, ws_bytes)
        if st:
            raise NNError(st, "nn_neighbors_chunked")
        self.torch.cuda.synchronize(self.device)
        res = {"status": int(self.status.item()), "chunks": chunks}
        for k, (rp, col) in out.items():
            nnz = int(rp[-1].item()) if res["status"] == 0 else col.numel()
            res[k] = (rp, col[:nnz])
        return res

    def build(self, dm: DeviceMesh, want: int = WANT_BOTH):
        """Build and return {'status': int, 'nodes': (row_ptr, col), 'elems': (row_ptr, col)} (col trimmed)."""
        out = self.alloc_outputs(dm, want)
        st = self.launch(dm, want, out)
        if st:
            raise NNError(st, "launch")
        self.torch.cuda.synchronize(self.device)
        res = {"status": int(self.status.item())}
        for k, (rp, col) in out.items():
            nnz = int(rp[-1].item()) if res["status"] == 0 else col.numel()
            res[k] = (rp, col[:nnz])
        return res


class BatchBuilder:
    """Batched builds: one launch sequence for many meshes (capacity fixed at creation).

    ``prepare`` writes a batch into pinned host staging (host only); ``launch``
    enqueues it.  ``launch`` may be captured once in a CUDA graph and the graph
    replayed after each ``prepare``."""

    def __init__(self, max_meshes: int, max_elems: int, max_nodes: int, max_conn: int, want: int = WANT_BOTH,
                 sb: int = 0, device=None, handle=None, extra_ws: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.own = handle is None
        with torch.cuda.device(self.device):
            self.h = handle if handle is not None else nn_create()
        self.caps = NNBatchCaps(max_meshes, want, max_elems, max_nodes, max_conn, sb)
        self.ws_bytes, self.staging_bytes = nn_batch_query(self.h, self.caps)
        self.ws_bytes += extra_ws
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.staging = torch.empty(self.staging_bytes, dtype=torch.uint8, pin_memory=True)
        self.status = torch.zeros(max_meshes, dtype=torch.int32, device=self.device)
        self.want = want

    def close(self):
        if self.own and self.h:
            nn_destroy(self.h)
        self.h = None

    def alloc_outputs(self, dm: DeviceMesh):
        torch = self.torch
        nc = (2 if dm.etype in (TRI, QUAD) else 3) * dm.n_conn
        out = {}
        if self.want & WANT_NODES:
            out["nodes"] = (torch.empty(dm.n_nodes + 1, dtype=torch.int64, device=self.device),
                            torch.empty(max(nc, 1), dtype=torch.int32, device=self.device))
        if self.want & WANT_ELEMS:
            out["elems"] = (torch.empty(dm.n_nodes + 1, dtype=torch.int64, device=self.device),
                            torch.empty(max(dm.n_conn, 1), dtype=torch.int32, device=self.device))
        return out

    def prepare(self, dmeshes, outs) -> int:
        n = len(dmeshes)
        M = (NNMesh * max(n, 1))(*[d.struct() for d in dmeshes])

        def csrs(key):
            if not (self.want & (WANT_NODES if key == "nodes" else WANT_ELEMS)):
                return None
            return (NNCSR * max(n, 1))(*[NNCSR(o[key][0].data_ptr(), o[key][1].data_ptr(), o[key][1].numel())
                                          for o in outs])
        self._keep = (M, csrs("nodes"), csrs("elems"))
        return nn_batch_prepare(self.h, self.caps, M, self._keep[1], self._keep[2], self.status.data_ptr(), n,
                                self.staging.data_ptr(), self.staging_bytes)

    def launch(self, stream=None) -> int:
        s = (stream or self.torch.cuda.current_stream(self.device)).cuda_stream
        return nn_batch_launch(self.h, self.caps, self.staging.data_ptr(), self.ws.data_ptr(), self.ws_bytes, s)

    def run(self, dmeshes):
        """Build a batch, wait, and return per-mesh results (col trimmed) and statuses."""
        outs = [self.alloc_outputs(d) for d in dmeshes]
        st = self.prepare(dmeshes, outs)
        if st:
            raise NNError(st, "nn_batch_prepare")
        st = self.launch()
        if st:
            raise NNError(st, "nn_batch_launch")
        self.torch.cuda.synchronize(self.device)
        stat = self.status[: len(dmeshes)].cpu().tolist()
        res = []
        for o, s_ in zip(outs, stat):
            r = {"status": int(s_)}
            for k, (rp, col) in o.items():
                r[k] = (rp, col[: int(rp[-1].item())] if s_ == 0 else col)
            res.append(r)
        return res
