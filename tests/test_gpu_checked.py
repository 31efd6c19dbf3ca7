"""The bounds-checked build, libnn_checked.so (compiled with -DNN_CHECKED).

In it every computed global index of the build's kernels (histogram,
partition passes, bucket pass, node-row placement) is tested against its
buffer's length; a violation would record NN_ERR_BOUNDS in the device status
and skip the access, never trap.  Here it builds the small-mesh parity set
-- every element type, mixed, holes, degenerate elements, a fan of high
valence -- through the C ABI into buffers followed by canary words: the
results equal the oracle's, the status stays NN_OK (no index left its
buffer), and every canary after the outputs and after the workspace is
intact."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn

pytestmark = pytest.mark.gpu

CANARY = 0x5A5A5A5A
TAIL = 64  # canary words after each buffer


@pytest.fixture(scope="module")
def lib():
    from paper_1604_04689_gb300 import build
    path = build.build(checked=True)
    L = C.CDLL(path)
    P = C.c_void_p
    L.nn_create.argtypes = [C.POINTER(P)]
    L.nn_destroy.argtypes = [P]
    L.nn_query.argtypes = [P, P, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.nn_neighbors_both.argtypes = [P, P, P, P, P, C.c_size_t, P, P]
    return L


def fan(n_tris):
    """A triangle fan around node 0: node 0 has n_tris triangles."""
    conn = np.zeros((n_tris, 3), dtype=np.int32)
    conn[:, 1] = 1 + np.arange(n_tris)
    conn[:, 2] = 1 + (np.arange(n_tris) + 1) % n_tris
    return mg.Mesh(mg.TRI, n_tris + 1, conn.reshape(-1), name="fan")


MESHES = {
    "tri64": lambda: mg.tri_grid(64, 51),
    "tri_holes": lambda: mg.tri_grid(90, 52, holes=0.05),
    "quad40": lambda: mg.quad_grid(40, 53),
    "tet15": lambda: mg.tet_grid(15, 54),
    "hex21": lambda: mg.hex_grid(21, 55),
    "mixed13": lambda: mg.mixed_grid(13, 56),
    "fan": lambda: fan(3000),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_checked_build_matches_oracle_with_canaries_intact(lib, name):
    import torch
    mesh = MESHES[name]()
    dm = nn.DeviceMesh.from_host(mesh)
    h = C.c_void_p()
    assert lib.nn_create(C.byref(h)) == 0
    try:
        ms = dm.struct()
        ws_bytes, ncap, ecap = C.c_size_t(), C.c_int64(), C.c_int64()
        assert lib.nn_query(h, C.byref(ms), nn.WANT_BOTH, C.byref(ws_bytes), C.byref(ncap), C.byref(ecap)) == 0
        N = mesh.n_nodes

        def canaried(n, dtype):
            t = torch.empty(n + TAIL * (2 if dtype == torch.int32 else 1), dtype=dtype, device="cuda")
            t.view(torch.int32).fill_(CANARY)
            return t
        rp_n, rp_e = canaried(N + 1, torch.int64), canaried(N + 1, torch.int64)
        col_n, col_e = canaried(ncap.value, torch.int32), canaried(ecap.value, torch.int32)
        ws = torch.empty(ws_bytes.value + 4 * TAIL, dtype=torch.uint8, device="cuda")
        ws.view(torch.int32).fill_(CANARY)
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        nodes = nn.NNCSR(rp_n.data_ptr(), col_n.data_ptr(), ncap.value)
        elems = nn.NNCSR(rp_e.data_ptr(), col_e.data_ptr(), ecap.value)
        stream = torch.cuda.current_stream().cuda_stream
        assert lib.nn_neighbors_both(h, C.byref(ms), C.byref(nodes), C.byref(elems), ws.data_ptr(), ws_bytes.value,
                                     status.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0, nn.STATUS.get(int(status.item()))
        ref = oracle.neighbors(mesh, oracle.BOTH)
        for key, rp, col in (("nodes", rp_n, col_n), ("elems", rp_e, col_e)):
            r = rp[: N + 1].cpu().numpy()
            np.testing.assert_array_equal(r, ref[key][0], err_msg=f"{key} row_ptr")
            np.testing.assert_array_equal(col.cpu().numpy()[: r[-1]], ref[key][1], err_msg=f"{key} col")
        for what, t, n in (("node row_ptr", rp_n, N + 1), ("element row_ptr", rp_e, N + 1),
                           ("node col", col_n, ncap.value), ("element col", col_e, ecap.value)):
            tail = t[n:].view(torch.int32).cpu().numpy()
            assert (tail == CANARY).all(), f"{what}: canary overwritten"
        tail = ws[ws_bytes.value:].view(torch.int32).cpu().numpy()
        assert (tail == CANARY).all(), "workspace canary overwritten"
    finally:
        lib.nn_destroy(h)
