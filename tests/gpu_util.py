"""Helpers for the GPU parity tests: run a build through the C ABI and compare
it with the CPU oracle element by element."""
import os

import numpy as np

import oracle
from paper_1604_04689_gb300 import nn

KEYS = {nn.WANT_NODES: ("nodes",), nn.WANT_ELEMS: ("elems",), nn.WANT_BOTH: ("nodes", "elems")}


def gpu_build(mesh, want=nn.WANT_BOTH, builder=None, ws_extra=0, **kw):
    """Build through the C ABI; ws_extra adds bytes to the recommended workspace."""
    b = builder or nn.Builder()
    dm = nn.DeviceMesh.from_host(mesh)
    out = b.alloc_outputs(dm, want, **kw)
    ws = ws_bytes = None
    if ws_extra:
        ws_bytes = b.query(dm, want)[0] + ws_extra
        ws = b.workspace(ws_bytes)
    st = b.launch(dm, want, out, ws=ws, ws_bytes=ws_bytes)
    assert st == 0, nn.STATUS.get(st, st)
    import torch
    torch.cuda.synchronize()
    status = int(b.status.item())
    res = {"status": status}
    for k, (rp, col) in out.items():
        rp = rp.cpu().numpy()
        res[k] = (rp, col.cpu().numpy()[: rp[-1]] if status == 0 else col.cpu().numpy())
    return res


def assert_same(res, ref, want=nn.WANT_BOTH):
    assert res["status"] == ref["status"] == 0, (res["status"], ref["status"])
    for k in KEYS[want]:
        np.testing.assert_array_equal(res[k][0], ref[k][0], err_msg=f"{k} row_ptr")
        np.testing.assert_array_equal(res[k][1], ref[k][1], err_msg=f"{k} col")


def check_against_oracle(mesh, want=nn.WANT_BOTH, builder=None, ws_extra=0):
    res = gpu_build(mesh, want, builder, ws_extra=ws_extra)
    ref = oracle.neighbors(mesh, want)
    assert_same(res, ref, want)
    return res


class env:
    """Temporarily set environment variables read by nn_create."""

    def __init__(self, **kv):
        self.kv = {k: str(v) for k, v in kv.items()}
        self.old = {}

    def __enter__(self):
        for k, v in self.kv.items():
            self.old[k] = os.environ.get(k)
            os.environ[k] = v
        return self

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
