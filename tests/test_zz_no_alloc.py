"""The allocation-free entry point, nn_neighbors_both_noalloc.

It exists for callers that may not allocate device memory (an application
that owns all device memory through its own pool, or a loop that must never
enter the CUDA allocator): the build uses a fixed scratch array that the
library keeps in device memory instead of a caller workspace.  Here it is
called through the C ABI twice in a row and checked, bit for bit, against the
existing entry point nn_neighbors_both on the same mesh.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


def _outputs(torch, b, dm):
    return b.alloc_outputs(dm, nn.WANT_BOTH)


def _csr(pair):
    rp, col = pair
    return nn.NNCSR(rp.data_ptr(), col.data_ptr(), col.numel())


def _host(torch, out):
    res = {}
    for k, (rp, col) in out.items():
        rp = rp.cpu().numpy()
        res[k] = (rp, col.cpu().numpy()[: rp[-1]])
    return res


@pytest.mark.parametrize("mesh_fn", [lambda: mg.tet_grid(30, 21), lambda: mg.mixed_grid(25, 22),
                                     lambda: mg.tri_grid(400, 23, holes=0.05)],
                         ids=["tet30", "mixed25", "tri400_holes"])
def test_noalloc_matches_workspace_entry_point(mesh_fn):
    import torch
    mesh = mesh_fn()
    b = nn.Builder()
    dm = nn.DeviceMesh.from_host(mesh)
    stream = torch.cuda.current_stream().cuda_stream

    ref_out = _outputs(torch, b, dm)
    assert b.launch(dm, nn.WANT_BOTH, ref_out) == 0           # existing entry point, caller workspace
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    ref = _host(torch, ref_out)

    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    outs = [_outputs(torch, b, dm) for _ in range(2)]
    torch.cuda.synchronize()
    free_before = None
    for call in range(2):                                        # two calls in a row share the scratch
        out = outs[call]
        for rp, col in out.values():                             # poison the outputs
            rp.fill_(-7)
            col.fill_(-7)
        st = nn.nn_neighbors_both_noalloc(dm.struct(), _csr(out["nodes"]), _csr(out["elems"]),
                                          status.data_ptr(), stream)
        assert st == 0, nn.STATUS.get(st, st)
        torch.cuda.synchronize()
        # the first call of the process may load the library's code and with
        # it the scratch array itself (lazy module loading); from then on a
        # call takes no device memory
        free_now = torch.cuda.mem_get_info()[0]
        if free_before is not None:
            assert free_now == free_before, f"call {call} took {free_before - free_now} bytes of device memory"
        free_before = free_now
        assert int(status.item()) == 0, f"call {call}: device status {int(status.item())}"
        got = _host(torch, out)
        for k in ("nodes", "elems"):
            np.testing.assert_array_equal(got[k][0], ref[k][0], err_msg=f"call {call} {k} row_ptr")
            np.testing.assert_array_equal(got[k][1], ref[k][1], err_msg=f"call {call} {k} col")


def test_noalloc_rejects_meshes_beyond_the_scratch():
    import torch
    mesh = mg.tet_grid(81, 1)                                    # ~12.3M incidences: needs ~200 MB of scratch
    dm = nn.DeviceMesh.from_host(mesh)
    b = nn.Builder()
    out = b.alloc_outputs(dm, nn.WANT_BOTH)
    status = torch.full((1,), -9, dtype=torch.int32, device="cuda")  # poisoned: a call that enqueued would clear it
    for rp, _ in out.values():
        rp.fill_(-7)
    torch.cuda.synchronize()
    st = nn.nn_neighbors_both_noalloc(dm.struct(), _csr(out["nodes"]), _csr(out["elems"]), status.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert st == 2                                               # NN_ERR_WORKSPACE, nothing enqueued
    torch.cuda.synchronize()
    assert int(status.item()) == -9
    for rp, _ in out.values():
        assert bool((rp == -7).all())
