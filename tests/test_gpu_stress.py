"""Repeated builds with 8-byte records, each compared with the oracle.

A record is 8 bytes when its fields fit 64 bits: element rows alone on
mid-size meshes, node rows of triangles, or both results on small meshes.
Tets and mixed meshes then take the lanes' hash-table path for their
neighbour rows.  Each case builds 20 times in one process (reusing the
workspace and outputs, poisoned before every build) and every result must
equal the oracle's bit for bit: rows are sets (Sec. 2.1.1), so one extra or
missing neighbour in any build fails."""
import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn

pytestmark = pytest.mark.gpu

CASES = {
    "tet41_elems": (lambda: mg.tet_grid(41, 31), nn.WANT_ELEMS),
    "mixed41_elems": (lambda: mg.mixed_grid(41, 32), nn.WANT_ELEMS),
    "tet11_both": (lambda: mg.tet_grid(11, 33), nn.WANT_BOTH),
    "mixed9_both": (lambda: mg.mixed_grid(9, 34), nn.WANT_BOTH),
    "tri400_nodes": (lambda: mg.tri_grid(400, 35, holes=0.02), nn.WANT_NODES),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


@pytest.mark.parametrize("name", list(CASES))
def test_eight_byte_records_twenty_builds(name):
    import torch
    make, want = CASES[name]
    mesh = make()
    ref = oracle.neighbors(mesh, want)
    b = nn.Builder()
    dm = nn.DeviceMesh.from_host(mesh)
    assert nn.nn_plan_info(b.h, dm.struct(), want)["record_bytes"] == 8, "the case must use 8-byte records"
    ws_bytes = b.query(dm, want)[0]
    ws = b.workspace(ws_bytes)
    out = b.alloc_outputs(dm, want)
    for it in range(20):
        for rp, col in out.values():
            rp.fill_(-1)
            col.fill_(-1)
        assert b.launch(dm, want, out, ws=ws, ws_bytes=ws_bytes) == 0
        torch.cuda.synchronize()
        assert int(b.status.item()) == 0, f"build {it}: {nn.STATUS[int(b.status.item())]}"
        for key, (rp, col) in out.items():
            rp = rp.cpu().numpy()
            np.testing.assert_array_equal(rp, ref[key][0], err_msg=f"build {it} {key} row_ptr")
            np.testing.assert_array_equal(col.cpu().numpy()[: rp[-1]], ref[key][1], err_msg=f"build {it} {key} col")
