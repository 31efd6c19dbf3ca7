"""Autotuned launches give the same CSR bit for bit as the automatic plan, on
every element type, for every candidate tuning; the tuner caches and reapplies
its choice."""
import numpy as np
import pytest

import oracle
from paper_1604_04689_gb300 import autotune as at
from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn

pytestmark = pytest.mark.gpu

MESHES = {
    "tri300": lambda: mg.tri_grid(300, 21, holes=0.03),
    "tet41": lambda: mg.tet_grid(41, 22),
    "hex61": lambda: mg.hex_grid(61, 23),
    "mixed41": lambda: mg.mixed_grid(41, 24),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()


def host(out):
    return {k: (rp.cpu().numpy(), col.cpu().numpy()[: int(rp[-1].item())]) for k, (rp, col) in out.items()}


@pytest.mark.parametrize("name", list(MESHES))
def test_every_candidate_matches_oracle(name):
    import torch
    mesh = MESHES[name]()
    ref = oracle.neighbors(mesh, nn.WANT_BOTH)
    b = nn.Builder()
    dm = nn.DeviceMesh.from_host(mesh)
    cands = at.candidates(b, dm, nn.WANT_BOTH)
    assert len(cands) >= 4
    seen = []

    def verify(out):
        got = host(out)
        for k in ("nodes", "elems"):
            np.testing.assert_array_equal(got[k][0], ref[k][0], err_msg=f"{name} {k} row_ptr")
            np.testing.assert_array_equal(got[k][1], ref[k][1], err_msg=f"{name} {k} col")
        seen.append(1)

    best, results = at.tune(b, dm, nn.WANT_BOTH, reps=1, cands=cands, verify=verify)
    assert len(seen) == len(cands) == len(results)
    assert best in cands
    torch.cuda.synchronize()


def test_tuned_caches_and_reapplies(tmp_path):
    mesh = MESHES["tet41"]()
    path = str(tmp_path / "tune.json")
    b = nn.Builder()
    dm = nn.DeviceMesh.from_host(mesh)
    best = at.tuned(b, dm, nn.WANT_BOTH, path=path)
    cache = at.load_cache(path)
    assert len(cache) == 1 and list(cache.values())[0]["tuning"] == best
    b2 = nn.Builder()
    assert at.tuned(b2, dm, nn.WANT_BOTH, path=path) == best
    plan1 = nn.nn_plan_info(b.h, dm.struct(), nn.WANT_BOTH)
    plan2 = nn.nn_plan_info(b2.h, dm.struct(), nn.WANT_BOTH)
    assert plan1 == plan2


def test_invalid_tunings_rejected():
    b = nn.Builder()
    for t in ({"sb": 3}, {"sb": 12}, {"bucket_threads": 512}, {"bucket_threads": 64}, {"bucket_ctas_per_sm": 9},
              {"bucket_ctas_per_sm": -1}):
        with pytest.raises(nn.NNError):
            nn.nn_set_tuning(b.h, t)
    nn.nn_set_tuning(b.h, None)
