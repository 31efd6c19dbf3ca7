"""Failure detection without a GPU fault: the bounded wait of the single-pass
scans gives up when its predecessor never publishes, reports NN_ERR_TIMEOUT
on the device status word, publishes its own tile, and leaves the context
usable (a build right after it equals the oracle)."""
import pytest

from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn
from tests.gpu_util import check_against_oracle

pytestmark = pytest.mark.gpu

LB_INC = 2 << 62
LB_VAL = (1 << 62) - 1
M64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_04689_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def test_wait_without_predecessor_times_out_and_context_survives():
    import torch
    state = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert nn.nn_diag_wait_timeout(state.data_ptr(), status.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 6 == [k for k, v in nn.STATUS.items() if v == "NN_ERR_TIMEOUT"][0]
    s = [x & M64 for x in state.cpu().tolist()]
    assert s[0] == 0                                 # the predecessor never published
    assert (s[1] & ~LB_VAL & M64) == LB_INC          # the probed tile published an inclusive prefix
    assert (s[1] & LB_VAL) == 1                      # its own aggregate, nothing from the missing tile
    assert 1.9e9 <= s[2] <= 20e9                     # gave up after the ~2 s limit, not at once
    # the context still works: an ordinary build right after equals the oracle
    check_against_oracle(mg.tri_grid(40, 21), nn.WANT_BOTH)

