"""The replica path of bench.py on two gloo ranks (CPU): the timed region's
maximum over ranks and the whole-job value computed from it."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (t, bench.whole_job_value(1000, 5, world, t))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_max_over_ranks_and_value_two_gloo_ranks():
    world, port = 2, _free_port()
    times = [12.5, 20.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    assert res[0][1] == pytest.approx(2 * 1000 * 5 / 20e-3 / 1e6)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_value(2_000_000, 10, 1, 1000.0) == pytest.approx(20.0)
