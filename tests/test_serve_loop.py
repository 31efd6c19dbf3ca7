"""The serving loops' host logic on the CPU: BatchServer and PlainServer run
their real event loops against fake CUDA streams, events and builders (each
"GPU" unit completes a fixed time after it is enqueued behind the stream's
earlier work), so admission, the in-flight depth, completion bookkeeping,
rejection of oversized requests and the statistics are checked without a
GPU; and a stream that never completes trips the host watchdog instead of
spinning forever."""
import contextlib
import time

import pytest
import torch

from paper_1604_04689_gb300 import meshgen as mg
from paper_1604_04689_gb300 import nn, serve
from paper_1604_04689_gb300.serve import BatchServer, LaneCaps, PlainServer, Request

GPU_S = 0.002        # simulated device time of one enqueued batch or build


class FakeStream:
    hang = False     # set on the class by a test: nothing recorded on any stream ever completes

    def __init__(self, device=None):
        self.cuda_stream = 0
        self.busy_until = 0.0

    def enqueue(self):
        self.busy_until = max(self.busy_until, time.perf_counter()) + GPU_S

    def wait_event(self, ev):
        if ev.t is not None:
            self.busy_until = max(self.busy_until, ev.t)


class FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        s = stream if stream is not None else _DEFAULT
        self.t = float("inf") if FakeStream.hang and s is not _DEFAULT else max(s.busy_until, time.perf_counter())

    def query(self):
        return self.t is not None and time.perf_counter() >= self.t

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


_DEFAULT = FakeStream()


class FakeBatchBuilder:
    launches = 0

    def __init__(self, max_meshes, max_elems, max_nodes, max_conn, want=nn.WANT_BOTH, device=None, **kw):
        self.ws_bytes = 1 << 20
        self.status = torch.zeros(max_meshes, dtype=torch.int32)
        self.n = 0

    def prepare(self, dmeshes, outs):
        self.n = len(dmeshes)
        return 0

    def launch(self, stream):
        FakeBatchBuilder.launches += 1
        stream.enqueue()
        return 0


class FakeBuilder:
    launches = 0

    def __init__(self, device=None):
        pass

    def query(self, dm, want):
        return 1 << 20, 0, 0

    def workspace(self, nbytes):
        return torch.empty(16, dtype=torch.uint8)

    def launch(self, dm, want, out, ws=None, ws_bytes=None, stream=None, status=None):
        FakeBuilder.launches += 1
        stream.enqueue()
        return 0


def fake_generate_grid(etype, n, seed, permute_nodes=True, permute_elems=None, device=None, stream=None):
    return nn.DeviceMesh(etype, 0, torch.zeros(0, dtype=torch.int32))


@pytest.fixture
def fake_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: _DEFAULT)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda device=None: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(nn, "BatchBuilder", FakeBatchBuilder)
    monkeypatch.setattr(nn, "Builder", FakeBuilder)
    monkeypatch.setattr(nn, "generate_grid", fake_generate_grid)
    FakeStream.hang = False
    FakeBatchBuilder.launches = 0
    FakeBuilder.launches = 0
    yield
    FakeStream.hang = False


def small_requests(n, rate=2000.0):
    """Tiny grids (so the CPU output buffers stay small), arriving at ``rate``."""
    reqs = []
    for i in range(n):
        t = (mg.TRI, mg.TET, mg.HEX)[i % 3]
        reqs.append(Request(i, t, 3 + i % 4, i, i / rate))
    return reqs


def test_batch_server_serves_every_request(fake_cuda):
    reqs = small_requests(40)
    srv = BatchServer(budget_bytes=1 << 30, lanes=2, caps=LaneCaps(max_meshes=8), device="cpu", use_graph=False)
    st = srv.run(reqs)
    assert st["requests"] == 40 and st["failed"] == 0 and st["rejected"] == 0
    assert all(r.t_done >= r.arrival for r in reqs)           # completion after arrival
    assert all(r.t_done >= r.t_start >= 0 for r in reqs)
    # a lone request runs as a single-mesh build, several as one batch launch
    assert st["batches"] == FakeBatchBuilder.launches + FakeBuilder.launches and 5 <= st["batches"] <= 40
    assert FakeBatchBuilder.launches >= 1                      # at most 8 per batch
    assert st["max_ms"] >= st["p999_ms"] >= st["p99_ms"] >= st["p50_ms"] > 0


def test_batch_server_light_load_builds_each_request_alone(fake_cuda):
    # arrivals further apart than a unit's device time: every request finds
    # the stream below its depth and is built at once, on its own
    reqs = [Request(i, (mg.TRI, mg.TET, mg.HEX)[i % 3], 4, i, i * 3 * GPU_S) for i in range(12)]
    srv = BatchServer(budget_bytes=1 << 30, lanes=2, caps=LaneCaps(max_meshes=8), device="cpu", use_graph=False)
    st = srv.run(reqs)
    assert st["failed"] == 0 and st["batches"] == 12
    assert FakeBuilder.launches == 12 and FakeBatchBuilder.launches == 0
    assert all(r.t_done - r.arrival < 10 * GPU_S for r in reqs)   # never queued behind a backlog


def test_batch_server_holds_arrivals_beyond_its_depth_for_one_batch(fake_cuda):
    # one stream, two units in flight: a burst leaves as batches of at most
    # max_meshes while both slots are free, the remainder once a unit completes
    reqs = [Request(i, mg.TRI, 4, i, 0.0) for i in range(20)]
    srv = BatchServer(budget_bytes=1 << 30, lanes=2, caps=LaneCaps(max_meshes=8), device="cpu", use_graph=False,
                      streams=1, depth=2, batch_min=2)
    st = srv.run(reqs)
    assert st["failed"] == 0 and st["requests"] == 20
    assert FakeBatchBuilder.launches == 3 and FakeBuilder.launches == 0 and st["batches"] == 3   # 8 + 8 + 4
    # one stream: units complete in the order they were admitted
    done = [r.t_done for r in reqs]
    assert done == sorted(done)


def test_batch_server_small_queues_go_alone_on_the_least_loaded_stream(fake_cuda):
    # fewer queued requests than batch_min: each leaves alone, spread over
    # the two streams; a longer queue makes a batch
    reqs = [Request(i, mg.TRI, 4, i, 0.0) for i in range(3)]
    srv = BatchServer(budget_bytes=1 << 30, lanes=2, caps=LaneCaps(max_meshes=8), device="cpu", use_graph=False,
                      streams=2, depth=1, batch_min=4)
    st = srv.run(reqs)
    assert st["failed"] == 0 and FakeBuilder.launches == 3 and FakeBatchBuilder.launches == 0
    # two streams: the third request waits behind one of the first two
    assert reqs[2].t_done > min(reqs[0].t_done, reqs[1].t_done)
    reqs = [Request(i, mg.TRI, 4, i, 0.0) for i in range(12)]
    st = srv.run(reqs)
    assert st["failed"] == 0 and FakeBatchBuilder.launches >= 1


def test_batch_server_keeps_batching_a_backlog_until_it_empties(fake_cuda):
    # one stream of depth one, batches from eight waiting requests: a burst of
    # nine leaves as a batch of eight (max_meshes) with one request left; the
    # three that arrive while the batch runs make a queue of four -- fewer
    # than eight, but the backlog has not emptied, so the four leave as one
    # batch instead of four single builds
    reqs = [Request(i, mg.TRI, 4, i, 0.0) for i in range(9)]
    reqs += [Request(9 + i, mg.TRI, 4, 9 + i, 0.2 * GPU_S) for i in range(3)]
    srv = BatchServer(budget_bytes=1 << 30, lanes=2, caps=LaneCaps(max_meshes=8), device="cpu", use_graph=False,
                      streams=1, depth=1, batch_min=8)
    st = srv.run(reqs)
    assert st["failed"] == 0 and st["requests"] == 12
    assert FakeBuilder.launches == 0 and FakeBatchBuilder.launches == 2 and st["batches"] == 2


def test_batch_server_rejects_what_no_lane_holds(fake_cuda):
    reqs = small_requests(6)
    reqs.append(Request(6, mg.TRI, 200, 1, 0.001))            # 79,202 triangles: more than a lane's capacity
    srv = BatchServer(budget_bytes=1 << 30, lanes=2, caps=LaneCaps(max_meshes=4, max_elems=10_000), device="cpu",
                      use_graph=False)
    st = srv.run(reqs)
    assert st["rejected"] == 1 and st["requests"] == 6
    assert reqs[-1].status == 7 and reqs[-1].t_done < 0


def test_plain_server_serves_in_arrival_order(fake_cuda):
    reqs = small_requests(20)
    srv = PlainServer(Request(0, mg.HEX, 6, 1, 0.0), device="cpu")
    st = srv.run(reqs)
    assert st["requests"] == 20 and st["failed"] == 0
    done = [r.t_done for r in sorted(reqs, key=lambda r: r.arrival)]
    assert done == sorted(done)                                # one stream: completions in order


def test_check_deadline():
    serve.check_deadline(10.0, 5.0, "x", now=14.9)
    with pytest.raises(serve.ServeTimeout, match="deadline 5.0 s"):
        serve.check_deadline(10.0, 5.0, "x", now=15.1)


def test_batch_server_watchdog_on_a_stream_that_never_completes(fake_cuda):
    FakeStream.hang = True
    srv = BatchServer(budget_bytes=1 << 30, lanes=2, caps=LaneCaps(max_meshes=4), device="cpu", use_graph=False,
                      deadline_s=0.2)
    t = time.perf_counter()
    with pytest.raises(serve.ServeTimeout, match="unit of"):
        srv.run(small_requests(10))
    assert 0.2 <= time.perf_counter() - t < 5.0


def test_plain_server_watchdog_on_a_stream_that_never_completes(fake_cuda):
    FakeStream.hang = True
    srv = PlainServer(Request(0, mg.HEX, 6, 1, 0.0), device="cpu", deadline_s=0.2)
    t = time.perf_counter()
    with pytest.raises(serve.ServeTimeout, match="build of request 0"):
        srv.run(small_requests(5))
    assert 0.2 <= time.perf_counter() - t < 5.0
