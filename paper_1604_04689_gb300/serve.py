"""Serving loop: continuous batching of neighbour-CSR build requests.

Requests (a seeded grid mesh: type, grid side, seed) arrive over time.  The
batched server keeps ``lanes`` independent lanes (a CUDA stream, a batch
workspace with fixed capacity, pinned staging and a CUDA graph captured once
around the batched launch).  Whenever a lane is free it admits the requests
that have arrived, in arrival order, while they fit the lane's capacity and
the device-memory budget, materialises their connectivity on the lane's stream
(device generator, the stand-in for an upload), prepares the batch tables and
replays the lane's graph.  While one lane's batch runs on the GPU, the next
batch is admitted and launched on another lane, so work overlaps on the device
and requests are admitted as lanes and memory free up.  The plain server
answers the same requests one build call per mesh on one stream.

Latency of a request = completion (CUDA event at the end of its batch, mapped
to the host clock) - arrival.  Results are identical whether a request is
built alone or in a batch (see tests/test_gpu_serve.py).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import meshgen, nn

NPE = {meshgen.TRI: 3, meshgen.QUAD: 4, meshgen.TET: 4, meshgen.HEX: 8}
K_EDGES = {meshgen.TRI: 2, meshgen.QUAD: 2, meshgen.TET: 3, meshgen.HEX: 3}


@dataclass
class Request:
    rid: int
    etype: int
    n: int                 # grid side in nodes
    seed: int
    arrival: float         # seconds from the start of the run
    n_nodes: int = 0
    n_elems: int = 0
    t_done: float = -1.0
    t_start: float = -1.0  # device time its build was enqueued behind (after its input was generated)
    status: int = -1
    result: Optional[dict] = None

    def __post_init__(self):
        m = self.n - 1
        d3 = self.etype in (meshgen.TET, meshgen.HEX)
        self.n_nodes = self.n ** 3 if d3 else self.n ** 2
        cells = m ** 3 if d3 else m * m
        self.n_elems = {meshgen.TRI: 2 * cells, meshgen.QUAD: cells, meshgen.TET: 6 * cells,
                        meshgen.HEX: cells}[self.etype]

    @property
    def n_conn(self) -> int:
        return self.n_elems * NPE[self.etype]

    def device_bytes(self) -> int:
        """Connectivity + both outputs at their capacity bounds."""
        return 4 * self.n_conn + 2 * 8 * (self.n_nodes + 1) + 4 * K_EDGES[self.etype] * self.n_conn + 4 * self.n_conn


def make_requests(n_requests: int, rate: float, base_seed: int = 4) -> List[Request]:
    """The seeded request stream: per-request type/size/seed, Poisson arrivals."""
    arr = meshgen.poisson_arrivals(n_requests, rate, base_seed) if rate > 0 else np.zeros(n_requests)
    out = []
    for i in range(n_requests):
        t, n, s = meshgen.request_spec(i, base_seed)
        out.append(Request(i, t, n, s, float(arr[i])))
    return out


@dataclass
class LaneCaps:
    max_meshes: int = 1024
    max_elems: int = 24_000_000
    max_nodes: int = 24_000_000
    max_conn: int = 64_000_000


class ServeTimeout(RuntimeError):
    """A batch (or a plain build) whose completion event did not fire within
    the host deadline.  The device kernels bound their own waits, so this is
    a backstop: the loop stops with an error instead of polling forever."""


def check_deadline(t_launch: float, deadline_s: float, what: str, now: Optional[float] = None) -> None:
    """Raise ServeTimeout if ``what``, enqueued at host time ``t_launch``, is
    still running ``deadline_s`` seconds later."""
    now = time.perf_counter() if now is None else now
    if now - t_launch > deadline_s:
        raise ServeTimeout(f"{what} not complete {now - t_launch:.1f} s after launch (deadline {deadline_s} s)")


class Admission:
    """Which waiting requests go into the next batch (host logic only).

    FIFO: take requests in arrival order while the batch stays within the lane
    capacity and the free device-memory budget; stop at the first that does
    not fit (no overtaking, so latency stays fair).  A request larger than a
    whole empty lane is rejected."""

    def __init__(self, caps: LaneCaps):
        self.caps = caps

    def fits_alone(self, r: Request) -> bool:
        c = self.caps
        return r.n_elems <= c.max_elems and r.n_nodes <= c.max_nodes and r.n_conn <= c.max_conn

    def form(self, queue: deque, free_bytes: int) -> list:
        c = self.caps
        batch, e, nn_, cc, b = [], 0, 0, 0, 0
        while queue and len(batch) < c.max_meshes:
            r = queue[0]
            if (e + r.n_elems > c.max_elems or nn_ + r.n_nodes > c.max_nodes or cc + r.n_conn > c.max_conn
                    or b + r.device_bytes() > free_bytes):
                break
            queue.popleft()
            batch.append(r)
            e += r.n_elems
            nn_ += r.n_nodes
            cc += r.n_conn
            b += r.device_bytes()
        return batch


class _Lane:
    def __init__(self, torch, caps: LaneCaps, device, want: int, use_graph: bool):
        self.torch = torch
        self.stream = torch.cuda.Stream(device)
        self.bb = nn.BatchBuilder(caps.max_meshes, caps.max_elems, caps.max_nodes, caps.max_conn, want=want,
                                  device=device)
        self.graph = None
        self.use_graph = use_graph
        self.event = torch.cuda.Event(enable_timing=True)
        self.ev_start = torch.cuda.Event(enable_timing=True)
        self.reqs = None
        self.bufs = None
        self.t_launch = 0.0    # host time the lane's current batch was enqueued

    def workspace_bytes(self) -> int:
        return self.bb.ws_bytes

    def launch(self):
        torch = self.torch
        if not self.use_graph:
            st = self.bb.launch(self.stream)
            if st:
                raise nn.NNError(st, "nn_batch_launch")
            return
        if self.graph is None:  # first batch: run once eagerly, then capture the launch
            st = self.bb.launch(self.stream)
            if st:
                raise nn.NNError(st, "nn_batch_launch")
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                st = self.bb.launch(self.stream)
            if st:
                raise nn.NNError(st, "nn_batch_launch")
            # the eager run already built this batch; replaying again is harmless
        with torch.cuda.stream(self.stream):
            self.graph.replay()


def _alloc_and_generate(torch, r: Request, device, stream, want):
    dm = nn.generate_grid(r.etype, r.n, r.seed, device=device, stream=stream)
    out = {}
    if want & nn.WANT_NODES:
        out["nodes"] = (torch.empty(r.n_nodes + 1, dtype=torch.int64, device=device),
                        torch.empty(max(K_EDGES[r.etype] * r.n_conn, 1), dtype=torch.int32, device=device))
    if want & nn.WANT_ELEMS:
        out["elems"] = (torch.empty(r.n_nodes + 1, dtype=torch.int64, device=device),
                        torch.empty(max(r.n_conn, 1), dtype=torch.int32, device=device))
    return dm, out


def _stats(reqs: List[Request], t_first: float, t_last: float) -> dict:
    lat = np.array([r.t_done - r.arrival for r in reqs])
    build = np.array([r.t_done - r.t_start for r in reqs if r.t_start >= 0])
    elems = sum(r.n_elems for r in reqs)
    span = max(t_last - t_first, 1e-9)
    out = {"requests": len(reqs), "elements": int(elems), "makespan_s": span,
           "req_per_s": len(reqs) / span, "melem_per_s": elems / span / 1e6,
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "p999_ms": float(np.percentile(lat, 99.9) * 1e3),
           "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
           "failed": int(sum(1 for r in reqs if r.status != 0))}
    if build.size:  # completion minus the start of the request's build (queueing and generation excluded)
        out.update(build_p50_ms=float(np.percentile(build, 50) * 1e3), build_p99_ms=float(np.percentile(build, 99) * 1e3))
    return out


class BatchServer:
    def __init__(self, budget_bytes: int = 40 << 30, lanes: int = 2, caps: Optional[LaneCaps] = None,
                 want: int = nn.WANT_BOTH, device=None, use_graph: bool = True, keep_results: bool = False,
                 deadline_s: float = 60.0):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.deadline_s = deadline_s
        self.caps = caps or LaneCaps()
        self.want = want
        self.keep = keep_results
        self.lanes = [_Lane(torch, self.caps, self.device, want, use_graph) for _ in range(lanes)]
        self.budget = budget_bytes - sum(l.workspace_bytes() for l in self.lanes)
        if self.budget <= 0:
            raise ValueError("budget smaller than the lane workspaces")
        self.admission = Admission(self.caps)
        self.batches = 0

    def run(self, requests: List[Request]) -> dict:
        torch = self.torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue, free, busy = deque(), list(self.lanes), []
        used = 0
        ev0 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(self.device)
        ev0.record(torch.cuda.current_stream(self.device))
        t0 = time.perf_counter()
        rejected = []
        while pending or queue or busy:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                (queue if self.admission.fits_alone(r) else rejected).append(r)
            still = []
            for lane in busy:
                if lane.event.query():
                    t_done = ev0.elapsed_time(lane.event) * 1e-3
                    stat = lane.bb.status[: len(lane.reqs)].cpu().tolist()
                    t_start = ev0.elapsed_time(lane.ev_start) * 1e-3
                    for r, (dm, out), s in zip(lane.reqs, lane.bufs, stat):
                        r.t_done = t_done
                        r.t_start = t_start
                        r.status = int(s)
                        if self.keep:
                            r.result = {k: (rp, col) for k, (rp, col) in out.items()}
                        used -= r.device_bytes()
                    lane.reqs = lane.bufs = None
                    free.append(lane)
                else:
                    check_deadline(lane.t_launch, self.deadline_s, f"batch of {len(lane.reqs)} requests")
                    still.append(lane)
            busy = still
            if free and queue:
                batch = self.admission.form(queue, self.budget - used)
                if batch:
                    lane = free.pop()
                    with torch.cuda.stream(lane.stream):
                        bufs = [_alloc_and_generate(torch, r, self.device, lane.stream, self.want) for r in batch]
                    for r in batch:
                        used += r.device_bytes()
                    st = lane.bb.prepare([d for d, _ in bufs], [o for _, o in bufs])
                    if st:
                        raise nn.NNError(st, "nn_batch_prepare")
                    lane.ev_start.record(lane.stream)
                    lane.t_launch = time.perf_counter()
                    lane.launch()
                    lane.event.record(lane.stream)
                    lane.reqs, lane.bufs = batch, bufs
                    busy.append(lane)
                    self.batches += 1
                    continue
            if not busy and not queue and pending:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.001)))
            elif busy:
                time.sleep(20e-6)
        for r in rejected:
            r.status = 7  # NN_ERR_BUDGET: larger than an empty lane
        served = [r for r in requests if r.t_done >= 0]
        st = _stats(served, min(r.arrival for r in requests), max(r.t_done for r in served))
        st.update(batches=self.batches, rejected=len(rejected))
        return st


class PlainServer:
    """One nn_neighbors_both call per request, in arrival order, on one stream."""

    def __init__(self, max_request: Request, want: int = nn.WANT_BOTH, device=None, keep_results: bool = False,
                 deadline_s: float = 60.0):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.deadline_s = deadline_s
        self.b = nn.Builder(self.device)
        self.stream = torch.cuda.Stream(self.device)
        self.want = want
        self.keep = keep_results
        big = nn.generate_grid(max_request.etype, max_request.n, 1, device=self.device)
        self.ws_bytes = self.b.query(big, want)[0]
        self.ws = self.b.workspace(self.ws_bytes)
        del big

    def run(self, requests: List[Request]) -> dict:
        torch = self.torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        ev0 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(self.device)
        ev0.record(torch.cuda.current_stream(self.device))
        t0 = time.perf_counter()
        inflight = deque()
        status = torch.zeros(len(requests), dtype=torch.int32, device=self.device)
        idx = {}
        while pending or inflight:
            now = time.perf_counter() - t0
            while inflight and inflight[0][1].query():
                r, ev, out, ev_s, _ = inflight.popleft()
                r.t_done = ev0.elapsed_time(ev) * 1e-3
                r.t_start = ev0.elapsed_time(ev_s) * 1e-3
                if self.keep:
                    r.result = out
            if pending and pending[0].arrival <= now:
                r = pending.popleft()
                idx[r.rid] = len(idx)
                ev_s = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(self.stream):
                    dm, out = _alloc_and_generate(torch, r, self.device, self.stream, self.want)
                    ev_s.record(self.stream)
                    st_ = self.b.launch(dm, self.want, out, ws=self.ws, ws_bytes=self.ws_bytes, stream=self.stream,
                                        status=status[idx[r.rid]:idx[r.rid] + 1])
                if st_:
                    raise nn.NNError(st_, "plain build")
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(self.stream)
                inflight.append((r, ev, out, ev_s, time.perf_counter()))
                continue
            if inflight:
                check_deadline(inflight[0][4], self.deadline_s, f"build of request {inflight[0][0].rid}")
                time.sleep(20e-6)
            elif pending:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.001)))
        torch.cuda.synchronize(self.device)
        st_all = status.cpu().tolist()
        for r in requests:
            r.status = int(st_all[idx[r.rid]])
        return _stats(requests, min(r.arrival for r in requests), max(r.t_done for r in requests))
