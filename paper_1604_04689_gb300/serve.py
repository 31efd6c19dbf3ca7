"""Serving loop: continuous batching of neighbour-CSR build requests.

Requests (a seeded grid mesh: type, grid side, seed) arrive over time.  The
batched server owns ``streams`` CUDA streams, a single-mesh builder per
stream and ``lanes`` batch slots (a slot: batch workspaces of a small and of
the full capacity, pinned staging and a CUDA graph captured once around each
batched launch).  Work goes to the streams as units; each stream holds at
most ``depth`` units in flight, and a new unit goes to the open stream with
the fewest elements in flight.  Whenever a stream is open, the requests that
have arrived are admitted at once: fewer than ``batch_min`` waiting requests
leave one by one as single-mesh builds; ``batch_min`` or more leave together
as one batch on a free slot, and once such a backlog has formed every queue
of two or more leaves as a batch until the queue has emptied (so a loaded
server does not fall back to single builds while a backlog remains) (in arrival order, while they fit the slot's
capacity, ``batch_elems`` elements and the device-memory budget).  So a lightly loaded server answers
each request as soon as it arrives, with small requests running beside large
ones instead of behind them, and a loaded one amortises the launch sequence
over every request that queued while all streams were busy.  Each request's
connectivity is materialised on its stream (device generator, the stand-in
for an upload).  The plain server answers the same requests one build call
per mesh on one stream.

Latency of a request = completion (CUDA event at the end of its unit, mapped
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

    def holds_caps(self, other: "LaneCaps") -> bool:
        """True when this class is no larger than `other` in every capacity."""
        return (self.max_meshes <= other.max_meshes and self.max_elems <= other.max_elems
                and self.max_nodes <= other.max_nodes and self.max_conn <= other.max_conn
                and self != other)

    def holds(self, batch) -> bool:
        return (len(batch) <= self.max_meshes and sum(r.n_elems for r in batch) <= self.max_elems
                and sum(r.n_nodes for r in batch) <= self.max_nodes and sum(r.n_conn for r in batch) <= self.max_conn)


# The small capacity class of every lane: a batch launch's fixed costs (its
# bucket tables, scans and grids) follow the capacity it was captured for, so
# a batch that fits runs on this class's own graph instead of the full one.
SMALL_CAPS = LaneCaps(max_meshes=64, max_elems=2_500_000, max_nodes=2_500_000, max_conn=8_000_000)


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

    def form(self, queue: deque, free_bytes: int, limit: Optional[int] = None,
             max_elems: Optional[int] = None) -> list:
        c = self.caps
        cap = c.max_meshes if limit is None else min(limit, c.max_meshes)
        emax = c.max_elems if max_elems is None else min(max_elems, c.max_elems)
        batch, e, nn_, cc, b = [], 0, 0, 0, 0
        while queue and len(batch) < cap:
            r = queue[0]
            if (e + r.n_elems > (emax if batch else c.max_elems) or nn_ + r.n_nodes > c.max_nodes
                    or cc + r.n_conn > c.max_conn or b + r.device_bytes() > free_bytes):
                break
            queue.popleft()
            batch.append(r)
            e += r.n_elems
            nn_ += r.n_nodes
            cc += r.n_conn
            b += r.device_bytes()
        return batch


class _Graph:
    """One capacity class of a lane: a batch workspace and the CUDA graph
    captured around its launch on the lane's stream."""

    def __init__(self, torch, caps: LaneCaps, device, want: int, use_graph: bool, stream):
        self.torch = torch
        self.caps = caps
        self.stream = stream
        self.bb = nn.BatchBuilder(caps.max_meshes, caps.max_elems, caps.max_nodes, caps.max_conn, want=want,
                                  device=device)
        self.graph = None
        self.use_graph = use_graph

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


class _Lane:
    """A batch slot: its capacity classes (small first, then the slot's full
    capacity; a batch runs on the smallest class that holds it), each with a
    batch workspace, pinned staging and a graph captured on the server's
    stream.  A slot takes a new batch once its previous one has completed, so
    its staging is never rewritten while a launch may still read it."""

    def __init__(self, torch, caps: LaneCaps, device, want: int, use_graph: bool, stream):
        self.torch = torch
        self.want = want
        self.stream = stream
        classes = [SMALL_CAPS] if SMALL_CAPS.holds_caps(caps) else []
        self.classes = [_Graph(torch, c, device, want, use_graph, self.stream) for c in classes + [caps]]
        self.cls = None        # the class running the slot's current batch
        self.busy = False

    @property
    def bb(self):
        return (self.cls or self.classes[-1]).bb

    def workspace_bytes(self) -> int:
        return sum(g.bb.ws_bytes for g in self.classes)

    def pick(self, batch):
        self.cls = next(g for g in self.classes if g.caps.holds(batch))
        return self.cls

    def launch(self):
        self.cls.launch()


class _Sizes:
    """A request's mesh sizes in the C ABI's mesh form, for host-only sizing
    queries (the connectivity pointer is a placeholder no query reads)."""

    def __init__(self, r: Request):
        self.r = r

    def struct(self):
        r = self.r
        return nn.NNMesh(type=r.etype, n_nodes=r.n_nodes, n_elems=r.n_elems, n_conn=r.n_conn, conn=256,
                         elem_ptr=None, elem_type=None)


def single_ws_bytes(builder, r: Request, want: int) -> int:
    """Workspace of one single-mesh build of request `r` (host-only query on
    the request's sizes)."""
    return builder.query(_Sizes(r), want)[0]


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
                 deadline_s: float = 60.0, streams: int = 2, depth: int = 2, batch_min: int = 8,
                 batch_elems: Optional[int] = None):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.deadline_s = deadline_s
        self.caps = caps or LaneCaps()
        self.want = want
        self.keep = keep_results
        self.depth = max(1, depth)          # units in flight per stream
        self.batch_min = max(2, batch_min)  # queued requests that make a batch (fewer: the oldest alone)
        # elements a batch takes: at most the small capacity class, whose graph's
        # fixed costs are small (this bounds the latency of a batch's members)
        self.batch_elems = batch_elems if batch_elems is not None else SMALL_CAPS.max_elems
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max(1, streams))]
        self.lanes = [_Lane(torch, self.caps, self.device, want, use_graph, self.streams[i % len(self.streams)])
                      for i in range(lanes)]
        self.singles = [nn.Builder(self.device) for _ in self.streams]
        self.single_ws = [None] * len(self.streams)
        self.single_ws_bytes = 0
        self.budget = budget_bytes - sum(l.workspace_bytes() for l in self.lanes)
        if self.budget <= 0:
            raise ValueError("budget smaller than the lane workspaces")
        self.admission = Admission(self.caps)
        self.batches = 0

    def size_single(self, requests) -> int:
        """Workspace of each stream's single-mesh builder for the largest of
        `requests` (grown, never shrunk; host sizing only).  Returns the bytes
        added."""
        need = max((single_ws_bytes(self.singles[0], r, self.want) for r in requests), default=0)
        if need <= self.single_ws_bytes:
            return 0
        added = (need - self.single_ws_bytes) * len(self.streams)
        self.single_ws = [b.workspace(need) for b in self.singles]
        self.single_ws_bytes = need
        return added

    def warm(self, request: Request) -> None:
        """Build `request` once on every capacity class of every slot, so that
        every graph is captured before any timed run."""
        torch = self.torch
        for lane in self.lanes:
            for g in lane.classes:
                if not g.caps.holds([request]):
                    continue
                with torch.cuda.stream(lane.stream):
                    dm, out = _alloc_and_generate(torch, request, self.device, lane.stream, self.want)
                lane.cls = g
                st = g.bb.prepare([dm], [out])
                if st:
                    raise nn.NNError(st, "nn_batch_prepare")
                g.launch()
                lane.stream.synchronize()
                lane.cls = None

    def run(self, requests: List[Request]) -> dict:
        torch = self.torch
        # the single-mesh builders sized for the largest request of the run
        # (outside the timed loop; their workspaces count against the budget)
        self.budget -= self.size_single([r for r in requests if self.admission.fits_alone(r)])
        if self.budget <= 0:
            raise ValueError("budget smaller than the lane workspaces")
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue, inflight = deque(), []
        draining = False                 # a backlog formed: batch every queue of two or more until it empties
        load = [0] * len(self.streams)   # units in flight per stream
        work = [0] * len(self.streams)   # their elements: a unit goes to the least loaded stream
        # statuses: each unit writes those of its requests at their admission
        # positions, on its stream (read once, after the run)
        status = torch.zeros(max(len(requests), 1), dtype=torch.int32, device=self.device)
        admitted = []
        used = 0
        ev0 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(self.device)
        ev0.record(torch.cuda.current_stream(self.device))
        t0 = time.perf_counter()
        rejected = []
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                (queue if self.admission.fits_alone(r) else rejected).append(r)
            still = []
            for u in inflight:
                if u["done"].query():
                    t_done = ev0.elapsed_time(u["done"]) * 1e-3
                    t_start = ev0.elapsed_time(u["start"]) * 1e-3
                    for r, (dm, out) in zip(u["reqs"], u["bufs"]):
                        r.t_done = t_done
                        r.t_start = t_start
                        if self.keep:
                            r.result = {k: (rp, col) for k, (rp, col) in out.items()}
                        used -= r.device_bytes()
                    if u["lane"] is not None:
                        u["lane"].busy = False
                    load[u["si"]] -= 1
                    work[u["si"]] -= sum(r.n_elems for r in u["reqs"])
                else:
                    check_deadline(u["t_launch"], self.deadline_s, f"unit of {len(u['reqs'])} requests")
                    still.append(u)
            inflight = still
            open_ = [i for i in range(len(self.streams)) if load[i] < self.depth]
            si = min(open_, key=lambda i: work[i]) if open_ else 0
            if queue and open_:
                s = self.streams[si]
                lane = next((l for l in self.lanes if not l.busy and l.stream is s), None)
                if lane is None:
                    lane = next((l for l in self.lanes if not l.busy), None)
                if len(queue) >= self.batch_min:
                    draining = True
                many = (len(queue) >= self.batch_min or (draining and len(queue) >= 2)) and lane is not None
                batch = self.admission.form(queue, self.budget - used, limit=None if many else 1,
                                            max_elems=self.batch_elems)
                if batch:
                    k0 = len(admitted)
                    admitted.extend(batch)
                    with torch.cuda.stream(s):
                        bufs = [_alloc_and_generate(torch, r, self.device, s, self.want) for r in batch]
                    for r in batch:
                        used += r.device_bytes()
                    ev_start, ev_done = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    if len(batch) == 1:  # a lone request: the single-mesh build, no batch tables
                        lane = None
                        ev_start.record(s)
                        (dm, out), = bufs
                        st = self.singles[si].launch(dm, self.want, out, ws=self.single_ws[si],
                                                     ws_bytes=self.single_ws_bytes, stream=s,
                                                     status=status[k0:k0 + 1])
                        if st:
                            raise nn.NNError(st, "single build")
                    else:
                        if lane.stream is not s:  # the slot's graph replays on its own stream
                            ev_in = torch.cuda.Event()
                            ev_in.record(s)
                            lane.stream.wait_event(ev_in)
                        lane.pick(batch)
                        st = lane.bb.prepare([d for d, _ in bufs], [o for _, o in bufs])
                        if st:
                            raise nn.NNError(st, "nn_batch_prepare")
                        ev_start.record(lane.stream)
                        lane.launch()
                        lane.busy = True
                        with torch.cuda.stream(lane.stream):
                            status[k0:k0 + len(batch)].copy_(lane.bb.status[:len(batch)], non_blocking=True)
                        if lane.stream is not s:
                            ev_out = torch.cuda.Event()
                            ev_out.record(lane.stream)
                            s.wait_event(ev_out)
                    ev_done.record(s)
                    load[si] += 1
                    work[si] += sum(r.n_elems for r in batch)
                    inflight.append(dict(reqs=batch, bufs=bufs, start=ev_start, done=ev_done, lane=lane, si=si,
                                         t_launch=time.perf_counter()))
                    self.batches += 1
                    if not queue:
                        draining = False
                    continue
            if not queue:
                draining = False
            if not inflight and not queue and pending:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.001)))
            elif inflight:
                time.sleep(20e-6)
        torch.cuda.synchronize(self.device)
        st_all = status.cpu().tolist()
        for i, r in enumerate(admitted):
            r.status = int(st_all[i])
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
