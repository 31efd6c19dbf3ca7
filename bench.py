#!/usr/bin/env python
"""Benchmark: one-ring neighbor CSR build throughput on GB300.

One step = one full build of BOTH results (neighbor-node CSR and
neighbor-element CSR) for one seeded synthetic mesh, through the C ABI, with
the connectivity already resident in HBM.  Metric: Melem/s (mesh elements
processed per second, whole job).  Default workload: the hex grid 257^3
(16,974,593 nodes, 16,777,216 hexes, node ids permuted), the largest of the
benchmark's meshes; the triangle grid 2048^2, the Kuhn tet grid 161^3
and the mixed hex/tet variant of the hex grid are timed in the same run under
"per_config", and a bounded serving run (batched vs one build per mesh)
under "serving".

Prints ONE JSON line (rank 0).  "roofline": the compulsory bytes of one build
(read the connectivity once, write both CSRs once) over the CUDA-event time
of the dominant kernel, against the measured copy bandwidth; the kernel's own
implementation bytes and its ncu DRAM bytes (when a capture of the current
source exists) are reported beside it under their own names.  "pipeline":
the same compulsory bytes over the whole step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Under torchrun (N > 1) every rank builds its own replica of the workload on its
own GPU (weak scaling, no collective on the data path); the timed region is
bracketed by barriers and the max over ranks is reported.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (mesh generator, taking the meshgen module; description)
    "tri2048": (lambda mg: mg.workload_mesh("tri2048"),
                "triangle grid 2048x2048 (4,194,304 nodes, 8,380,418 tris), seed 1, "
                "random diagonals, node ids and element order permuted"),
    "tri2048_holes": (lambda mg: mg.workload_mesh("tri2048_holes"),
                      "triangle grid 2048x2048 with 5% of triangles deleted, seed 100"),
    "tet161": (lambda mg: mg.workload_mesh("tet161"),
               "Kuhn tet grid 161^3 (4,173,281 nodes, 24,576,000 tets), seed 2, permuted"),
    "hex257": (lambda mg: mg.workload_mesh("hex257"),
               "hex grid 257^3 (16,974,593 nodes, 16,777,216 hexes), seed 3, node ids permuted"),
    "mixed257": (lambda mg: mg.workload_mesh("mixed257"),
                 "hex grid 257^3 with 30% of cells split into 6 tets, seed 103"),
    "tet101": (lambda mg: mg.tet_grid(101, 6),
               "Kuhn tet grid 101^3 (1,030,301 nodes, 6,000,000 tets), seed 6, permuted; a profiling case"),
    "hex129": (lambda mg: mg.hex_grid(129, 7),
               "hex grid 129^3 (2,146,689 nodes, 2,097,152 hexes), seed 7, node ids permuted; a profiling case"),
    "tri1448": (lambda mg: mg.tri_grid(1448, 5),
                "triangle grid 1448x1448 (2,096,704 nodes, 4,187,618 tris), seed 5, permuted "
                "(the profiling case: records exceed L2, a few hundred MB on the device)"),
    "tri64": (lambda mg: mg.workload_mesh("tri64"),
              "triangle grid 64x64 (4,096 nodes, 7,938 tris), seed 0, permuted"),
    "serve": (None, "stream of 10,000 mesh requests (tri / Kuhn tet / hex grids, elements log-uniform "
                    "1e3-2e6, per-request seeds), Poisson arrivals at 0.8x the plain saturated rate, "
                    "40 GB device-memory budget; batched continuous serving vs one build per mesh"),
}
# the headline metric: build throughput in mesh elements per second, with the
# dominant kernel's fraction of the HBM roofline in "roofline" and, for the
# serving workload, batched p50/p99 latency beside one build per mesh
METRIC = "neighbor-CSR build Melem/s and % of HBM roofline; batched p50/p99 vs plain"
WANT = {"both": 3, "nodes": 1, "elems": 2}
KERNEL_OF_STAGE = {"hist": "k_hist", "offsets": "k_offsets", "part": "k_part_coarse", "part_fine": "k_part_fine",
                   "bucket": "k_bucket", "place": "k_node_scan+k_node_copy"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference", "sortpipe"], default="ours",
                    help="sortpipe: the paper's sort / unique-by-key pipeline on the GPU with library primitives "
                         "(benchmark-only comparison, not part of the library)")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="hex257")
    ap.add_argument("--configs", default="tri2048,tet161,mixed257",
                    help="further workloads timed in the same run (per_config); empty: none")
    ap.add_argument("--no-serving", action="store_true", help="skip the bounded serving run of the default line")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests per load of the bounded serving run")
    ap.add_argument("--mesh-file", default="",
                    help="build a surface mesh read from this .ply or .obj file instead of a generated workload")
    ap.add_argument("--want", choices=list(WANT), default="both")
    ap.add_argument("--no-baseline", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--elem-adj", action="store_true",
                    help="also time element face adjacency from the built node -> element CSR")
    ap.add_argument("--tune", choices=["auto", "off", "sweep"], default="auto",
                    help="launch tuning: cached or timed once (auto), planner default (off), re-timed (sweep)")
    ap.add_argument("--requests", type=int, default=10000, help="serve workload: number of requests")
    ap.add_argument("--load", type=float, default=0.8, help="serve workload: arrival rate / plain saturated rate")
    ap.add_argument("--loads", default="", help="serve workload: also sweep these comma-separated loads")
    ap.add_argument("--table1", action="store_true",
                    help="time triangle grids at the vertex counts of the paper's Table 1 (synthetic stand-in)")
    ap.add_argument("--chunk-frac", type=float, default=0.0,
                    help="chunked build with this fraction of the whole-mesh workspace (prints its own line)")
    ap.add_argument("--host-io", action="store_true",
                    help="chunked build: connectivity and both CSRs in pinned host memory (out of core)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_mesh(name):
    from paper_1604_04689_gb300 import meshgen
    return WORKLOADS[name][0](meshgen)


def load_workload(args):
    """(workload name, description, mesh) of a single-mesh run: the generated
    workload, or the surface mesh of --mesh-file."""
    if args.mesh_file:
        from paper_1604_04689_gb300 import meshio
        mesh = meshio.read_mesh(args.mesh_file)
        base = os.path.basename(args.mesh_file)
        return (f"file:{base}", f"surface mesh read from {base} ({mesh.n_nodes} vertices, {mesh.n_elems} faces)",
                mesh)
    return args.workload, WORKLOADS[args.workload][1], make_mesh(args.workload)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            with open(self.path) as f:
                lines = f.readlines()
            os.unlink(self.path)
        except Exception:
            return None
        return parse_clock_samples(lines)


def parse_clock_samples(lines):
    """Summary of nvidia-smi samples of ClockSampler.FIELDS (csv, no header,
    no units): median SM clock, the maximum SM clock, and every throttle
    reason seen active in any sample; None without a valid sample."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts))
        except ValueError:      # a field nvidia-smi could not read ("[N/A]") or a torn line
            continue
    if not rows:
        return None
    sm = sorted(r[0] for r in rows)
    reasons = set()
    for _, _, parts in rows:
        for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                             parts[5:9]):
            if val.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": rows[0][1], "reasons": sorted(reasons),
            "samples": len(rows)}


# ---------------------------------------------------------------- baseline

def oracle_sample(workload):
    """A bounded sample of the same kind of mesh as `workload` for the CPU
    oracle: (mesh, description, elements of the sample / elements of the
    workload)."""
    from paper_1604_04689_gb300 import meshgen
    full = {"hex257": 16777216, "mixed257": 41924166, "tet161": 24576000, "tri2048": 8380418}.get(workload)
    if workload in ("hex257", "hex129"):
        n, mesh = 101, meshgen.hex_grid(101, 3)
        desc = f"hex grid {n}^3 ({mesh.n_elems} hexes, seed 3, node ids permuted)"
    elif workload == "mixed257":
        n, mesh = 65, meshgen.mixed_grid(65, 103)
        desc = f"hex grid {n}^3 with 30% of cells split into 6 tets ({mesh.n_elems} elements, seed 103)"
    elif workload in ("tet161", "tet101"):
        n, mesh = 51, meshgen.tet_grid(51, 2)
        desc = f"Kuhn tet grid {n}^3 ({mesh.n_elems} tets, seed 2, permuted)"
    else:
        n, mesh = 1024, meshgen.tri_grid(1024, 1)
        desc = f"triangle grid {n}x{n} ({mesh.n_elems} tris, seed 1, permuted)"
    return mesh, desc, (mesh.n_elems / full if full else None)


def pinned_core():
    """The host core the oracle is pinned to (the last one this process may use)."""
    try:
        return max(os.sched_getaffinity(0))
    except Exception:
        return None


def oracle_baseline(workload, runs=3):
    """The CPU oracle, as it stands, on a bounded sample of the same kind of
    mesh as the workload: median of `runs` builds, this process pinned to one
    host core meanwhile."""
    import oracle
    mesh, desc, ratio = oracle_sample(workload)
    core = pinned_core()
    old = None
    try:
        if core is not None:
            old = os.sched_getaffinity(0)
            os.sched_setaffinity(0, {core})
        times = []
        for _ in range(runs):
            t0 = time.perf_counter()
            r = oracle.neighbors(mesh, oracle.BOTH)
            times.append(time.perf_counter() - t0)
            assert r["status"] == 0
    finally:
        if old is not None:
            os.sched_setaffinity(0, old)
    dt = sorted(times)[len(times) // 2]
    return {"value": mesh.n_elems / dt / 1e6, "unit": "Melem/s", "cores": 1, "kind": "oracle", "host": host_info(),
            "runs": runs, "core": core, "seconds": times,
            "sample": f"{desc}, both CSRs, single-threaded std::set oracle, median of {runs} runs pinned to host "
                      f"core {core}; the sample has {ratio:.4f} of the workload's elements" if ratio else
                      f"{desc}, both CSRs, single-threaded std::set oracle, median of {runs} runs pinned to host "
                      f"core {core}"}


def host_info():
    """The host the oracle ran on: model name and core count (one core used)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return f"{model or 'unknown CPU'}, 1 of {os.cpu_count()} cores used"


def reference_arm(args):
    """--impl reference: the CPU oracle, as it stands, timed on a bounded
    sample of the same kind of mesh as the workload per step, pinned to one
    host core; rank 0 alone runs it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1604_04689_gb300 import meshgen
    if args.workload in ("hex257", "hex129", "mixed257"):
        n = 41
        mesh = meshgen.hex_grid(n, 3) if args.workload != "mixed257" else meshgen.mixed_grid(n, 103)
        sample = f"{'hex' if args.workload != 'mixed257' else 'mixed hex/tet'} grid {n}^3 ({mesh.n_elems} elements)"
    elif args.workload in ("tet161", "tet101"):
        n = 31
        mesh = meshgen.tet_grid(n, 2)
        sample = f"Kuhn tet grid {n}^3 ({mesh.n_elems} tets)"
    else:
        n = 256
        mesh = meshgen.tri_grid(n, 1)
        sample = f"triangle grid {n}x{n} ({mesh.n_elems} tris)"
    core = pinned_core()
    if core is not None:
        os.sched_setaffinity(0, {core})
    for _ in range(args.warmup):
        oracle.neighbors(mesh, WANT[args.want])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.neighbors(mesh, WANT[args.want])
        assert r["status"] == 0
    dt = time.perf_counter() - t0
    v = mesh.n_elems * args.steps / dt / 1e6
    sample = (f"{sample} per step, seeded and permuted like the workload, single-threaded std::set oracle on the "
              f"host, pinned to core {core}")
    line = {"metric": METRIC, "value": v, "unit": "Melem/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "want": args.want, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "Melem/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_info()},
            "e2e": {"value": v, "unit": "Melem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- paper's pipeline

LOCAL_EDGES = {0: ((0, 1), (1, 2), (2, 0)), 1: ((0, 1), (1, 2), (2, 3), (3, 0)),
               2: ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)),
               3: ((0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6), (3, 7))}


def sortpipe_build(torch, conn, etype, n_nodes):
    """The paper's GPU recipe (Sec. 2.2.1) with library primitives: every
    element of a uniform mesh (conn: int64 [T, npe] on the device) emits its
    directed edge pairs (both orientations) and its (node, element) pairs as
    64-bit keys; a radix sort orders them by key and unique-by-key gives the
    rows, repeats dropped (the set reading of a one-ring).  Returns (rp_n,
    col_n, rp_e, col_e).  Benchmark and test use only: it is the comparison
    the paper's design makes possible, not a code path of the library."""
    N, T = n_nodes, conn.shape[0]
    dev = conn.device
    eid = torch.arange(T, device=dev, dtype=torch.int64)
    edges = LOCAL_EDGES[etype]
    a = torch.cat([conn[:, i] for i, j in edges] + [conn[:, j] for i, j in edges])
    b = torch.cat([conn[:, j] for i, j in edges] + [conn[:, i] for i, j in edges])
    keep = a != b
    keys = torch.sort((a * N + b)[keep]).values
    u = torch.unique_consecutive(keys)
    rp_n = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    rp_n[1:] = torch.cumsum(torch.bincount(u // N, minlength=N), 0)
    col_n = (u % N).to(torch.int32)
    ek = torch.unique_consecutive(torch.sort((conn * T + eid[:, None]).reshape(-1)).values)
    rp_e = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    rp_e[1:] = torch.cumsum(torch.bincount(ek // T, minlength=N), 0)
    col_e = (ek % T).to(torch.int32)
    return rp_n, col_n, rp_e, col_e


def sortpipe_arm(args):
    """--impl sortpipe: the paper's pipeline (sortpipe_build) timed on this
    GPU, checked against the library's own build once, bit for bit."""
    import torch
    from paper_1604_04689_gb300 import nn
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    mesh = make_mesh(args.workload)
    if mesh.etype not in LOCAL_EDGES:
        print(json.dumps({"impl": "sortpipe", "unavailable": "uniform element types only"}))
        return
    N, T = mesh.n_nodes, mesh.n_elems
    conn = torch.from_numpy(mesh.conn).to(dev).view(T, -1).to(torch.int64)

    def build():
        return sortpipe_build(torch, conn, mesh.etype, N)

    ref = nn.Builder(dev).build(nn.DeviceMesh.from_host(mesh, device=dev))
    got = build()
    match = all(torch.equal(x, y.to(x.dtype)) for x, y in
                zip(got, (ref["nodes"][0], ref["nodes"][1], ref["elems"][0], ref["elems"][1])))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 1)):
        build()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        build()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    print(json.dumps({"metric": METRIC, "value": T / (ms * 1e-3) / 1e6, "unit": "Melem/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "int64 keys", "data": "synthetic", "impl": "sortpipe",
                      "config": {"workload": args.workload, "want": "both",
                                 "pipeline": "torch.sort (radix) + unique_consecutive + bincount/cumsum"},
                      "matches_library": bool(match)}), flush=True)


# ---------------------------------------------------------------- ours

# Table 1's scanned surfaces (vertex and triangle counts as the table prints
# them, in thousands), the paper's GT640 node / element times (ms), and the
# side of the random-diagonal triangle grid with about as many vertices
TABLE1 = (("Armadillo", 172000, 346000, 50.0, 22.1, 415), ("Angel", 237000, 474000, 66.7, 29.4, 487),
          ("Skeleton Hand", 327000, 655000, 89.1, 38.3, 572), ("Dragon", 437000, 871000, 112.7, 48.5, 661),
          ("Happy Buddha", 543000, 1088000, 138.5, 60.6, 737),
          ("Turbine Blade", 882000, 1765000, 221.3, 93.3, 939))


def table1_sweep(args):
    """Synthetic stand-in for Table 1: a triangle grid per scanned surface,
    with about its vertex count (same ~2 triangles per vertex and mean valence
    ~6), timed for the node rows, the element rows and both (CUDA events, L2
    flushed before each build, median of --steps).  The paper's own GT640
    times are printed beside them for context."""
    import torch
    from paper_1604_04689_gb300 import meshgen as mg
    from paper_1604_04689_gb300 import nn
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20), dtype=torch.uint8, device=dev)
    b = nn.Builder(dev)
    rows = []
    for name, v_paper, t_paper, node_ms, elem_ms, n in TABLE1:
        mesh = mg.tri_grid(n, 7)
        dm = nn.DeviceMesh.from_host(mesh, device=dev)
        row = {"mesh": name, "paper_V": v_paper, "paper_T": t_paper, "paper_gt640_ms": [node_ms, elem_ms],
               "grid": f"{n}x{n}", "V": mesh.n_nodes, "T": mesh.n_elems}
        for label, want in (("nodes", nn.WANT_NODES), ("elems", nn.WANT_ELEMS), ("both", nn.WANT_BOTH)):
            ws_bytes = b.query(dm, want)[0]
            ws = b.workspace(ws_bytes)
            out = b.alloc_outputs(dm, want)
            for _ in range(max(args.warmup, 3)):
                b.launch(dm, want, out, ws=ws, ws_bytes=ws_bytes)
            times = []
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = b.launch(dm, want, out, ws=ws, ws_bytes=ws_bytes)
                e1.record(stream)
                if st:
                    raise nn.NNError(st, "launch")
                torch.cuda.synchronize(dev)
                times.append(e0.elapsed_time(e1))
            if int(b.status.item()) != 0:
                raise RuntimeError("device status " + nn.STATUS[int(b.status.item())])
            times.sort()
            ms = times[len(times) // 2]
            row[f"{label}_ms"] = ms
            row[f"{label}_mtri_per_s"] = mesh.n_elems / (ms * 1e-3) / 1e6
            del ws, out
        rows.append(row)
    print(json.dumps({"table1_stand_in": rows, "steps": args.steps, "l2": "flushed before every timed build",
                      "data": "synthetic: random-diagonal triangle grids, seed 7, node ids and element order permuted"}),
          flush=True)


def chunked_bench(args):
    """Chunked build (nodes in consecutive-id chunks, each within a bounded
    workspace) beside the single build of the same mesh, same process, L2
    flushed before every step.  The chunk plan is made once (a count pass
    and a host plan) and its time reported apart; the timed step is the
    chunked build itself.  With --host-io the connectivity and both CSRs
    live in pinned host memory and the GPU reads and writes them in place."""
    import torch
    from paper_1604_04689_gb300 import nn
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    mesh = make_mesh(args.workload)
    want = WANT[args.want]
    b = nn.Builder(dev)
    dm = nn.DeviceMesh.from_host(mesh, device=dev)
    whole, nc, ec = b.query(dm, want)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize(dev)
        times = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2]

    out1 = b.alloc_outputs(dm, want)
    ws1 = torch.empty(whole, dtype=torch.uint8, device=dev)
    single_ms = timed(lambda: b.launch(dm, want, out1, ws=ws1, ws_bytes=whole))

    if args.host_io:
        conn = torch.from_numpy(mesh.conn).pin_memory()
        cdm = nn.DeviceMesh(dm.etype, dm.n_nodes, conn,
                            None if mesh.elem_ptr is None else torch.from_numpy(mesh.elem_ptr).pin_memory(),
                            None if mesh.elem_type is None else torch.from_numpy(mesh.elem_type).pin_memory())

        def host(n, dt):
            return torch.empty(n, dtype=dt, pin_memory=True)
        out = {}
        if want & nn.WANT_NODES:
            out["nodes"] = (host(mesh.n_nodes + 1, torch.int64), host(nc, torch.int32))
        if want & nn.WANT_ELEMS:
            out["elems"] = (host(mesh.n_nodes + 1, torch.int64), host(ec, torch.int32))
    else:
        cdm, out = dm, b.alloc_outputs(dm, want)
    ws_bytes = int(args.chunk_frac * whole)
    t0 = time.perf_counter()
    chunks = b.plan_chunks(cdm, want, ws_bytes)
    plan_s = time.perf_counter() - t0
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    chunk_ms = timed(lambda: b.launch_chunked(cdm, want, out, chunks, ws, ws_bytes))
    st = int(b.status.item())
    match = st == 0
    for k, (rp, col) in out.items():
        rp1, col1 = out1[k]
        nnz = int(rp1[-1].item())
        match = match and torch.equal(rp.to(dev), rp1) and torch.equal(col[:nnz].to(dev), col1[:nnz])
    T = mesh.n_elems
    print(json.dumps({"metric": METRIC, "value": T / (chunk_ms * 1e-3) / 1e6,
                      "unit": "Melem/s", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
                      "ms_per_step": chunk_ms, "higher_is_better": True, "dtype": "int32", "data": "synthetic",
                      "impl": "chunked",
                      "config": {"workload": args.workload, "want": args.want, "chunks": len(chunks),
                                 "ws_bytes": ws_bytes, "whole_mesh_ws_bytes": whole,
                                 "host_io": bool(args.host_io), "l2": "flushed (256 MiB write) before each step"},
                      "single_build_ms": single_ms, "single_build_value": T / (single_ms * 1e-3) / 1e6,
                      "plan_s": plan_s, "matches_single_build": bool(match)}), flush=True)


def serve_bench(args):
    """Serving workload: plain (one build per mesh) vs batched continuous serving on one arrival trace."""
    import copy
    import torch
    from paper_1604_04689_gb300 import nn
    from paper_1604_04689_gb300.serve import BatchServer, PlainServer, make_requests

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    budget = 40 << 30
    n = args.requests
    base = make_requests(n, 0.0)                     # sizes/types/seeds; arrivals set below
    big = max(base, key=lambda r: r.n_conn)
    plain = PlainServer(big)
    batched = BatchServer(budget_bytes=budget, lanes=2)
    # warm-up: every batch graph captured, then both servers on a short saturated prefix
    batched.warm(min(base, key=lambda r: r.n_conn))
    w = max(args.warmup, 1) * 20
    plain.run(copy.deepcopy(base[:w]))
    batched.run(copy.deepcopy(base[:min(n, 2000)]))  # every graph, batch and buffer size seen first
    # plain saturated rate R (all requests present at t = 0)
    n_sat = min(n, 2000)
    sat = plain.run(copy.deepcopy(base[:n_sat]))
    rate = args.load * sat["req_per_s"]
    trace = make_requests(n, rate)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    if not args.no_clocks:
        sampler.start()
    res_p = plain.run(copy.deepcopy(trace))
    res_b = batched.run(copy.deepcopy(trace))
    sweep = {}
    for ld in [float(x) for x in args.loads.split(",") if x.strip()]:
        tr = make_requests(n, ld * sat["req_per_s"])
        sweep[str(ld)] = {"rate_req_per_s": ld * sat["req_per_s"], "plain": plain.run(copy.deepcopy(tr)),
                          "batched": batched.run(copy.deepcopy(tr))}
    clocks = None if args.no_clocks else sampler.stop()
    line = {"metric": METRIC, "value": res_b["melem_per_s"], "unit": "Melem/s",
            "n_gpus": 1, "steps": n, "warmup": w, "ms_per_step": res_b["makespan_s"] * 1e3 / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "serve", "description": WORKLOADS["serve"][1], "requests": n,
                       "arrival_rate_req_per_s": rate, "load": args.load, "budget_bytes": budget,
                       "inputs": "generated on the device per request (stand-in for the upload)",
                       "l2": "inputs of the whole stream exceed L2"},
            "serving": {"plain_saturated": sat, "plain": res_p, "batched": res_b,
                        "batches": batched.batches, "streams": len(batched.streams), "depth": batched.depth,
                        "batch_min": batched.batch_min, "batch_slots": len(batched.lanes), "load_sweep": sweep},
            "clocks": clocks, "gpu_launches": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.impl == "sortpipe":
        sortpipe_arm(args)
        return
    if args.workload == "serve":
        serve_bench(args)
        return
    if args.chunk_frac > 0:
        chunked_bench(args)
        return
    if args.table1:
        table1_sweep(args)
        return

    import torch
    import torch.distributed as dist
    from paper_1604_04689_gb300 import nn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    want = WANT[args.want]
    workload, description, mesh = load_workload(args)
    head = time_build(torch, nn, dev, workload, description, mesh, args, want, world, barrier,
                      clocks=not args.no_clocks, e2e=not args.no_e2e, elem_adj=args.elem_adj)
    del mesh

    # further configurations in the same run (single GPU only: their timed
    # regions are their own, after the headline's)
    per_config = {}
    if world == 1 and not args.mesh_file:
        for name in [x.strip() for x in args.configs.split(",") if x.strip() and x.strip() != workload]:
            m = make_mesh(name)
            r = time_build(torch, nn, dev, name, WORKLOADS[name][1], m, args, want, world, barrier)
            per_config[name] = {k: r[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "config",
                                                  "roofline", "pipeline", "gpu_launches")}
            del m
            torch.cuda.empty_cache()

    serving = None
    if world == 1 and not args.no_serving:
        torch.cuda.empty_cache()
        serving = serving_summary(args)

    baseline = None
    if rank == 0 and world == 1 and not args.no_baseline:
        baseline = oracle_baseline(workload)

    line = {
        "metric": METRIC,
        "value": head["value"], "unit": "Melem/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": head["config"],
        "roofline": head["roofline"],
        "pipeline": head["pipeline"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "e2e": head["e2e"],
        "cpu_baseline": baseline,
        "per_config": per_config,
        "serving": serving,
    }
    if head.get("element_adjacency") is not None:
        line["element_adjacency"] = head["element_adjacency"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def time_build(torch, nn, dev, workload, description, mesh, args, want, world, barrier, clocks=False, e2e=False,
               elem_adj=False):
    """Time `args.steps` builds of `mesh` (after `args.warmup` untimed ones,
    L2 flushed before each, CUDA events on the launching stream, barriers and
    the maximum over ranks around the timed region) and account its bytes."""
    b = nn.Builder(dev)
    dm = nn.DeviceMesh.from_host(mesh, device=dev)
    tuning = None
    if args.tune != "off":
        from paper_1604_04689_gb300 import autotune
        tuning = autotune.tuned(b, dm, want, retune=args.tune == "sweep")
    ws_bytes, ncap, ecap = b.query(dm, want)
    plan = nn.nn_plan_info(b.h, dm.struct(), want)
    ws = b.workspace(ws_bytes)
    out = b.alloc_outputs(dm, want)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20), dtype=torch.uint8, device=dev)

    def step():
        st = b.launch(dm, want, out, ws=ws, ws_bytes=ws_bytes)
        if st:
            raise nn.NNError(st, "launch")

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    assert int(b.status.item()) == 0, nn.STATUS[int(b.status.item())]

    # ---- timed region: K builds, L2 flushed before each (outside the events)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    if clocks:
        sampler.start()
        time.sleep(0.3)
    nn.nn_profile_enable(b.h, True)
    stream = torch.cuda.current_stream(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    t_wall = time.perf_counter() - t_wall
    stage_ms, calls = nn.nn_profile_read(b.h)
    nn.nn_profile_enable(b.h, False)
    clk = sampler.stop() if clocks else None
    status = int(b.status.item())
    assert status == 0, nn.STATUS[status]
    per_step = sorted(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_ms = max_over_ranks(sum(per_step), world, dev)

    # ---- result sizes and bytes
    nnz = {k: int(rp[-1].item()) for k, (rp, col) in out.items()}
    N, T, n_conn = mesh.n_nodes, mesh.n_elems, mesh.n_conn
    ms_per_step = total_ms / args.steps
    stage = {k: v / max(calls, 1) for k, v in stage_ms.items()}
    acc = roofline_accounting(plan, N, T, n_conn, nnz, stage, workload, args.want)
    value = whole_job_value(T, args.steps, world, total_ms)
    pipeline = {"alg_bytes_per_step": acc["compulsory"],
                "achieved_gbs": acc["compulsory"] / (ms_per_step * 1e-3) / 1e9,
                "frac": acc["compulsory"] / (ms_per_step * 1e-3) / 1e9 / acc["peak"],
                "stage_ms_per_step": stage,
                "step_ms_median": per_step[len(per_step) // 2],
                "step_ms_p95": per_step[min(len(per_step) - 1, int(0.95 * len(per_step)))],
                "wall_s": t_wall}

    r = {"value": value, "unit": "Melem/s", "ms_per_step": ms_per_step, "steps": args.steps, "warmup": args.warmup,
         "config": {"workload": workload, "description": description,
                    "want": args.want, "n_nodes": N, "n_elems": T, "nnz": nnz,
                    "l2": f"flushed before every timed step ({flush.numel() >> 20} MiB write)",
                    "parallelism": "replicas" if world > 1 else "single GPU", "plan": plan,
                    "tuning": tuning},
         "roofline": acc["roofline"], "pipeline": pipeline,
         "gpu_launches": launches_per_build(plan, args.want) * args.steps, "clocks": clk, "e2e": None}
    if e2e:
        r["e2e"] = end_to_end(torch, nn, b, mesh, dm, want, ws, ws_bytes, out, args.steps, dev, world)
    if elem_adj and "elems" in out:
        r["element_adjacency"] = time_adjacency(torch, nn, b, dm, out, flush, stream, max(args.steps // 2, 3))
    del ws, out, flush, dm
    return r


def roofline_accounting(plan, N, T, n_conn, nnz, stage, workload, want):
    """Roofline of the dominant kernel.  frac: the compulsory bytes of one
    build -- the connectivity read once, each CSR (row pointers and columns)
    written once -- over the dominant kernel's CUDA-event time per launch,
    against the measured copy bandwidth.  Beside it, under their own names:
    the kernel's own implementation bytes per launch (records it reads,
    tables, rows it writes) and, when a capture of the current source
    exists, its ncu DRAM bytes per launch."""
    rb, G, B = plan["record_bytes"], plan["emit_ctas"], plan["n_buckets"]
    out_bytes = sum(8 * (N + 1) + 4 * v for v in nnz.values())
    compulsory = 4 * n_conn + out_bytes
    two_level = plan["partition"] > 0
    own = {  # bytes each kernel moves by its design, per launch
        "hist": 4 * n_conn + 4 * G * B,
        "offsets": 3 * 4 * G * B + 4 * (B + 1),
        "part": 4 * n_conn + rb * n_conn,
        "part_fine": 2 * rb * n_conn if two_level else 0,
        "bucket": rb * n_conn + 4 * (B + 1) + out_bytes,
        "place": 2 * (8 * (N + 1) + 4 * nnz["nodes"]) if "nodes" in nnz else 0,
    }
    peak, peak_src = measured_peaks()
    kernels = {k: v for k, v in stage.items() if k in KERNEL_OF_STAGE}
    dom = max(kernels, key=kernels.get)
    dom_ms = kernels[dom]
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            with open(tpath) as f:
                tr = json.load(f)
            key = f"{workload}:{want}:{KERNEL_OF_STAGE[dom]}"
            if key in tr and tr[key].get("source") == source_digest():
                traffic = tr[key]["bytes_per_launch"]
        except Exception:
            traffic = None
    gbs = lambda nbytes: nbytes / (dom_ms * 1e-3) / 1e9
    kernel = KERNEL_OF_STAGE[dom] if (dom != "part" or two_level) else "k_part"
    roof = {"bound": "hbm", "kernel": kernel, "achieved": gbs(compulsory), "peak": peak,
            "peak_source": f"{peak_src} copy bandwidth", "unit": "GB/s", "frac": gbs(compulsory) / peak,
            "traffic": traffic, "alg_bytes_per_launch": compulsory, "ms_per_launch": dom_ms,
            "alg_bytes": "compulsory bytes of one build: 4 n_conn + sum over CSRs of (8 (N+1) + 4 nnz)",
            "kernel_own_bytes_per_launch": own[dom],
            "kernel_own_bytes_frac": gbs(own[dom]) / peak,
            "ncu_dram_frac": (gbs(traffic) / peak) if traffic else None}
    return {"compulsory": compulsory, "peak": peak, "roofline": roof}


P99_TARGET_MS = 10.0  # the stated latency at which the two servers' throughputs are compared


def sustained_at_p99(loads, server, target_ms):
    """Throughput a server sustains at a stated p99: the requests per second
    it served at the highest offered load (key: load as a string) whose p99
    latency was at most target_ms; None if no load met it."""
    ok = [(float(ld), x[server]["req_per_s"]) for ld, x in loads.items() if x[server]["p99_ms"] <= target_ms]
    return max(ok)[1] if ok else None


def serving_summary(args):
    """A bounded serving run for the default line: the plain server's
    saturated rate R, then the same Poisson trace at 0.5, 0.8, 1.0, 1.2 and
    1.5 R served by one build per mesh (plain) and by continuous batching (two
    streams of at most two units in flight, batches from eight waiting
    requests, two batch slots); throughput and latency percentiles of each,
    and for each server the highest of these loads it sustains at a p99 of at
    most P99_TARGET_MS."""
    import copy
    from paper_1604_04689_gb300.serve import BatchServer, PlainServer, make_requests
    n = max(args.serve_requests, 100)
    base = make_requests(n, 0.0)
    big = max(base, key=lambda r: r.n_conn)
    plain = PlainServer(big)
    batched = BatchServer(budget_bytes=40 << 30, lanes=2)
    w = min(200, n)
    batched.warm(min(base, key=lambda r: r.n_conn))
    plain.run(copy.deepcopy(base[:w]))
    # the whole request set at once: every graph, batch size and buffer size
    # the timed runs will meet is seen (and cached by the allocator) first
    batched.run(copy.deepcopy(base))
    sat = plain.run(copy.deepcopy(base))
    keys = ("req_per_s", "melem_per_s", "p50_ms", "p99_ms", "p999_ms", "build_p99_ms", "failed")
    loads = {}
    for ld in (0.5, 0.8, 1.0, 1.2, 1.5):
        tr = make_requests(n, ld * sat["req_per_s"])
        rp = plain.run(copy.deepcopy(tr))
        rb = batched.run(copy.deepcopy(tr))
        loads[str(ld)] = {"rate_req_per_s": ld * sat["req_per_s"],
                          "plain": {k: rp.get(k) for k in keys}, "batched": {k: rb.get(k) for k in keys}}
    policy = {"streams": len(batched.streams), "depth": batched.depth, "batch_min": batched.batch_min,
              "batch_elems": batched.batch_elems,
              "batch_slots": len(batched.lanes)}
    del plain, batched

    return {"requests": n, "plain_saturated_req_per_s": sat["req_per_s"], "budget_bytes": 40 << 30,
            "policy": policy,
            "at_p99_target": {"p99_ms": P99_TARGET_MS,
                              "plain_req_per_s": sustained_at_p99(loads, "plain", P99_TARGET_MS),
                              "batched_req_per_s": sustained_at_p99(loads, "batched", P99_TARGET_MS)},
            "description": "tri / Kuhn tet / hex grid requests (1e3-2e6 elements, log-uniform, seeded), "
                           "connectivity generated on the device per request; latency = completion - arrival",
            "loads": loads}


E2E_SLOTS = 2  # buffer sets of the end-to-end pipeline: a build waits for the downloads two steps back


def end_to_end(torch, nn, b, mesh, dm, want, ws, ws_bytes, out, steps, dev, world):
    """Same metric through the C ABI with host buffers.  Every step copies its
    connectivity host -> device from pinned memory, builds, and copies both
    CSRs device -> host into pinned memory (row pointers, then the used part of
    col).  Steps are pipelined the way a host-fed service runs them: uploads on
    one stream, builds on another, row-pointer downloads on a third and column
    downloads on a fourth, E2E_SLOTS buffer sets, and the column downloads of step i
    enqueued once its row pointers (and so its sizes) have arrived, while step
    i + 1 uploads and builds.  (Row pointers and columns take separate streams:
    in one stream the row pointers of step i + 1, which wait for its build,
    would hold back the column downloads of step i queued behind them.)"""
    sA = torch.cuda.current_stream(dev)            # builds
    sU, sD = torch.cuda.Stream(dev), torch.cuda.Stream(dev)   # uploads, column downloads
    sR = torch.cuda.Stream(dev)                    # row-pointer downloads
    h_conn = torch.from_numpy(mesh.conn).pin_memory()
    slots = []
    for k in range(E2E_SLOTS):
        d_conn = torch.empty_like(dm.conn)
        o = out if k == 0 else b.alloc_outputs(dm, want)
        slots.append(dict(
            d_conn=d_conn, dm=nn.DeviceMesh(dm.etype, dm.n_nodes, d_conn, dm.elem_ptr, dm.elem_type), out=o,
            h_rp={c: torch.empty(rp.numel(), dtype=torch.int64, pin_memory=True) for c, (rp, _) in o.items()},
            h_col={c: torch.empty(col.numel(), dtype=torch.int32, pin_memory=True) for c, (_, col) in o.items()},
            up=torch.cuda.Event(), built=torch.cuda.Event(), rp=torch.cuda.Event(), done=torch.cuda.Event()))
        slots[-1]["done"].record(sA)
    counts = {"h2d": 0, "d2h": 0}

    def start(i):                                  # upload, build and row-pointer download of step i
        sl = slots[i % E2E_SLOTS]
        sU.wait_event(sl["built"])                 # the build E2E_SLOTS steps back has read this connectivity
        with torch.cuda.stream(sU):
            sl["d_conn"].copy_(h_conn, non_blocking=True)
        sl["up"].record(sU)
        sA.wait_event(sl["up"])
        sA.wait_event(sl["done"])                  # the downloads E2E_SLOTS steps back have read these outputs
        st = b.launch(sl["dm"], want, sl["out"], ws=ws, ws_bytes=ws_bytes, stream=sA)
        if st:
            raise nn.NNError(st, "launch")
        sl["built"].record(sA)
        sR.wait_event(sl["built"])
        sR.wait_event(sl["done"])                  # the host row pointers E2E_SLOTS steps back have been read
        with torch.cuda.stream(sR):
            for c, (rp, _) in sl["out"].items():
                sl["h_rp"][c].copy_(rp, non_blocking=True)
        sl["rp"].record(sR)
        counts["h2d"] += h_conn.numel() * 4

    def finish(i):                                 # column downloads of step i, sized by its row pointers
        sl = slots[i % E2E_SLOTS]
        sl["rp"].synchronize()
        sD.wait_event(sl["rp"])
        with torch.cuda.stream(sD):
            for c, (_, col) in sl["out"].items():
                n = int(sl["h_rp"][c][-1])
                sl["h_col"][c][:n].copy_(col[:n], non_blocking=True)
                counts["d2h"] += 8 * sl["h_rp"][c].numel() + 4 * n
        sl["done"].record(sD)

    start(0)
    finish(0)
    torch.cuda.synchronize(dev)
    link = host_link(torch, dev, slots[0], h_conn, sU, sD)
    counts["h2d"] = counts["d2h"] = 0
    t0 = time.perf_counter()
    for i in range(steps):
        start(i)
        if i > 0:
            finish(i - 1)
    finish(steps - 1)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    if int(b.status.item()) != 0:
        raise RuntimeError("device status after end-to-end leg: " + nn.STATUS[int(b.status.item())])
    ms = dt * 1e3 / steps
    link["frac"] = link["bound_ms_per_step"] / ms  # the step's share of its host-link bound
    return {"value": world * mesh.n_elems * steps / dt / 1e6, "unit": "Melem/s",
            "h2d_bytes_per_step": counts["h2d"] // steps, "d2h_bytes_per_step": counts["d2h"] // steps,
            "ms_per_step": ms, "pipelined": f"uploads, builds, row-pointer and column downloads on four streams, {E2E_SLOTS} buffer sets",
            "host_link": link}


def host_link(torch, dev, sl, h_conn, s_up, s_down):
    """The host link's own rate on one step's transfers: the connectivity
    upload alone, then the downloads of both CSRs alone (row pointers and the
    used part of col, as a step makes them), pinned memory, CUDA events on the
    copy stream, best of three.  A pipelined step cannot beat the slower of
    the two directions, so that time is the step's host-link bound."""
    def timed(stream, fn):
        best = float("inf")
        for _ in range(3):
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                nbytes = fn()
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best, nbytes

    def up():
        sl["d_conn"].copy_(h_conn, non_blocking=True)
        return h_conn.numel() * 4

    def down():
        nbytes = 0
        for c, (rp, col) in sl["out"].items():
            n = int(sl["h_rp"][c][-1])
            sl["h_rp"][c].copy_(rp, non_blocking=True)
            sl["h_col"][c][:n].copy_(col[:n], non_blocking=True)
            nbytes += 8 * rp.numel() + 4 * n
        return nbytes

    up_ms, up_b = timed(s_up, up)
    down_ms, down_b = timed(s_down, down)
    return {"h2d_gbs": up_b / (up_ms * 1e-3) / 1e9, "d2h_gbs": down_b / (down_ms * 1e-3) / 1e9,
            "bound_ms_per_step": max(up_ms, down_ms),
            "note": "each direction timed alone on this step's transfers; the step's bound is the slower one"}


def time_adjacency(torch, nn, b, dm, out, flush, stream, steps):
    """Element face adjacency from the node -> element CSR just built: CUDA-event time per call, L2 flushed."""
    rp_e, col_e = out["elems"]
    node_elems = (rp_e, col_e)
    rp, col = b.element_neighbors(dm, node_elems)          # sizes the output, checks the status
    ws_bytes, _ = nn.nn_element_neighbors_query(b.h, dm.struct())
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=rp.device)
    col_full = torch.empty(max(col.numel(), 1), dtype=torch.int32, device=rp.device)
    ne = nn.NNCSR(rp_e.data_ptr(), col_e.data_ptr(), col_e.numel())
    dst = nn.NNCSR(rp.data_ptr(), col_full.data_ptr(), col_full.numel())
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = nn.nn_element_neighbors(b.h, dm.struct(), ne, dst, ws.data_ptr(), ws_bytes, b.status.data_ptr(),
                                     stream.cuda_stream)
        e1.record(stream)
        if st:
            raise nn.NNError(st, "nn_element_neighbors")
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    assert int(b.status.item()) == 0
    ms = sorted(times)[len(times) // 2]
    return {"ms_median": ms, "melem_per_s": dm.n_elems / (ms * 1e-3) / 1e6, "nnz": int(col.numel()),
            "gpu_launches_per_call": 3, "steps": steps}


def max_over_ranks(x, world, device):
    """The slowest rank's time: every rank contributes, all receive the maximum."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n_elems, steps, world, total_ms):
    """Melem/s of the whole job: every replica builds the same mesh `steps` times within the slowest
    rank's time (weak scaling)."""
    return world * n_elems * steps / (total_ms * 1e-3) / 1e6


def launches_per_build(plan, want="both"):
    """Kernels one build launches: histogram, offsets, partition (one pass, or
    coarse + fine when the buckets span more than 256 coarse digits), bucket,
    and for node rows their placement (scan + copy)."""
    return 3 + (2 if plan["partition"] > 0 else 1) + (2 if want in ("both", "nodes") else 0)


# the sources that compile the single-mesh build's kernels and their launch
# plan: traffic counters taken on other sources no longer describe them
MEASURED_SOURCES = ("nn_api.cu", "nn_bucket.cu", "nn_bulk.cuh", "nn_compact.cu", "nn_device.cuh", "nn_emit.cu",
                    "nn_internal.h")


def source_digest():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1604_04689_gb300", "csrc")
    for f in MEASURED_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
