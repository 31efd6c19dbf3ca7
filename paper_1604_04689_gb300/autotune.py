"""Autotuner for the build's launch shape.

Times candidate launch tunings of the bucket pass -- threads per CTA, bucket
CTAs per SM (which sets the shared memory each CTA may use) and the bucket
width around the planner's choice -- on a mesh, keeps the fastest, and caches
it per (GPU, element type, log2 of the element count, wanted results) in a
JSON file (``NN_AUTOTUNE_CACHE``, default ``~/.cache/nn_autotune.json``).
Results never depend on the tuning; only speed and workspace size do.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

from . import nn

# (threads per bucket CTA, bucket CTAs per SM)
SHAPES = ((256, 1), (256, 2), (128, 2), (128, 4), (128, 6))
SB_DELTAS = (-1, 0, 1)


def cache_path() -> str:
    return os.environ.get("NN_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "nn_autotune.json"))


def size_class(n_elems: int) -> int:
    return int(math.log2(max(int(n_elems), 1)))


def cache_key(device_name: str, etype: int, n_elems: int, want: int) -> str:
    return f"{device_name}|type={etype}|log2elems={size_class(n_elems)}|want={want}"


def load_cache(path: Optional[str] = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path: Optional[str] = None) -> None:
    path = path or cache_path()
    d = load_cache(path)
    d.update(entries)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(builder: "nn.Builder", dm: "nn.DeviceMesh", want: int):
    """Distinct candidate tunings (the automatic one first)."""
    out, seen = [], set()
    nn.nn_set_tuning(builder.h, None)
    auto = nn.nn_plan_info(builder.h, dm.struct(), want)
    out.append({"sb": 0, "bucket_threads": 0, "bucket_ctas_per_sm": 0})
    seen.add((auto["sb"], auto["bucket_threads"], auto["bucket_smem"]))
    for threads, cps in SHAPES:
        nn.nn_set_tuning(builder.h, {"bucket_threads": threads, "bucket_ctas_per_sm": cps})
        base = nn.nn_plan_info(builder.h, dm.struct(), want)
        for d in SB_DELTAS:
            sb = base["sb"] + d
            if not 4 <= sb <= 11:
                continue
            t = {"sb": sb, "bucket_threads": threads, "bucket_ctas_per_sm": cps}
            try:
                nn.nn_set_tuning(builder.h, t)
                plan = nn.nn_plan_info(builder.h, dm.struct(), want)
            except nn.NNError:
                continue
            sig = (plan["sb"], plan["bucket_threads"], plan["bucket_smem"])
            if sig not in seen:
                seen.add(sig)
                out.append(t)
    nn.nn_set_tuning(builder.h, None)
    return out


def tune(builder: "nn.Builder", dm: "nn.DeviceMesh", want: int = nn.WANT_BOTH, reps: int = 3,
         cands=None, verify=None, flush_bytes: int = 256 << 20):
    """Time every candidate on this mesh; apply and return (best tuning, [(tuning, ms)]).

    Each timed build starts with L2 flushed (a write of ``flush_bytes``), as a
    build of a mesh that was just produced elsewhere would.  ``verify(out)``
    (optional) is called on each candidate's outputs."""
    import torch
    cands = cands or candidates(builder, dm, want)
    stream = torch.cuda.current_stream(builder.device)
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device=builder.device)
    results = []
    out = builder.alloc_outputs(dm, want)
    for t in cands:
        nn.nn_set_tuning(builder.h, t)
        ws_bytes = builder.query(dm, want)[0]
        ws = builder.workspace(ws_bytes)
        if builder.launch(dm, want, out, ws=ws, ws_bytes=ws_bytes) != 0:
            continue
        torch.cuda.synchronize(builder.device)
        if int(builder.status.item()) != 0:
            continue
        if verify is not None:
            verify(out)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            builder.launch(dm, want, out, ws=ws, ws_bytes=ws_bytes)
            e1.record(stream)
        torch.cuda.synchronize(builder.device)
        if int(builder.status.item()) != 0:
            continue
        results.append((t, min(e0.elapsed_time(e1) for e0, e1 in ev)))
    if not results:
        raise RuntimeError("autotune: no candidate built this mesh")
    best = min(results, key=lambda r: r[1])[0]
    nn.nn_set_tuning(builder.h, best)
    return best, results


def tuned(builder: "nn.Builder", dm: "nn.DeviceMesh", want: int = nn.WANT_BOTH, path: Optional[str] = None,
          retune: bool = False) -> dict:
    """Apply the cached tuning for this mesh class, tuning (and caching) it first if absent."""
    import torch
    name = torch.cuda.get_device_name(builder.device)
    key = cache_key(name, dm.etype, dm.n_elems, want)
    cache = load_cache(path)
    if key in cache and not retune:
        nn.nn_set_tuning(builder.h, cache[key]["tuning"])
        return cache[key]["tuning"]
    best, results = tune(builder, dm, want)
    store_cache({key: {"tuning": best, "ms": {json.dumps(t, sort_keys=True): ms for t, ms in results}}}, path)
    return best
