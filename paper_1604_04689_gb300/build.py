"""Compile libnn.so (CUDA, sm_103a) in-tree with nvcc.

The translation units are compiled in parallel and linked with the static
CUDA runtime; the result sits next to this file as ``libnn.so``.  With
``checked=True`` the same sources are compiled with -DNN_CHECKED into
``libnn_checked.so``: every computed global index of the build's kernels is
tested against its buffer's length, and a violation sets NN_ERR_BOUNDS in the
device status and skips the access (for testing; slower).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libnn.so")
LIB_CHECKED = os.path.join(HERE, "libnn_checked.so")
SOURCES = ["nn_emit.cu", "nn_bucket.cu", "nn_batch.cu", "nn_compact.cu", "nn_adj.cu", "nn_api.cu", "nn_noalloc.cu",
           "nn_gen.cu", "nn_diag.cu", "nn_submit.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out_dir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    flags = FLAGS + (["-DNN_CHECKED"] if checked else [])
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "nn.h"))
    nvcc = _nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src[:-3] + ".o")
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc, *ARCH, *flags, "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for cmd, r in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or r.returncode:
                print(" ".join(cmd)); print(r.stdout); print(r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    objs = [os.path.join(out_dir, s[:-3] + ".o") for s in SOURCES]
    if force or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        r = subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs],
                           capture_output=True, text=True)
        if r.returncode:
            print(r.stdout, r.stderr)
            raise RuntimeError(f"link of {os.path.basename(lib)} failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
