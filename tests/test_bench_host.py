"""Host arithmetic of the benchmark line (no GPU): kernels per build, the
roofline peak and its fallback, and the source digest that keeps stale
traffic counters out of the line."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_launches_per_build():
    # histogram, offsets, partition (1 or 2 passes), bucket, and for node rows their placement (2)
    assert bench.launches_per_build({"partition": 6}, "both") == 7
    assert bench.launches_per_build({"partition": 0}, "both") == 6
    assert bench.launches_per_build({"partition": -1}, "nodes") == 6
    assert bench.launches_per_build({"partition": 3}, "elems") == 5


def test_whole_job_value_is_weak_scaling():
    one = bench.whole_job_value(8_380_418, 20, 1, 22.0)
    assert abs(one - 8_380_418 * 20 / 0.022 / 1e6) < 1e-6
    assert abs(bench.whole_job_value(8_380_418, 20, 4, 22.0) - 4 * one) < 1e-6


def test_peak_is_the_measured_copy_bandwidth_else_the_fallback(tmp_path, monkeypatch):
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        import json
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            want = float(json.load(f)["hbm_gbs"])
        assert bench.measured_peaks() == (want, "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")


def test_source_digest_follows_only_the_measured_sources(tmp_path, monkeypatch):
    csrc = os.path.join(ROOT, "paper_1604_04689_gb300", "csrc")
    copy = tmp_path / "paper_1604_04689_gb300" / "csrc"
    shutil.copytree(csrc, copy)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.source_digest()
    assert d0 == bench.source_digest()
    (copy / "nn_diag.cu").write_text("// not a measured source\n")
    assert bench.source_digest() == d0
    with open(copy / "nn_bucket.cu", "a") as f:
        f.write("\n")
    assert bench.source_digest() != d0


def test_load_workload_generated_and_from_file(tmp_path, monkeypatch):
    from paper_1604_04689_gb300 import meshgen as mg
    from paper_1604_04689_gb300 import meshio
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "tri64"])
    name, desc, mesh = bench.load_workload(bench.parse())
    assert name == "tri64" and desc == bench.WORKLOADS["tri64"][1] and mesh.n_elems == 7938
    path = tmp_path / "bunny.ply"
    meshio.write_ply(mg.tri_grid(50, 2), str(path))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--mesh-file", str(path)])
    name, desc, mesh = bench.load_workload(bench.parse())
    assert name == "file:bunny.ply" and "2500 vertices, 4802 faces" in desc
    assert mesh.etype == mg.TRI and mesh.n_nodes == 2500
