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


def test_roofline_is_the_compulsory_bytes_over_the_dominant_kernel():
    plan = {"record_bytes": 16, "emit_ctas": 152, "n_buckets": 66308, "partition": 9}
    N, T, n_conn = 16_974_593, 16_777_216, 134_217_728
    nnz = {"nodes": 101_451_264, "elems": 134_217_728}
    stage = {"init": 0.01, "hist": 0.3, "offsets": 0.03, "part": 1.0, "part_fine": 1.4, "bucket": 2.4, "place": 0.2}
    acc = bench.roofline_accounting(plan, N, T, n_conn, nnz, stage, "hex257", "both")
    compulsory = 4 * n_conn + 2 * 8 * (N + 1) + 4 * (nnz["nodes"] + nnz["elems"])
    assert acc["compulsory"] == compulsory == 1_751_140_384  # 1751.1 MB: read conn once, write both CSRs once
    r = acc["roofline"]
    assert r["kernel"] == "k_bucket" and r["ms_per_launch"] == 2.4  # the slowest kernel stage ("init" is no kernel)
    assert abs(r["achieved"] - compulsory / 2.4e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["alg_bytes_per_launch"] == compulsory
    own = 16 * n_conn + 4 * (66308 + 1) + compulsory - 4 * n_conn
    assert r["kernel_own_bytes_per_launch"] == own
    # the fine partition as the slowest stage is named for its own kernel
    stage["part_fine"] = 3.0
    assert bench.roofline_accounting(plan, N, T, n_conn, nnz, stage, "hex257", "both")["roofline"]["kernel"] == \
        "k_part_fine"


def test_oracle_samples_match_the_workload_kind():
    mesh, desc, ratio = bench.oracle_sample("hex257")
    assert mesh.etype == 3 and "hex grid 101^3" in desc and abs(ratio - 100 ** 3 / 256 ** 3) < 1e-12
    mesh, desc, ratio = bench.oracle_sample("tri2048")
    assert mesh.etype == 0 and abs(ratio - mesh.n_elems / 8_380_418) < 1e-12


def test_throughput_at_a_stated_p99_is_the_highest_load_within_it():
    loads = {"0.5": {"plain": {"req_per_s": 2700.0, "p99_ms": 2.6}, "batched": {"req_per_s": 2701.0, "p99_ms": 2.4}},
             "0.8": {"plain": {"req_per_s": 4300.0, "p99_ms": 4.6}, "batched": {"req_per_s": 4310.0, "p99_ms": 4.6}},
             "1.0": {"plain": {"req_per_s": 5280.0, "p99_ms": 11.4}, "batched": {"req_per_s": 5365.0, "p99_ms": 7.2}},
             "1.5": {"plain": {"req_per_s": 5560.0, "p99_ms": 113.0}, "batched": {"req_per_s": 5960.0, "p99_ms": 90.5}}}
    assert bench.sustained_at_p99(loads, "plain", 10.0) == 4300.0
    assert bench.sustained_at_p99(loads, "batched", 10.0) == 5365.0
    assert bench.sustained_at_p99(loads, "batched", 100.0) == 5960.0   # a later load within the bound counts
    assert bench.sustained_at_p99(loads, "plain", 1.0) is None
