"""Host logic of the autotuner (no GPU): cache keys, size classes, the JSON
cache, the candidate list (distinct plans, the automatic one first) on an
offline handle, and a cached mesh class applied without timing."""
import json

from paper_1604_04689_gb300 import autotune as at


def test_size_class_is_log2_floor():
    assert at.size_class(0) == 0 and at.size_class(1) == 0
    assert at.size_class(1023) == 9 and at.size_class(1024) == 10
    assert at.size_class(8_388_608) == 23


def test_cache_key_separates_device_type_size_and_want():
    keys = {at.cache_key(d, t, n, w) for d in ("A", "B") for t in (0, 2) for n in (1000, 5000) for w in (1, 3)}
    assert len(keys) == 16
    assert at.cache_key("A", 0, 1025, 3) == at.cache_key("A", 0, 2047, 3)


def test_cache_roundtrip_and_merge(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    assert at.load_cache(path) == {}
    t1 = {"sb": 8, "bucket_threads": 256, "bucket_ctas_per_sm": 4}
    at.store_cache({"k1": {"tuning": t1}}, path)
    at.store_cache({"k2": {"tuning": {"sb": 0, "bucket_threads": 0, "bucket_ctas_per_sm": 0}}}, path)
    d = at.load_cache(path)
    assert d["k1"]["tuning"] == t1 and set(d) == {"k1", "k2"}
    with open(path) as f:
        assert json.load(f) == d


def test_corrupt_cache_reads_empty(tmp_path, monkeypatch):
    path = tmp_path / "c.json"
    path.write_text("{not json")
    monkeypatch.setenv("NN_AUTOTUNE_CACHE", str(path))
    assert at.cache_path() == str(path)
    assert at.load_cache() == {}


class _OfflineBuilder:
    """What candidates() and tuned() use of a Builder: its handle (offline here)."""

    def __init__(self):
        from paper_1604_04689_gb300 import build, nn
        build.build()
        self.h = nn.nn_create_offline()
        self.device = "cpu"


class _Mesh:
    def __init__(self, etype, n_nodes, n_elems):
        from paper_1604_04689_gb300 import nn
        self.etype, self.n_nodes, self.n_elems = etype, n_nodes, n_elems
        self.n_conn = n_elems * nn.NPE[etype]

    def struct(self):
        from paper_1604_04689_gb300 import nn
        return nn.NNMesh(self.etype, self.n_nodes, self.n_elems, self.n_conn, 1 << 20, None, None)


def test_candidates_are_distinct_valid_plans_with_the_automatic_first():
    from paper_1604_04689_gb300 import nn
    b = _OfflineBuilder()
    try:
        for m in (_Mesh(nn.TRI, 4_194_304, 8_380_418), _Mesh(nn.TET, 4_173_281, 24_576_000),
                  _Mesh(nn.HEX, 300_000, 290_000)):
            auto = nn.nn_plan_info(b.h, m.struct(), nn.WANT_BOTH)
            cands = at.candidates(b, m, nn.WANT_BOTH)
            assert cands[0] == {"sb": 0, "bucket_threads": 0, "bucket_ctas_per_sm": 0}
            assert len(cands) > 3
            sigs = set()
            for t in cands:
                nn.nn_set_tuning(b.h, t)
                p = nn.nn_plan_info(b.h, m.struct(), nn.WANT_BOTH)
                assert 4 <= p["sb"] <= 11 and p["bucket_threads"] in (128, 256)
                sigs.add((p["sb"], p["bucket_threads"], p["bucket_smem"]))
            assert len(sigs) == len(cands)                    # no two candidates time the same plan
            nn.nn_set_tuning(b.h, None)
            assert nn.nn_plan_info(b.h, m.struct(), nn.WANT_BOTH) == auto   # candidates() left the handle automatic
    finally:
        nn.nn_destroy(b.h)


def test_tuned_applies_a_cached_entry_without_timing(tmp_path, monkeypatch):
    import torch
    from paper_1604_04689_gb300 import nn
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "FakeGPU")

    def no_timing(*a, **k):
        raise AssertionError("a cached class must not be re-timed")
    monkeypatch.setattr(at, "tune", no_timing)
    b = _OfflineBuilder()
    try:
        m = _Mesh(nn.TRI, 1_000_000, 1_990_000)
        t = {"sb": 6, "bucket_threads": 128, "bucket_ctas_per_sm": 4}
        path = str(tmp_path / "c.json")
        at.store_cache({at.cache_key("FakeGPU", m.etype, m.n_elems, nn.WANT_BOTH): {"tuning": t}}, path)
        assert at.tuned(b, m, nn.WANT_BOTH, path=path) == t
        p = nn.nn_plan_info(b.h, m.struct(), nn.WANT_BOTH)
        assert (p["sb"], p["bucket_threads"]) == (6, 128)        # the cached tuning is applied to the handle
    finally:
        nn.nn_destroy(b.h)
