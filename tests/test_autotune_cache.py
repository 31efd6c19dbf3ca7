"""Host logic of the autotuner: cache keys, size classes and the JSON cache
(no GPU)."""
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
