"""Host logic of the autotuner: cache file round trip and workload keys (no GPU)."""
import json

from paper_2607_23122_gb300 import autotune


def test_cache_round_trip_and_bad_files(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("OCC_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune.load_cache() == {}                      # missing file
    entry = {"best": {"reuse_tile_rows": 8, "reuse_window_path": 1},
             "timings": [{"config": {}, "ms": 0.5}]}
    autotune.save_cache({"k": entry})
    assert autotune.load_cache() == {"k": entry}
    assert json.loads(path.read_text()) == {"k": entry}
    assert not [p for p in path.parent.iterdir() if ".tmp" in p.name]
    path.write_text("{not json")
    assert autotune.load_cache() == {}                      # corrupt file: start over


def test_candidates_are_valid_tuning_values():
    for c in autotune.REUSE_CANDIDATES:
        assert c["reuse_tile_rows"] in (0, 4, 8, 16) and c["reuse_window_path"] in (1, 2, 3)
    assert all(0 <= c["batch_ctas_per_sm"] <= 16 for c in autotune.BATCH_CANDIDATES)
    assert all(c["group_prefetch"] in (1, 2, 3) for c in autotune.GROUP_CANDIDATES)
    for c in autotune.TRACE_CANDIDATES:
        assert c["trace_path"] in (1, 2)
        assert 0 <= c.get("trace_refill", 0) <= 32 and 0 <= c.get("trace_ctas_per_sm", 0) <= 16
        assert c.get("trace_order", 0) in (0, 1, 2)


def test_layout_candidates_and_key():
    assert autotune.LAYOUT_CANDIDATES == ("linear", "tiled")

    class _Pat:
        kind, gw, gh, K = 2, 0, 0, 8

    class _Buf:
        W, H, packed = 1920, 1080, False

    key = autotune.layout_key(_Buf(), _Buf(), _Pat(), 1, 0)
    assert key.startswith("layout/1920x1080/") and "K8" in key and "est1" in key
    # a different pattern or estimator is a different workload
    assert key != autotune.layout_key(_Buf(), _Buf(), _Pat(), 2, 0)
