"""Autotuner host logic (no GPU needed): keys, buckets, the selection rule and the JSON cache."""
from paper_1402_2020_gb300 import autotune


def test_bucket_and_key():
    assert [autotune.bucket(v) for v in (1, 2, 3, 64, 65, 1390 * 1110)] == [1, 2, 4, 64, 128, 2 ** 21]
    k1 = autotune.key("GB300", 256, 5, 1390, 1110, 256)
    k2 = autotune.key("GB300", 256, 5, 1400, 1100, 200)
    assert k1 == k2 == "GB300|n256|win5|d256|px2097152|v4"
    assert autotune.key("GB300", 256, 5, 3840, 2160, 256) != k1


def test_choose_picks_fastest_and_keeps_first_on_ties():
    t = {16: 3.0, 32: 2.0, 64: 2.0, 128: 5.0}
    best, timings = autotune.choose([16, 32, 64, 128], lambda c: t[c])
    assert best == 32 and timings == {"16": 3.0, "32": 2.0, "64": 2.0, "128": 5.0}


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("BSM_AUTOTUNE_CACHE", str(tmp_path / "sub" / "cache.json"))
    assert autotune.load() == {}
    autotune.store({"a": {"cost_rows": 64}})
    assert autotune.load() == {"a": {"cost_rows": 64}}
    (tmp_path / "sub" / "cache.json").write_text("{not json")
    assert autotune.load() == {}
