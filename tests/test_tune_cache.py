"""The autotuner's result cache and candidate set (host logic, no GPU): a
cached workload signature returns its (tile, batch) choice and timings
without timing anything."""
import json

from paper_2509_25191_gb300 import tune


def test_cached_signature_short_circuits_the_search(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"GB300|n2^20|v1|px2^20|sh3": {"best": "32x16/2.1",
                                                               "ms": {"32x16/2.1": 0.87, "16x16/1.1": 0.93}}}))
    monkeypatch.setattr(tune, "signature", lambda g, views: "GB300|n2^20|v1|px2^20|sh3")

    def no_step(*a, **k):
        raise AssertionError("a cached signature must not build a step")

    monkeypatch.setattr(tune, "GraphStep", no_step)
    best, times = tune.autotune(None, None, None, cache_path=str(path))
    assert best == tune.Choice((32, 16), (2, 1)) and best.tile == (32, 16) and best.batch == (2, 1)
    assert times == {tune.Choice((32, 16), (2, 1)): 0.87, tune.Choice((16, 16), (1, 1)): 0.93}


def test_candidates_cover_every_tile_and_batch():
    cands = tune.candidates()
    assert len(cands) == len(tune.TILES) * len(tune.BATCHES) == len(set(cands))
    assert tune.Choice((32, 16), tune.DEFAULT_BATCH) in cands
    for c in cands:
        assert tune.parse_key(tune.key_str(c)) == c


def test_unreadable_cache_is_ignored(tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tune._load(str(bad)) == {} and tune._load(str(tmp_path / "missing.json")) == {}
