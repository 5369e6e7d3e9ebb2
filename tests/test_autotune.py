"""Autotuner host logic on the CPU: cache keys, the JSON cache, and the
coordinate-descent search (with a model standing in for the GPU timing)."""
import json

import pytest

from paper_1507_05086_gb300 import autotune


def test_graph_class_groups_by_size_degree_and_skew():
    a = autotune.graph_class(1 << 26, 2_103_822_292, 1_003_939)
    b = autotune.graph_class((1 << 26) + 1000, 2_100_000_000, 990_000)
    c = autotune.graph_class(1 << 24, 520_749_332, 406_524)
    assert a == b and a != c
    assert a.startswith("n2^26|") and "|d2^5|" in a


def test_cache_roundtrip_and_merge(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert autotune.load_cache(path) == {}
    autotune.store(path, "GB300|sm152|cc103", "rounds", "n2^26|d2^5|skew2^15", {"tuning": {"walk_batches": 2}, "ms": 1.0})
    autotune.store(path, "GB300|sm152|cc103", "batch", "count4096", {"tuning": {"batch_team_blocks": 16}, "ms": 2.0})
    autotune.store(path, "other", "rounds", "x", {"tuning": {}, "ms": 3.0})
    data = json.load(open(path))
    assert set(data) == {"GB300|sm152|cc103", "other"}
    assert autotune.lookup(path, "GB300|sm152|cc103", "rounds", "n2^26|d2^5|skew2^15")["tuning"] == {"walk_batches": 2}
    assert autotune.lookup(path, "GB300|sm152|cc103", "batch", "count4096")["ms"] == 2.0
    assert autotune.lookup(path, "GB300|sm152|cc103", "rounds", "missing") is None
    # a later store replaces one entry and keeps the others
    autotune.store(path, "GB300|sm152|cc103", "rounds", "n2^26|d2^5|skew2^15", {"tuning": {"walk_batches": 8}, "ms": 0.5})
    assert autotune.lookup(path, "GB300|sm152|cc103", "rounds", "n2^26|d2^5|skew2^15")["ms"] == 0.5
    assert autotune.lookup(path, "GB300|sm152|cc103", "batch", "count4096")["ms"] == 2.0


def test_corrupt_cache_reads_as_empty(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    assert autotune.load_cache(str(path)) == {}


def test_coordinate_descent_finds_the_separable_optimum():
    # a separable cost with its minimum at walk_batches=2, heavy_shift=2,
    # prefetch_ahead=0: every knob is visited once, in order
    opt = {"walk_batches": 2, "prefetch_ahead": 0, "heavy_shift": 2}
    seen = []

    def cost(s):
        seen.append(dict(s))
        return 10.0 + sum(abs(s[k] - v) for k, v in opt.items())

    start = {"walk_batches": 4, "prefetch_ahead": 2, "heavy_shift": 1}
    knobs = {k: autotune.ROUND_KNOBS[k] for k in start}
    best, best_ms, start_ms, evals = autotune.coordinate_descent(start, knobs, cost)
    assert best == opt and best_ms == 10.0 and start_ms == 15.0
    assert evals == len(seen) == 1 + sum(len(v) - 1 for v in knobs.values())


def test_coordinate_descent_keeps_the_default_without_a_real_gain():
    start = {"walk_batches": 4}
    best, best_ms, _, _ = autotune.coordinate_descent(
        start, {"walk_batches": (1, 2, 4, 8)}, lambda s: 100.0 - (0.5 if s["walk_batches"] == 8 else 0.0),
        min_gain=0.02)
    assert best == start and best_ms == 100.0


def test_coordinate_descent_stops_at_its_budget():
    calls = []
    autotune.coordinate_descent({"a": 0}, {"a": tuple(range(1, 1000))}, lambda s: calls.append(1) or 1.0,
                                budget_s=0.0)
    assert len(calls) == 1


def test_tuning_validation_without_gpu():
    cc = pytest.importorskip("paper_1507_05086_gb300")
    t = cc.default_tuning().to_dict()
    assert t["walk_batches"] == 4 and t["heavy_shift"] == 1 and t["batch_team_blocks"] == 8
    for k, bad in (("walk_batches", 0), ("walk_batches", 9), ("prefetch_ahead", -1), ("heavy_shift", 0),
                   ("heavy_shift", 5), ("inline_heavy", 70000), ("batch_team_blocks", 1),
                   ("batch_team_blocks", 17), ("batch_small_n", 0), ("warp_resolve_row", -1)):
        with pytest.raises(cc.CCError) as ei:
            cc.set_batch_tuning(dict(t, **{k: bad}))
        assert ei.value.status == -1
    with pytest.raises(cc.CCError):
        cc.set_batch_tuning(dict(t, batch_team_n=t["batch_small_n"] - 1))
    assert cc.get_batch_tuning() == t


def test_cache_path_from_environment(tmp_path, monkeypatch):
    monkeypatch.delenv("CC_TUNE_CACHE", raising=False)
    monkeypatch.delenv("CC_TUNING_CACHE", raising=False)
    assert autotune.default_cache_path().endswith("tuning.json")
    monkeypatch.setenv("CC_TUNING_CACHE", str(tmp_path / "b.json"))
    assert autotune.default_cache_path() == str(tmp_path / "b.json")
    monkeypatch.setenv("CC_TUNE_CACHE", str(tmp_path / "a.json"))
    assert autotune.default_cache_path() == str(tmp_path / "a.json")
