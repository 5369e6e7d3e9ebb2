"""Autotuner for the schedule settings of the library (cc_tuning).

The settings cut the work differently (edge-walker chunks and prefetch
depth, which heavy-list scans, Delta rebuild segments and C4 blocked sets
run inside a grid barrier, the heavy-list threshold, and the size classes
and team size of batched jobs); none changes a result.  This module picks
them by measurement, per device and per class of graph, and keeps the
choices in a JSON cache so that a later process reuses them:

    cache[device key]["rounds"][graph class] = {"tuning": {...}, "ms": ..., "default_ms": ...}
    cache[device key]["batch"][workload class] = {...}

The search is coordinate descent from the defaults: for each setting in
turn, every candidate value is timed with the others held, and the best one
is kept when it beats the current choice by more than `min_gain`.  Every
measured run is also checked against the default settings' results (rounds
and disagreements; they must be identical), so a tuned setting can never
change an output.  Timing goes through an `evaluate` callable, which the
CPU tests replace by a model.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
import time

from . import native

ROUND_KNOBS = {
    "walk_batches": (1, 2, 4, 8),
    "prefetch_ahead": (0, 1, 2, 4),
    "heavy_shift": (1, 2),
    "inline_heavy": (2048, 8192, 32768),
    "inline_rebuild": (2048, 8192, 32768),
    "inline_decide": (1024, 4096, 16384),
    "warp_resolve_row": (256, 1024, 4096),
}
BATCH_KNOBS = {
    "batch_team_blocks": (4, 8, 16),
    "batch_small_n": (1 << 14, 1 << 15, 1 << 16, 1 << 17),
}


def default_cache_path() -> str:
    """$CC_TUNE_CACHE (or $CC_TUNING_CACHE), else a file under ~/.cache."""
    for var in ("CC_TUNE_CACHE", "CC_TUNING_CACHE"):
        if os.environ.get(var):
            return os.environ[var]
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1507_05086_gb300", "tuning.json")


def device_key() -> str:
    """Device name, SM count and compute capability of the current GPU."""
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}|cc{p.major}{p.minor}"


def graph_class(n: int, nnz: int, max_degree: int) -> str:
    """Graphs that share a class are expected to share their best settings:
    size (log2 of n), mean degree (log2) and skew (log2 of the largest
    degree over the mean)."""
    mean = max(nnz / max(n, 1), 1.0)
    skew = max(max_degree / mean, 1.0)
    return f"n2^{round(math.log2(max(n, 1)))}|d2^{round(math.log2(mean))}|skew2^{round(math.log2(skew))}"


def load_cache(path: str | None = None) -> dict:
    path = path or default_cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(path: str | None, dev: str, kind: str, cls: str, entry: dict) -> None:
    """Merge one entry into the cache file (atomic replace)."""
    path = path or default_cache_path()
    data = load_cache(path)
    data.setdefault(dev, {}).setdefault(kind, {})[cls] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(path: str | None, dev: str, kind: str, cls: str):
    return load_cache(path).get(dev, {}).get(kind, {}).get(cls)


def coordinate_descent(start: dict, knobs: dict, evaluate, min_gain: float = 0.02, budget_s: float = 60.0):
    """Minimise evaluate(settings) -> ms over the candidate values of each knob
    in turn, from `start`.  Returns (best settings, best ms, start ms,
    evaluations)."""
    t_end = time.perf_counter() + budget_s
    best = dict(start)
    best_ms = start_ms = evaluate(best)
    seen = {tuple(sorted(best.items())): best_ms}      # a setting is timed once
    for knob, values in knobs.items():
        for v in values:
            cand = dict(best, **{knob: v})
            key = tuple(sorted(cand.items()))
            if key in seen or time.perf_counter() > t_end:
                continue
            ms = seen[key] = evaluate(cand)
            if ms < best_ms * (1.0 - min_gain):
                best, best_ms = cand, ms
    return best, best_ms, start_ms, len(seen)


def _rounds_evaluator(graph, algos, eps, seeds, reps):
    """Mean round-kernel time of the graph's clusterings under a setting; the
    first call's results are the reference every later call must match."""
    ref = {}

    def evaluate(settings):
        graph.set_tuning(settings)
        total = 0.0
        for a in algos:
            for s in seeds:
                for _ in range(reps):
                    _, r, d = graph.cluster(a, eps, s, want_labels=False)
                    total += graph.last_timings()[1]
                    key = (a, s)
                    if key in ref and ref[key] != (r, d):
                        raise AssertionError(f"tuning {settings} changed the result of {key}")
                    ref[key] = (r, d)
        return total / (len(algos) * len(seeds) * reps)

    return evaluate


def tune_rounds(graph, algos=("cw", "c4"), eps: float = 0.5, seeds=(101, 202), reps: int = 1,
                cache: str | None = None, budget_s: float = 30.0, force: bool = False, knobs=None):
    """Settings of the round kernel for this graph's class on this device:
    from the cache, else by coordinate descent (then stored).  Leaves the
    graph tuned.  Returns the cache entry with a "source" field."""
    dev = device_key()
    cls = graph_class(graph.n, graph.nnz, graph.max_degree)
    hit = None if force else lookup(cache, dev, "rounds", cls)
    if hit is not None:
        graph.set_tuning(hit["tuning"])
        return dict(hit, source="cache", graph_class=cls, device=dev)
    graph.set_timing(True)
    evaluate = _rounds_evaluator(graph, algos, eps, seeds, reps)
    start = {k: v for k, v in native.default_tuning().to_dict().items() if k in (knobs or ROUND_KNOBS)}
    best, best_ms, start_ms, evals = coordinate_descent(start, knobs or ROUND_KNOBS, evaluate, budget_s=budget_s)
    graph.set_tuning(best)
    entry = {"tuning": best, "ms": best_ms, "default_ms": start_ms, "evaluations": evals,
             "algos": list(algos), "eps": eps, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    store(cache, dev, "rounds", cls, entry)
    return dict(entry, source="tuned now", graph_class=cls, device=dev)


def batch_class(graphs) -> str:
    ns = sorted(g.n for g in graphs)
    return (f"count{len(graphs)}|n2^{round(math.log2(max(ns[0], 1)))}-2^{round(math.log2(max(ns[-1], 1)))}"
            f"|median2^{round(math.log2(max(ns[len(ns) // 2], 1)))}")


def tune_batch(graphs, algo: str = "cw", eps: float = 0.5, k_perms: int = 2, cache: str | None = None,
               budget_s: float = 60.0, force: bool = False, knobs=None):
    """Size classes and team size of batched jobs for a batch like `graphs`
    (timed on those graphs, k_perms permutations each): from the cache, else
    by coordinate descent.  Applies the choice process-wide
    (cc_set_batch_tuning) and returns the cache entry."""
    import numpy as np
    import torch
    dev = device_key()
    cls = batch_class(graphs)
    hit = None if force else lookup(cache, dev, "batch", cls)
    base = native.default_tuning().to_dict()
    if hit is not None:
        native.set_batch_tuning(dict(base, **hit["tuning"]))
        return dict(hit, source="cache", batch_class=cls, device=dev)
    seeds = np.arange(len(graphs), dtype=np.uint64) * 7 + 1
    ref = {}

    def evaluate(settings):
        native.set_batch_tuning(dict(base, **settings))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D, R = native.batch_jobs(graphs, algo, eps, seeds, k_perms)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        if "D" in ref and not (np.array_equal(ref["D"], D) and np.array_equal(ref["R"], R)):
            raise AssertionError(f"batch tuning {settings} changed a result")
        ref["D"], ref["R"] = D, R
        return ms

    start = {k: base[k] for k in (knobs or BATCH_KNOBS)}
    best, best_ms, start_ms, evals = coordinate_descent(start, knobs or BATCH_KNOBS, evaluate, budget_s=budget_s)
    native.set_batch_tuning(dict(base, **best))
    entry = {"tuning": best, "ms": best_ms, "default_ms": start_ms, "evaluations": evals, "algo": algo,
             "k_perms": k_perms, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    store(cache, dev, "batch", cls, entry)
    return dict(entry, source="tuned now", batch_class=cls, device=dev)
