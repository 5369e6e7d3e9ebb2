#!/usr/bin/env python
"""Quality study of C4 and ClusterWild! on the synthetic stand-in graphs.

Sec. 6 of the paper reports, over 100 random orders per graph: the number of
synchronisation rounds against eps, the share of C4 actives that are blocked
(waiting on an earlier active neighbour; under 0.2 % on all its graphs), and
the objective of ClusterWild! against serial KwikCluster, which C4 returns
exactly (at most 1 % worse on all its graphs).  This script measures the same
quantities on the seeded synthetic graphs of ``graphgen`` through the C ABI:

* objective and rounds of every (graph, eps, permutation) job come from the
  batched entry point (``cc_batch_jobs``), C4 and ClusterWild! on the same
  permutations (seed_j = base + j);
* blocked counts come from the per-round statistics of ``cc_cluster_ex``
  (C4 on the first ``--stats-perms`` permutations), and for C4 without rounds
  (Alg. 3, ``CC_ALGO_C4_ASYNC``) from its one statistics record: the
  vertices that waited on an undecided earlier neighbour.  The paper finds
  fewer blocked vertices under the bulk-synchronous C4 than the asynchronous
  one; its objective must equal C4's (both are KwikCluster).

Prints one JSON object.  ``python quality.py --perms 100`` runs the paper's
protocol on the small graphs; the defaults finish in about a minute.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRAPHS = {
    "er10k": "G(n=10,000, p=20/9,999)",
    "planted1m": "planted partition, n=1e6, 2,000 Zipf clusters, 4M noise pairs",
    "rmat20": "R-MAT scale 20, edge factor 16",
}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--graphs", default="er10k,planted1m,rmat20")
    p.add_argument("--eps", default="0.1,0.5,0.9")
    p.add_argument("--perms", type=int, default=20, help="random orders per (graph, eps)")
    p.add_argument("--stats-perms", type=int, default=5, help="orders with per-round statistics (C4)")
    p.add_argument("--seed", type=int, default=100)
    return p.parse_args(argv)


def summarize(xs):
    import numpy as np
    a = np.asarray(xs, dtype=np.float64)
    return {"mean": float(a.mean()), "min": float(a.min()), "max": float(a.max())}


def study(cc, g, eps: float, perms: int, stats_perms: int, seed: int):
    import numpy as np
    seeds = np.array([seed], dtype=np.uint64)
    with cc.Graph(g.off, g.col) as graph:
        d4, r4 = cc.batch_jobs([graph], "c4", eps, seeds, perms)
        dw, rw = cc.batch_jobs([graph], "cw", eps, seeds, perms)
        d4, r4, dw, rw = (np.asarray(x).reshape(-1) for x in (d4, r4, dw, rw))
        blocked, blocked_async = [], []
        for j in range(min(stats_perms, perms)):
            _, _, d, st = graph.cluster("c4", eps, seed + j, want_labels=False, stats_cap=1_000_000)
            assert d == d4[j]
            blocked.append(float(st["blocked"].sum()) / g.n)
            _, _, da, sa = graph.cluster("c4-async", eps, seed + j, want_labels=False, stats_cap=1)
            assert da == d4[j]
            blocked_async.append(float(sa["blocked"][0]) / g.n)
    ratio = dw / np.maximum(d4, 1)
    return {
        "eps": eps,
        "perms": perms,
        "rounds_c4": summarize(r4),
        "rounds_cw": summarize(rw),
        "objective_c4_equals_kwikcluster": summarize(d4),
        "objective_cw": summarize(dw),
        "cw_over_c4": summarize(ratio),
        "cw_worse_by_pct_mean": float((ratio.mean() - 1) * 100),
        "c4_blocked_pct_of_vertices": summarize(np.asarray(blocked) * 100) if blocked else None,
        "c4_async_blocked_pct_of_vertices": summarize(np.asarray(blocked_async) * 100) if blocked_async else None,
    }


def main(argv=None):
    args = parse_args(argv)
    import graphgen
    import paper_1507_05086_gb300 as cc
    graphgen.build()
    out = {"study": "quality of C4 / ClusterWild! on synthetic stand-ins (objective, rounds, blocked)",
           "seed_base": args.seed, "results": []}
    t0 = time.perf_counter()
    for name in args.graphs.split(","):
        g = graphgen.workload(name)
        for eps in (float(e) for e in args.eps.split(",")):
            r = study(cc, g, eps, args.perms, args.stats_perms, args.seed)
            r.update({"graph": name, "graph_desc": GRAPHS.get(name, name), "n": g.n, "m": g.m})
            out["results"].append(r)
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out))


if __name__ == "__main__":
    main()
