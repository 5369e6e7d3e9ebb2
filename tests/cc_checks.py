"""Independent checks shared by the CPU and GPU tests.

Each helper recomputes a property straight from its definition in the paper,
without calling the oracle's round code, so that a mistake in either side
shows up as a mismatch.
"""
from __future__ import annotations

import itertools

import numpy as np


def neighbours(off, col, v):
    return col[off[v]:off[v + 1]]


def check_partition_invariants(off, col, labels, order=None):
    """Output invariants of any peeling algorithm (Alg. 1 / Alg. 2 output):
    every vertex has one label; the label is a vertex that labels itself (a
    center); a non-center is adjacent to its center."""
    n = off.size - 1
    labels = np.asarray(labels)
    assert labels.shape == (n,)
    if n == 0:
        return
    assert labels.min() >= 0 and labels.max() < n
    assert np.all(labels[labels] == labels), "a center must be in its own cluster"
    for v in np.nonzero(labels != np.arange(n))[0]:
        c = labels[v]
        nb = neighbours(off, col, v)
        i = np.searchsorted(nb, c)
        assert i < nb.size and nb[i] == c, f"vertex {v} is not adjacent to its center {c}"


def removal_rounds(labels, active_round):
    """Round in which each vertex left the graph: the round its center was active."""
    return np.asarray(active_round)[np.asarray(labels)]


def check_round_structure(off, col, order, labels, active_round, stats, eps_ppm, algo,
                          batch_size, max_vertices_for_delta=200_000):
    """Re-derive n_i, Delta_i, k_i and A_i of every round from the final labels
    and the recorded active rounds (Alg. 2), and compare with the stats.

    A_i must be the first k_i vertices of pi among those alive at round i,
    k_i = batch_size(eps_ppm, n_i, Delta_i), Delta_i = the maximum number of
    alive neighbours of an alive vertex.
    """
    n = off.size - 1
    labels = np.asarray(labels)
    ar = np.asarray(active_round)
    rr = removal_rounds(labels, ar)
    R = int(rr.max()) + 1 if n else 0
    assert stats is None or len(stats["k"]) == R
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    src = np.repeat(np.arange(n), np.diff(off))
    for i in range(R):
        alive = rr >= i
        n_i = int(alive.sum())
        if n <= max_vertices_for_delta:
            both = alive[src] & alive[col]
            resid = np.bincount(src[both], minlength=n)
            delta = int(resid[alive].max()) if n_i else 0
        else:
            delta = int(stats["delta"][i])
        k = batch_size(eps_ppm, n_i, delta)
        act = np.nonzero(ar == i)[0]
        assert act.size == k, (i, act.size, k)
        alive_by_rank = order[alive[order]]
        assert np.array_equal(np.sort(act), np.sort(alive_by_rank[:k])), f"round {i}: A is not a pi-prefix"
        if stats is not None:
            assert stats["n_alive"][i] == n_i
            assert stats["delta"][i] == delta
            assert stats["k"][i] == k
            assert stats["removed"][i] == int((rr == i).sum())
            centers = act if algo == 2 else act[labels[act] == act]
            assert stats["centers"][i] == centers.size
    return R


def check_min_rank_center(off, col, order, labels, active_round, algo):
    """Concurrency rule 2 (Sec. 2.1): a clustered non-center joins the
    lowest-ranked center among its neighbours that were centers in its removal
    round.  C4 centers form an independent set; ClusterWild! centers are
    adjacent only inside one active set (Sec. 2.2)."""
    n = off.size - 1
    labels = np.asarray(labels)
    ar = np.asarray(active_round)
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    is_center = labels == np.arange(n)
    rr = removal_rounds(labels, ar)
    for v in range(n):
        nb = neighbours(off, col, v)
        if is_center[v]:
            cn = nb[is_center[nb]]
            if algo == 1:
                # C4: no two adjacent centers at all (KwikCluster's output)
                assert cn.size == 0, f"C4 centers {v} and {cn[:3]} are adjacent"
            else:
                assert np.all(ar[cn] == ar[v]), "CW centers adjacent across rounds"
            continue
        cand = nb[is_center[nb] & (ar[nb] == rr[v])]
        assert cand.size > 0
        best = cand[np.argmin(rank[cand])]
        assert labels[v] == best, f"vertex {v}: label {labels[v]} is not min-rank center {best}"


def noisy_graph(off, col, active_round):
    """G-hat (Sec. 3.2): G with every edge between two vertices that were
    active in the same round deleted."""
    n = off.size - 1
    ar = np.asarray(active_round)
    src = np.repeat(np.arange(n), np.diff(off))
    keep = ~((ar[src] >= 0) & (ar[src] == ar[col]))
    cnt = np.bincount(src[keep], minlength=n)
    off2 = np.zeros(n + 1, np.int64)
    np.cumsum(cnt, out=off2[1:])
    return off2, col[keep].astype(np.int32)


def peeling_cost_by_bad_triangles(adj, order, labels):
    """Lemma (cost of a peeling algorithm, Sec. 3.2 and its appendix proof):
    the disagreements equal, summed over the centers in peeling order, the
    bad triangles of the still-unclustered graph that contain the center.
    adj: dense 0/1 matrix."""
    n = adj.shape[0]
    labels = np.asarray(labels)
    remaining = np.ones(n, bool)
    total = 0
    seen = set()
    for v in order:
        c = labels[v]
        if c in seen or c != v:
            continue
        seen.add(c)
        rest = [u for u in range(n) if remaining[u] and u != v]
        for a, b in itertools.combinations(rest, 2):
            e = (adj[v, a], adj[v, b], adj[a, b])
            if sum(e) == 2:           # two positive, one negative: bad triangle
                total += 1
        remaining[labels == c] = False
    return total


def blocked_count(off, col, order, act_round_ids):
    """C4 blocked vertices of one round: actives with an earlier-ranked active
    neighbour (they would wait in isCenter)."""
    n = off.size - 1
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    act = set(int(a) for a in act_round_ids)
    b = 0
    for v in act:
        nb = neighbours(off, col, v)
        if any((int(u) in act) and rank[u] < rank[v] for u in nb):
            b += 1
    return b
