"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Every comparison is exact (integer work): permutations, labels, round counts,
per-round statistics and disagreements must be identical.
"""
import numpy as np
import pytest

import cc_checks as chk

pytestmark = pytest.mark.gpu

STAT_FIELDS = ("n_alive", "delta", "k", "centers", "removed", "blocked")


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1507_05086_gb300 as cc
    cc.load()
    return cc


def small_graphs(gg, seed):
    """Seeded graphs spanning several tiles and ragged tails: tiny random
    graphs, an ER graph, a planted partition, R-MAT and Chung-Lu power laws,
    and degenerate shapes."""
    rng = np.random.default_rng(seed)
    out = []
    for n in (1, 2, 3, 17, 33, 100, 513):
        out.append(gg.random_small(n, float(rng.random()) * 0.2, rng))
    out.append(gg.erdos_renyi(10_000, 20 / 9_999, seed=0))                # the 10k ER workload
    out.append(gg.planted_partition(n=20_000, q=60, seed=seed, noise=40_000))
    out.append(gg.rmat(14, 16, seed=seed))
    out.append(gg.chung_lu(30_000, 24.0, seed=seed))
    e = gg.from_edges(1000, np.zeros(0, np.int32), np.zeros(0, np.int32))   # edgeless
    out.append(e)
    star = gg.from_edges(2000, np.zeros(1999, np.int32), np.arange(1, 2000, dtype=np.int32))
    out.append(star)
    k = 60
    iu, ju = np.triu_indices(k, 1)
    out.append(gg.from_edges(k, iu.astype(np.int32), ju.astype(np.int32)))   # clique
    # rows of length one everywhere (a perfect matching) and many small stars:
    # list items that end exactly on the edge-walker's batch boundaries
    m = np.arange(0, 5000, 2, dtype=np.int32)
    out.append(gg.from_edges(5000, m, m + 1))
    hubs = np.repeat(np.arange(0, 6000, 7, dtype=np.int32), 6)
    leaves = (hubs + np.tile(np.arange(1, 7, dtype=np.int32), hubs.size // 6)).astype(np.int32)
    out.append(gg.from_edges(6006, hubs, leaves))
    return out


def oracle_run(ora, g, order, algo, eps):
    lab, r, ar, st = ora.rounds(g.off, g.col, order, algo, eps, 1, stats_cap=1_000_000,
                                want_active_round=True)
    return lab, r, ar, st


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 5), (768, 1), (769, 2), (10_000, 0), (100_003, 7),
                                    (1 << 20, 3), ((1 << 20) + 12345, 2**63 + 5)])
def test_permutation_matches_oracle(cc, ora, gg, n, seed):
    g = gg.from_edges(n, np.zeros(0, np.int32), np.zeros(0, np.int32))
    with cc.Graph(g.off, g.col) as graph:
        assert np.array_equal(graph.permutation(seed), ora.permutation(n, seed))


def _splitmix64_np(x):
    """The published SplitMix64 output for state x (numpy, uint64 wrap-around)."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


@pytest.mark.parametrize("n,seed", [(1 << 26, 9), (110_000_003, 4)])
def test_permutation_large_is_sorted_by_key(cc, gg, n, seed):
    """At the bench size (shared-memory bucket counters) and above 10^8
    vertices (global counters): pi is a permutation and ascending in
    (splitmix64(seed ^ v), v), which defines it uniquely."""
    off = np.zeros(n + 1, np.int64)
    with cc.Graph(off, np.zeros(0, np.int32)) as graph:
        order = graph.permutation(seed)
    assert order.shape == (n,)
    seen = np.zeros(n, np.bool_)
    seen[order] = True
    assert seen.all()
    keys = _splitmix64_np(np.uint64(seed) ^ order.astype(np.uint64))
    ka, kb = keys[:-1], keys[1:]
    assert bool(np.all((ka < kb) | ((ka == kb) & (order[:-1] < order[1:]))))


@pytest.mark.parametrize("algo", ["c4", "cw"])
@pytest.mark.parametrize("eps", [0.1, 0.5, 0.9, 1.0])
def test_cluster_matches_oracle(cc, ora, gg, algo, eps):
    a = 1 if algo == "c4" else 2
    for gi, g in enumerate(small_graphs(gg, 3)):
        with cc.Graph(g.off, g.col) as graph:
            for seed in (0, 1, 12345):
                order = ora.permutation(g.n, seed)
                olab, orr, ar, ost = oracle_run(ora, g, order, a, eps)
                lab, r, d, st = graph.cluster(algo, eps, seed, stats_cap=100_000)
                assert np.array_equal(lab, olab), (gi, seed)
                assert r == orr
                for f in STAT_FIELDS:
                    assert np.array_equal(st[f], ost[f]), (gi, seed, f)
                assert d == ora.disagreements(g.off, g.col, olab)
                if a == 1:
                    assert np.array_equal(lab, ora.kwik(g.off, g.col, order))


def test_er10k_many_permutations(cc, ora, gg):
    """The 10k ER workload over the paper's protocol of many random orders."""
    g = gg.erdos_renyi(10_000, 20 / 9_999, seed=0)
    with cc.Graph(g.off, g.col) as graph:
        for seed in range(40):
            order = ora.permutation(g.n, seed)
            lab, _, d = graph.cluster("c4", 0.5, seed)
            assert np.array_equal(lab, ora.kwik(g.off, g.col, order))
            olab, orr, _, _ = ora.rounds(g.off, g.col, order, 2, 0.5)
            lab, r, d = graph.cluster("cw", 0.5, seed)
            assert np.array_equal(lab, olab) and r == orr
            assert d == ora.disagreements(g.off, g.col, olab)


def test_singleton_batches_equal_kwikcluster(cc, ora, gg):
    g = gg.rmat(12, 8, seed=4)
    order = ora.permutation(g.n, 2)
    kc = ora.kwik(g.off, g.col, order)
    with cc.Graph(g.off, g.col) as graph:
        for algo in ("c4", "cw"):
            lab, r, d = graph.cluster(algo, 1e-6, 2)
            assert np.array_equal(lab, kc)


def test_invariants_and_round_structure_on_gpu_output(cc, ora, gg):
    g = gg.chung_lu(5000, 16.0, seed=9)
    with cc.Graph(g.off, g.col) as graph:
        for algo, a in (("c4", 1), ("cw", 2)):
            order = ora.permutation(g.n, 77)
            lab, r, d, st = graph.cluster(algo, 0.5, 77, stats_cap=100_000)
            chk.check_partition_invariants(g.off, g.col, lab)
            _, _, ar, _ = ora.rounds(g.off, g.col, order, a, 0.5, 1, want_active_round=True)
            chk.check_round_structure(g.off, g.col, order, lab, ar, st, 500_000, a, ora.batch_size)
            chk.check_min_rank_center(g.off, g.col, order, lab, ar, a)
            # every round took some device time, and no round took longer than the kernel
            graph.set_timing(True)
            _, _, _, st = graph.cluster(algo, 0.5, 77, stats_cap=100_000)
            assert (st["ns"] > 0).all()
            assert st["ns"].sum() <= graph.last_timings()[1] * 1e6 * 1.01 + 1e5
            graph.set_timing(False)


def test_disagreements_of_arbitrary_labels(cc, ora, gg):
    rng = np.random.default_rng(8)
    g = gg.planted_partition(n=50_000, q=200, seed=2, noise=100_000)
    with cc.Graph(g.off, g.col) as graph:
        assert graph.disagreements(g.aux) == ora.disagreements(g.off, g.col, g.aux)
        for _ in range(3):
            lab = rng.integers(0, rng.integers(1, g.n), g.n).astype(np.int32)
            assert graph.disagreements(lab) == ora.disagreements(g.off, g.col, lab)
        assert graph.disagreements(np.arange(g.n, dtype=np.int32)) == g.m
        with pytest.raises(cc.CCError):
            graph.disagreements(np.full(g.n, g.n, np.int32))


def test_device_pointers_and_determinism(cc, ora, gg):
    import torch
    g = gg.rmat(13, 16, seed=1)
    off = torch.from_numpy(g.off).cuda()
    col = torch.from_numpy(g.col).cuda()
    with cc.Graph(off, col) as graph:
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for algo in ("c4", "cw"):
            graph.cluster(algo, 0.5, 3, labels_out=out)
            torch.cuda.synchronize()
            first = out.cpu().numpy().copy()
            lab, _, _ = graph.cluster(algo, 0.5, 3)
            assert np.array_equal(first, lab)
            order = ora.permutation(g.n, 3)
            olab, _, _, _ = ora.rounds(g.off, g.col, order, 1 if algo == "c4" else 2, 0.5)
            assert np.array_equal(lab, olab)


def ora_free_disagreements(g, lab):
    """Disagreements from the definition (numpy): cut positive edges plus
    non-adjacent pairs inside clusters."""
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    intra = int(np.sum(lab[src] == lab[g.col])) // 2
    _, sizes = np.unique(lab, return_counts=True)
    return g.m - intra + int(np.sum(sizes * (sizes - 1) // 2)) - intra


def test_invalid_arguments_and_graphs(cc, gg):
    g = gg.rmat(8, 4, seed=0)
    with cc.Graph(g.off, g.col) as graph:
        for eps in (0.0, -0.5, 1.5, float("nan")):
            with pytest.raises(cc.CCError) as ei:
                graph.cluster("cw", eps, 0)
            assert ei.value.status == -1
        # the graph stays usable after an invalid argument
        graph.cluster("cw", 0.5, 0)
    bad = []
    off = np.array([0, 1, 1], np.int64)
    bad.append((off, np.array([1], np.int32)))                 # asymmetric
    bad.append((np.array([0, 1, 2], np.int64), np.array([0, 0], np.int32)))   # self loops
    bad.append((np.array([0, 2, 3, 4], np.int64), np.array([2, 1, 0, 0], np.int32)))  # unsorted row
    bad.append((np.array([0, 1, 2], np.int64), np.array([1, 5], np.int32)))   # out of range
    bad.append((np.array([0, 2, 1], np.int64), np.array([1, 0], np.int32)))   # decreasing offsets
    for off, col in bad:
        for exact in (False, True):
            with pytest.raises(cc.CCError) as ei:
                cc.Graph(off, col, exact_symmetry=exact)
            assert ei.value.status == -2
    # the exact symmetry check (reverse-entry search) accepts symmetric graphs
    # with long rows and rejects a row whose entry has no reverse
    g2 = gg.rmat(12, 8, seed=1)
    assert int(np.diff(g2.off).max()) > 100
    with cc.Graph(g2.off, g2.col, exact_symmetry=True) as gx:
        lab, r, d = gx.cluster("cw", 0.5, 1)
        assert r > 0 and d == ora_free_disagreements(g2, lab)
    e = gg.from_edges(6, np.array([0, 1, 2], np.int32), np.array([3, 4, 5], np.int32))
    ecol = e.col.copy()
    ecol[int(e.off[3])] = 1            # row 3 lists 1 instead of 0
    with pytest.raises(cc.CCError) as ei:
        cc.Graph(e.off, ecol, exact_symmetry=True)
    assert ei.value.status == -2


def test_planted_partition_1m_all_eps(cc, ora, gg):
    """The planted-partition workload at full size (n = 10^6, 2,000 Zipf
    clusters, 4M noise edges): C4 = KwikCluster, ClusterWild! = oracle rounds,
    at eps in {0.1, 0.5, 0.9}; D of the planted labels."""
    g = gg.workload("planted1m")
    with cc.Graph(g.off, g.col) as graph:
        assert graph.disagreements(g.aux) == ora.disagreements(g.off, g.col, g.aux)
        order = ora.permutation(g.n, 0)
        kc = ora.kwik(g.off, g.col, order)
        dkc = ora.disagreements(g.off, g.col, kc)
        for eps in (0.1, 0.5, 0.9):
            lab, r, d = graph.cluster("c4", eps, 0)
            assert np.array_equal(lab, kc) and d == dkc
            olab, orr, _, _ = ora.rounds(g.off, g.col, order, 2, eps)
            lab, r, d = graph.cluster("cw", eps, 0)
            assert np.array_equal(lab, olab) and r == orr
            assert d == ora.disagreements(g.off, g.col, olab)


# --------------------------------------------------------------------------
# Batched engine (many graphs x k permutations in one launch per size class)
# --------------------------------------------------------------------------
def batch_graphs(gg):
    """Chung-Lu power-law graphs across the batch size classes: one block per
    job (n <= 2^16) and eight-block teams (2^16 < n <= 2^21)."""
    sizes = [(300, 8.0), (1000, 12.0), (2500, 30.0), (9000, 16.0), (30000, 20.0), (65536, 8.0),
             (80000, 10.0), (250000, 24.0)]
    return [gg.chung_lu(n, d, seed=40 + i) for i, (n, d) in enumerate(sizes)]


@pytest.mark.parametrize("algo", ["cw", "c4"])
def test_batch_jobs_match_oracle(cc, ora, gg, algo):
    a = 1 if algo == "c4" else 2
    gs = batch_graphs(gg)
    graphs = [cc.Graph(g.off, g.col) for g in gs]
    try:
        seeds = np.array([17 * i + 3 for i in range(len(gs))], np.uint64)
        k = 3
        D, R = cc.batch_jobs(graphs, algo, 0.5, seeds, k)
        for i, g in enumerate(gs):
            for j in range(k):
                order = ora.permutation(g.n, int(seeds[i]) + j)
                lab, r, _, _ = ora.rounds(g.off, g.col, order, a, 0.5)
                assert R[i, j] == r, (i, j)
                assert D[i, j] == ora.disagreements(g.off, g.col, lab), (i, j)
        # each job gives the same result alone and inside the batch
        for i in (0, len(gs) - 1):
            _, r, d = graphs[i].cluster(algo, 0.5, int(seeds[i]) + 1, want_labels=False)
            assert (r, d) == (R[i, 1], D[i, 1])
    finally:
        for x in graphs:
            x.close()


def test_batch_run_best_of_k(cc, ora, gg):
    gs = batch_graphs(gg)[:5]
    graphs = [cc.Graph(g.off, g.col) for g in gs]
    try:
        seeds = np.arange(len(gs), dtype=np.uint64) * 1000
        bj, bd, br, labels = cc.batch_run(graphs, "cw", 0.9, seeds, 4, want_labels=True)
        for i, g in enumerate(gs):
            costs = []
            for j in range(4):
                order = ora.permutation(g.n, int(seeds[i]) + j)
                lab, r, _, _ = ora.rounds(g.off, g.col, order, 2, 0.9)
                costs.append((ora.disagreements(g.off, g.col, lab), j, lab, r))
            best = min(costs, key=lambda c: (c[0], c[1]))
            assert (bj[i], bd[i], br[i]) == (best[1], best[0], best[3])
            assert np.array_equal(labels[i], best[2])
    finally:
        for x in graphs:
            x.close()


def test_memory_pool_reuse_and_release(cc, ora, gg):
    """Graphs created after a destroyed one reuse the pool; releasing the
    unused reserve changes no result."""
    g = gg.rmat(14, 8, seed=12)
    order = ora.permutation(g.n, 5)
    expect, er, _, _ = ora.rounds(g.off, g.col, order, 2, 0.5)
    for round_ in range(3):
        with cc.Graph(g.off, g.col) as graph:
            lab, r, d = graph.cluster("cw", 0.5, 5)
            assert np.array_equal(lab, expect) and r == er
        if round_ == 1:
            cc.release_memory()
    cc.release_memory()


def test_hubs_losing_degree_while_alive_match_oracle(cc, ora, gg):
    """Three hubs of degree 66k-80k in a sparse background: their residual
    degrees (and Delta) fall over several rounds before they are clustered."""
    rng = np.random.default_rng(21)
    n = 300_000
    er = gg.erdos_renyi(n, 6.0 / n, seed=3)
    src = [np.repeat(np.arange(n, dtype=np.int32), np.diff(er.off).astype(np.int64))]
    dst = [er.col]
    for h, deg in ((0, 80_000), (1, 70_000), (17, 66_000)):
        leaves = rng.choice(n, deg + 10, replace=False).astype(np.int32)
        leaves = leaves[leaves != h][:deg]
        src.append(np.full(leaves.size, h, np.int32))
        dst.append(leaves)
    g = gg.from_edges(n, np.concatenate(src), np.concatenate(dst))
    assert np.diff(g.off).max() >= 65535
    with cc.Graph(g.off, g.col) as graph:
        for algo, a in (("cw", 2), ("c4", 1)):
            for eps, seed in ((0.5, 4), (0.9, 9)):
                order = ora.permutation(g.n, seed)
                olab, orr, _, ost = oracle_run(ora, g, order, a, eps)
                lab, r, d, st = graph.cluster(algo, eps, seed, stats_cap=100_000)
                assert np.array_equal(lab, olab) and r == orr, (algo, eps)
                for f in STAT_FIELDS:
                    assert np.array_equal(st[f], ost[f]), (algo, eps, f)
                assert d == ora.disagreements(g.off, g.col, olab)


@pytest.mark.parametrize("name", ["rmat17", "chung_lu400k", "planted200k"])
def test_larger_graphs_all_eps_match_oracle(cc, ora, gg, name):
    """Graphs of 1.3e5-4e5 vertices, many of them selected with residual
    degree 0 (singletons that keep their alive word): labels, rounds and
    every round's statistics equal the oracle's, for both algorithms and
    three eps, and for the Sec. 5 schedule."""
    g = {"rmat17": lambda: gg.rmat(17, 16, seed=8),
         "chung_lu400k": lambda: gg.chung_lu(400_000, 12.0, seed=4),
         "planted200k": lambda: gg.planted_partition(n=200_000, q=300, seed=2, noise=300_000)}[name]()
    with cc.Graph(g.off, g.col) as graph:
        for algo, a in (("cw", 2), ("c4", 1)):
            for eps, seed in ((0.1, 3), (0.5, 5), (0.9, 7)):
                order = ora.permutation(g.n, seed)
                olab, orr, _, ost = oracle_run(ora, g, order, a, eps)
                lab, r, d, st = graph.cluster(algo, eps, seed, stats_cap=100_000)
                assert np.array_equal(lab, olab) and r == orr, (algo, eps)
                for f in STAT_FIELDS:
                    assert np.array_equal(st[f], ost[f]), (algo, eps, f)
                assert d == ora.disagreements(g.off, g.col, olab)
        order = ora.permutation(g.n, 11)
        olab, orr, _, ost = ora.rounds_bsp(g.off, g.col, order, 2, 0.5, 11, stats_cap=100_000)
        lab, r, d, st = graph.cluster("cw-est", 0.5, 11, stats_cap=100_000)
        assert np.array_equal(lab, olab) and r == orr
        for f in STAT_FIELDS:
            assert np.array_equal(st[f], ost[f]), f


@pytest.mark.parametrize("algo,a", [("c4-est", 1), ("cw-est", 2)])
@pytest.mark.parametrize("eps", [0.1, 0.5, 1.0])
def test_sec5_schedule_matches_oracle(cc, ora, gg, algo, a, eps):
    """The practical schedule of Sec. 5 (Delta-hat halving, binomial batches
    over the unprocessed suffix of pi): labels, rounds and every round's
    statistics equal the oracle's; C4 still equals KwikCluster."""
    graphs = small_graphs(gg, 5) + [gg.from_edges(9, np.zeros(0, np.int32), np.zeros(0, np.int32))]
    for gi, g in enumerate(graphs):
        with cc.Graph(g.off, g.col) as graph:
            for seed in (0, 7, 2**45 + 11):
                order = ora.permutation(g.n, seed)
                olab, orr, _, ost = ora.rounds_bsp(g.off, g.col, order, a, eps, seed, stats_cap=1_000_000)
                lab, r, d, st = graph.cluster(algo, eps, seed, stats_cap=1_000_000)
                assert np.array_equal(lab, olab), (gi, seed)
                assert r == orr
                for f in STAT_FIELDS:
                    assert np.array_equal(st[f], ost[f]), (gi, seed, f)
                assert d == ora.disagreements(g.off, g.col, olab)
                if a == 1:
                    assert np.array_equal(lab, ora.kwik(g.off, g.col, order))


def test_sec5_schedule_larger_graphs_and_batches(cc, ora, gg):
    """R-MAT and planted graphs through the whole grid and through the
    batched engine (one block and eight-block teams)."""
    graphs = [gg.rmat(15, 8, seed=3), gg.planted_partition(n=60_000, q=150, seed=4, noise=80_000)]
    for g in graphs:
        with cc.Graph(g.off, g.col) as graph:
            for algo, a in (("cw-est", 2), ("c4-est", 1)):
                seed = 99
                order = ora.permutation(g.n, seed)
                olab, orr, _, _ = ora.rounds_bsp(g.off, g.col, order, a, 0.5, seed)
                lab, r, d = graph.cluster(algo, 0.5, seed)
                assert np.array_equal(lab, olab) and r == orr
                D, R = cc.batch_jobs([graph], algo, 0.5, np.array([seed], np.uint64), 2)
                for j in range(2):
                    o2 = ora.permutation(g.n, seed + j)
                    l2, r2, _, _ = ora.rounds_bsp(g.off, g.col, o2, a, 0.5, seed + j)
                    assert R[0, j] == r2 and D[0, j] == ora.disagreements(g.off, g.col, l2)
