"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is either
a published constant, a hand-derived case, a textbook identity, brute force,
or an independent recomputation from a definition (see tests/cc_checks.py).
"""
import math
import os

import numpy as np
import pytest

import cc_checks as chk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

BELL = [1, 1, 2, 5, 15, 52, 203, 877, 4140, 21147, 115975]


def csr_from_pairs(n, pairs):
    import graphgen
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    return graphgen.from_edges(n, pairs[:, 0], pairs[:, 1], threads=1)


# --------------------------------------------------------------------------
# SplitMix64 and the permutation pi
# --------------------------------------------------------------------------
def test_splitmix64_published_vectors(ora):
    rows = []
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                x, y = line.split()
                rows.append((int(x, 16), int(y, 16)))
    assert len(rows) == 3
    for x, y in rows:
        assert ora.splitmix64(x) == y
        # key(seed, v) = splitmix64(seed ^ v): any (seed, v) with seed ^ v = x
        assert ora.perm_key(x ^ 5, 5) == y


@pytest.mark.parametrize("n,seed", [(0, 0), (1, 3), (4, 0), (1000, 7), (65537, 2**63 + 11)])
def test_permutation_is_sorted_by_key_then_vertex(ora, n, seed):
    order = ora.permutation(n, seed)
    assert np.array_equal(np.sort(order), np.arange(n))
    keys = [ora.perm_key(seed, int(v)) for v in order[: min(n, 5000)]]
    for a, b, va, vb in zip(keys, keys[1:], order, order[1:]):
        assert a < b or (a == b and va < vb)


def test_permutation_tiny_hand_order(ora):
    # n = 4, seed 0: keys are splitmix64(v) for v = 0..3; the oracle must list
    # vertices by ascending key.
    keys = {v: ora.splitmix64(v) for v in range(4)}
    expect = sorted(range(4), key=lambda v: (keys[v], v))
    assert list(ora.permutation(4, 0)) == expect
    assert keys[0] == 0xE220A8397B1DCDAF


# --------------------------------------------------------------------------
# Objective (Sec. 2 definition)
# --------------------------------------------------------------------------
def test_disagreements_hand_cases(ora):
    g = csr_from_pairs(3, [(0, 1), (1, 2)])            # path a-b-c
    assert ora.disagreements_pairs(g.off, g.col, np.array([0, 0, 0])) == 1   # (a,c) negative inside
    assert ora.disagreements(g.off, g.col, np.array([0, 0, 0])) == 1
    assert ora.disagreements(g.off, g.col, np.array([0, 1, 2])) == 2        # both edges cut
    assert ora.disagreements(g.off, g.col, np.array([7, 7, 9])) == 1        # cut (b,c)
    k4 = csr_from_pairs(4, [(i, j) for i in range(4) for j in range(i + 1, 4)])
    assert ora.disagreements(k4.off, k4.col, np.zeros(4, np.int32)) == 0
    assert ora.disagreements(k4.off, k4.col, np.arange(4, dtype=np.int32)) == 6
    e = csr_from_pairs(5, np.zeros((0, 2), np.int32))
    assert ora.disagreements(e.off, e.col, np.arange(5, dtype=np.int32)) == 0
    assert ora.disagreements(e.off, e.col, np.zeros(5, np.int32)) == 10


def test_disagreements_pairs_equal_counts_random(ora, gg):
    rng = np.random.default_rng(1)
    for trial in range(20):
        n = int(rng.integers(1, 120))
        g = gg.random_small(n, float(rng.random()) * 0.3, rng)
        lab = rng.integers(0, max(1, n // 3), n).astype(np.int32)
        assert ora.disagreements(g.off, g.col, lab) == ora.disagreements_pairs(g.off, g.col, lab)
        lab2 = (rng.integers(-2**31, 2**31 - 1, n)).astype(np.int32)   # arbitrary int32 ids
        assert ora.disagreements(g.off, g.col, lab2) == ora.disagreements_pairs(g.off, g.col, lab2)


# --------------------------------------------------------------------------
# Exhaustive OPT
# --------------------------------------------------------------------------
def test_bruteforce_visits_bell_many_partitions(ora):
    for n in range(1, 11):
        _, count, _ = ora.opt_bruteforce(np.zeros((n, n), np.uint8))
        assert count == BELL[n]


def test_bruteforce_opt_hand_cases(ora, gg):
    def opt(n, pairs):
        return ora.opt_bruteforce(gg.adjacency_matrix(csr_from_pairs(n, pairs)))[0]
    assert opt(3, [(0, 1), (1, 2)]) == 1                 # one bad triangle
    assert opt(4, [(0, 1), (0, 2), (0, 3)]) == 2         # star K_{1,3}
    assert opt(5, [(i, j) for i in range(5) for j in range(i + 1, 5)]) == 0   # K_5
    assert opt(4, [(0, 1), (2, 3)]) == 0                 # two disjoint edges
    assert opt(6, np.zeros((0, 2))) == 0                 # all negative
    # a 4-cycle: every partition pays 2
    assert opt(4, [(0, 1), (1, 2), (2, 3), (3, 0)]) == 2


# --------------------------------------------------------------------------
# KwikCluster (Alg. 1)
# --------------------------------------------------------------------------
def test_kwik_hand_cases(ora):
    n = 6
    k6 = csr_from_pairs(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    lab = ora.kwik(k6.off, k6.col, np.array([3, 0, 1, 2, 4, 5], np.int32))
    assert np.all(lab == 3)
    # two disjoint triangles: recovered exactly under any order
    tri = csr_from_pairs(6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5)])
    for order in ([5, 0, 1, 2, 3, 4], [1, 4, 0, 2, 3, 5]):
        lab = ora.kwik(tri.off, tri.col, np.array(order, np.int32))
        assert ora.disagreements(tri.off, tri.col, lab) == 0
        assert len(set(lab[:3])) == 1 and len(set(lab[3:])) == 1 and lab[0] != lab[3]
    # star: hub 0 with leaves 1..4
    star = csr_from_pairs(5, [(0, i) for i in range(1, 5)])
    lab = ora.kwik(star.off, star.col, np.array([0, 1, 2, 3, 4], np.int32))
    assert np.all(lab == 0) and ora.disagreements(star.off, star.col, lab) == 6   # C(4,2) leaf pairs
    lab = ora.kwik(star.off, star.col, np.array([2, 0, 1, 3, 4], np.int32))
    assert list(lab) == [2, 1, 2, 3, 4]
    assert ora.disagreements(star.off, star.col, lab) == 3                        # hub-leaf cuts
    # path 0-1-2-3, order (1, ...): clusters {0,1,2}, {3}; D = 1 (0,2) + 1 cut (2,3)
    p4 = csr_from_pairs(4, [(0, 1), (1, 2), (2, 3)])
    lab = ora.kwik(p4.off, p4.col, np.array([1, 3, 0, 2], np.int32))
    assert list(lab) == [1, 1, 1, 3] and ora.disagreements(p4.off, p4.col, lab) == 2
    # edgeless: singletons
    e = csr_from_pairs(4, np.zeros((0, 2)))
    assert list(ora.kwik(e.off, e.col, np.array([2, 1, 3, 0], np.int32))) == [0, 1, 2, 3]


@pytest.mark.parametrize("n", [5, 7, 9])
def test_kwik_expected_cost_at_most_3opt(ora, gg, n):
    """E_pi[KwikCluster] <= 3 OPT on complete signed graphs (Sec. 1 and
    Sec. 3.2), summed exactly over all n! orders; also cost(pi) >= OPT."""
    rng = np.random.default_rng(100 + n)
    for trial in range(6):
        g = gg.random_small(n, [0.2, 0.4, 0.6][trial % 3], rng)
        adj = gg.adjacency_matrix(g)
        opt, _, _ = ora.opt_bruteforce(adj)
        total, perms, worst, best = ora.kwik_all_perms_total(adj)
        assert perms == math.factorial(n)
        assert best >= opt
        assert total <= 3 * opt * perms
        if opt == 0:
            assert total == 0   # a disjoint union of cliques is always recovered


def test_kwik_cost_equals_bad_triangles_at_centers(ora, gg):
    """Lemma (cost of any peeling algorithm): disagreements = number of bad
    triangles of the residual graph containing each center, summed."""
    rng = np.random.default_rng(5)
    for trial in range(15):
        n = int(rng.integers(3, 14))
        g = gg.random_small(n, float(rng.random()) * 0.7, rng)
        order = rng.permutation(n).astype(np.int32)
        lab = ora.kwik(g.off, g.col, order)
        chk.check_partition_invariants(g.off, g.col, lab)
        assert ora.disagreements(g.off, g.col, lab) == chk.peeling_cost_by_bad_triangles(
            gg.adjacency_matrix(g), order, lab)


# --------------------------------------------------------------------------
# Alg. 2 rounds
# --------------------------------------------------------------------------
def test_batch_size_hand_values(ora):
    assert ora.batch_size(500_000, 10, 3) == 2          # ceil(0.5*10/3)
    assert ora.batch_size(500_000, 10, 0) == 10         # Delta = 0: everyone
    assert ora.batch_size(100_000, 7, 1000) == 1        # clamp up to 1
    assert ora.batch_size(1_000_000, 5, 1) == 5         # eps = 1, Delta = 1
    assert ora.batch_size(900_000, 1_000_000, 7) == 128572   # ceil(900000/7)
    assert ora.batch_size(100_000, 10_000_000, 1_000_000) == 1
    assert ora.batch_size(100_000, 67_108_864, 3) == 2236963   # ceil(6710886.4/3)
    assert ora.eps_to_ppm(0.1) == 100_000 and ora.eps_to_ppm(0.9) == 900_000


def _graphs(gg, seed):
    rng = np.random.default_rng(seed)
    out = [gg.random_small(int(rng.integers(1, 60)), float(rng.random()) * 0.3, rng) for _ in range(6)]
    out.append(gg.erdos_renyi(3000, 12 / 2999, seed=seed))
    out.append(gg.rmat(11, 8, seed=seed))
    out.append(gg.chung_lu(2000, 10.0, seed=seed))
    return out


@pytest.mark.parametrize("eps", [0.1, 0.5, 0.9, 1.0])
def test_c4_equals_kwikcluster(ora, gg, eps):
    """C4 is serializable (Sec. 3.2): same clustering as KwikCluster under pi."""
    for gi, g in enumerate(_graphs(gg, 11)):
        for seed in (0, 1, 2**40 + 3):
            order = ora.permutation(g.n, seed)
            lab, r, ar, st = ora.rounds(g.off, g.col, order, ora.ALGO_C4, eps, 1,
                                        stats_cap=100000, want_active_round=True)
            assert np.array_equal(lab, ora.kwik(g.off, g.col, order)), (gi, seed)
            chk.check_partition_invariants(g.off, g.col, lab)
            chk.check_round_structure(g.off, g.col, order, lab, ar, st, ora.eps_to_ppm(eps), 1,
                                      ora.batch_size)


@pytest.mark.parametrize("eps", [0.1, 0.5, 0.9])
def test_clusterwild_equals_kwikcluster_on_noisy_graph(ora, gg, eps):
    """ClusterWild! = KwikCluster run on G-hat, the graph with every edge
    inside one round's active set deleted (Sec. 3.2, appendix)."""
    for gi, g in enumerate(_graphs(gg, 12)):
        for seed in (0, 5):
            order = ora.permutation(g.n, seed)
            lab, r, ar, st = ora.rounds(g.off, g.col, order, ora.ALGO_CW, eps, 1,
                                        stats_cap=100000, want_active_round=True)
            off2, col2 = chk.noisy_graph(g.off, g.col, ar)
            assert np.array_equal(lab, ora.kwik(off2, col2, order)), (gi, seed)
            chk.check_partition_invariants(g.off, g.col, lab)
            chk.check_round_structure(g.off, g.col, order, lab, ar, st, ora.eps_to_ppm(eps), 2,
                                      ora.batch_size)
            if g.n <= 3000:
                chk.check_min_rank_center(g.off, g.col, order, lab, ar, 2)


def test_rounds_with_singleton_batches_equal_kwikcluster(ora, gg):
    """With k_i = 1 every round, Alg. 2 is Alg. 1 for both variants."""
    for g in _graphs(gg, 13)[:7]:
        order = ora.permutation(g.n, 9)
        kc = ora.kwik(g.off, g.col, order)
        for algo in (ora.ALGO_C4, ora.ALGO_CW):
            lab, r, ar, st = ora.rounds(g.off, g.col, order, algo, 1e-6, 1, stats_cap=100000)
            assert np.array_equal(lab, kc)
            if g.n:   # Delta_i = 0 takes every remaining (isolated) vertex at once
                assert np.all((st["k"] == 1) | (st["delta"] == 0))


@pytest.mark.parametrize("eps", [0.1, 0.5, 0.9])
def test_round_count_within_the_analysis_bound(ora, gg, eps):
    """Sec. 4 bounds the rounds by O((1/eps) log n log Delta) with high
    probability; on graphs of 1e4-6e4 vertices the oracle's count stays under
    2 (1/eps) ln(n) log2(Delta) (a loose constant: informational, not the
    paper's)."""
    import math
    for g in (gg.erdos_renyi(10_000, 20 / 9_999, seed=0), gg.rmat(15, 16, seed=2),
              gg.planted_partition(n=60_000, q=200, seed=1, noise=60_000)):
        delta = int(np.diff(g.off).max())
        bound = 2.0 / eps * math.log(g.n) * math.log2(max(delta, 2))
        for seed in (0, 1):
            order = ora.permutation(g.n, seed)
            for algo in (ora.ALGO_C4, ora.ALGO_CW):
                _, r, _, _ = ora.rounds(g.off, g.col, order, algo, eps, 1)
                assert 1 <= r <= bound, (g.n, eps, seed, algo, r, bound)


def test_delta_scan_equals_degree_table(ora, gg):
    for g in _graphs(gg, 14):
        order = ora.permutation(g.n, 4)
        for algo in (1, 2):
            a = ora.rounds(g.off, g.col, order, algo, 0.5, 0, stats_cap=100000)
            b = ora.rounds(g.off, g.col, order, algo, 0.5, 1, stats_cap=100000)
            assert np.array_equal(a[0], b[0]) and a[1] == b[1]
            for f in a[3]:
                assert np.array_equal(a[3][f], b[3][f])


def test_c4_min_rank_rule_and_blocked_counts(ora, gg):
    g = gg.erdos_renyi(800, 30 / 799, seed=3)
    order = ora.permutation(g.n, 17)
    lab, r, ar, st = ora.rounds(g.off, g.col, order, 1, 0.9, 1, stats_cap=10000, want_active_round=True)
    chk.check_min_rank_center(g.off, g.col, order, lab, ar, 1)
    for i in range(r):
        assert st["blocked"][i] == chk.blocked_count(g.off, g.col, order, np.nonzero(ar == i)[0])
    assert st["blocked"].sum() > 0


def test_trivial_graphs(ora, gg):
    e = csr_from_pairs(7, np.zeros((0, 2)))
    order = ora.permutation(7, 0)
    for algo in (1, 2):
        lab, r, _, st = ora.rounds(e.off, e.col, order, algo, 0.5, 1, stats_cap=10)
        assert list(lab) == list(range(7)) and r == 1 and st["delta"][0] == 0
    k = csr_from_pairs(6, [(i, j) for i in range(6) for j in range(i + 1, 6)])
    order = ora.permutation(6, 0)
    lab, r, _, _ = ora.rounds(k.off, k.col, order, 1, 0.5, 1)
    assert np.all(lab == order[0]) and r == 1
    assert ora.disagreements(k.off, k.col, lab) == 0
    g0 = csr_from_pairs(0, np.zeros((0, 2)))
    lab, r, _, _ = ora.rounds(g0.off, g0.col, np.zeros(0, np.int32), 2, 0.5, 1)
    assert lab.size == 0 and r == 0


def test_planted_labels_of_noise_free_partition_cost_zero(ora, gg):
    # every cluster a clique (p = 1), no drop, no noise: planted labels cost 0
    g = gg.planted_partition(n=400, q=10, min_size=5, zipf=1.5, p_max=1.0, mean_intra=1e9,
                             drop=0.0, noise=0, seed=2)
    assert ora.disagreements(g.off, g.col, g.aux) == 0
    order = ora.permutation(g.n, 1)
    assert ora.disagreements(g.off, g.col, ora.kwik(g.off, g.col, order)) == 0


# ---- the practical schedule of Sec. 5 (Delta-hat halving, binomial batches) ----
_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def _py_splitmix64_np(x):
    """SplitMix64 output function on a uint64 array (x already advanced)."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _py_period(n, max_deg, eps_ppm):
    bits = lambda x: int(x).bit_length()
    L = bits(n) + bits(bits(max(max_deg, 2))) + 4
    return -(-2 * 693147 * L // eps_ppm)


def _py_delta_hat(max_deg, period, i):
    h = i // period
    return max(1, (max_deg >> h) if h < 63 else 0)


def _py_threshold(eps_ppm, dh):
    den = 10**6 * dh
    return None if eps_ppm >= den else (eps_ppm << 64) // den


def _py_batch(seed, i, trials, thr):
    if thr is None:
        return trials
    s = ((seed ^ 0x5851F42D4C957F2D ^ i) + _GAMMA) & _M64
    z = s
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    s = z ^ (z >> 31)
    j = np.arange(1, trials + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        states = np.uint64(s) + j * np.uint64(_GAMMA)
    return int((_py_splitmix64_np(states) < np.uint64(thr)).sum())


def test_bsp_schedule_matches_closed_forms(ora):
    """Period, Delta-hat, threshold and batch draw of the Sec. 5 schedule
    re-derived in Python integers and numpy (readings R13, R14)."""
    for n, D, eps in ((10_000, 40, 0.5), (1, 0, 1.0), (67_108_864, 1_003_939, 0.5), (5, 3, 0.1), (999, 1, 0.9)):
        ppm = ora.eps_to_ppm(eps)
        P = ora.bsp_period(n, D, eps)
        assert P == _py_period(n, D, ppm)
        for i in (0, 1, P - 1, P, 3 * P + 2, 80 * P):
            assert ora.bsp_delta_hat(D, P, i) == _py_delta_hat(D, P, i)
    assert ora.bsp_period(67_108_864, 1_003_939, 0.5) == 100
    for ppm, dh in ((500_000, 40), (1_000_000, 1), (1, 2**31 - 1), (999_999, 1), (100_000, 3), (1_000_000, 2)):
        t, all_ = ora.bsp_threshold(ppm / 1e6, dh)
        want = _py_threshold(ppm, dh)
        assert all_ == (want is None)
        if want is not None:
            assert t == want
    rng = np.random.default_rng(4)
    for _ in range(20):
        seed, i, trials = int(rng.integers(0, 2**63)), int(rng.integers(0, 500)), int(rng.integers(0, 20_000))
        thr = int(rng.integers(0, 2**63)) * 2
        assert ora.bsp_batch(seed, i, trials, thr, False) == _py_batch(seed, i, trials, thr)
    # the draw is a binomial: its mean over many rounds is trials * p
    thr = _py_threshold(500_000, 40)
    draws = [ora.bsp_batch(7, i, 10_000, thr, False) for i in range(400)]
    assert abs(np.mean(draws) - 10_000 / 80) < 4 * np.sqrt(10_000 / 80 / 400)


def _check_bsp_windows(off, col, order, labels, ar, stats, eps, seed):
    """A_i = the alive vertices among ranks [c_i, c_i + B_i) with B_i the
    round's binomial draw over n - c_i trials (R15), Delta-hat_i in the stats."""
    n = off.size - 1
    D = int(np.diff(off).max()) if n else 0
    ppm = round(eps * 10**6)
    P = _py_period(n, D, ppm)
    rr = chk.removal_rounds(labels, ar)
    R = len(stats["k"])
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    c = 0
    for i in range(R):
        dh = _py_delta_hat(D, P, i)
        b = _py_batch(seed, i, n - c, _py_threshold(ppm, dh))
        window = order[c:c + b]
        alive_in_window = window[rr[window] >= i]
        assert np.array_equal(np.sort(np.nonzero(ar == i)[0]), np.sort(alive_in_window)), i
        assert stats["delta"][i] == dh and stats["k"][i] == alive_in_window.size
        assert stats["n_alive"][i] == int((rr >= i).sum())
        c += b
    assert int((rr >= R).sum()) == 0


@pytest.mark.parametrize("eps", [0.1, 0.5, 1.0])
def test_bsp_c4_equals_kwikcluster(ora, gg, eps):
    """Serializability holds for any batch sequence: C4 with the Sec. 5
    schedule is KwikCluster under pi."""
    for gi, g in enumerate(_graphs(gg, 21)):
        for seed in (0, 3, 2**50 + 1):
            order = ora.permutation(g.n, seed)
            lab, r, ar, st = ora.rounds_bsp(g.off, g.col, order, ora.ALGO_C4, eps, seed,
                                            stats_cap=100000, want_active_round=True)
            assert np.array_equal(lab, ora.kwik(g.off, g.col, order)), (gi, seed)
            if g.n:
                _check_bsp_windows(g.off, g.col, order, lab, ar, st, eps, seed)


@pytest.mark.parametrize("eps", [0.1, 0.9])
def test_bsp_clusterwild_equals_kwikcluster_on_noisy_graph(ora, gg, eps):
    """ClusterWild! with the Sec. 5 schedule is KwikCluster on G-hat (edges
    inside one round's active set deleted)."""
    for gi, g in enumerate(_graphs(gg, 22)):
        for seed in (1, 6):
            order = ora.permutation(g.n, seed)
            lab, r, ar, st = ora.rounds_bsp(g.off, g.col, order, ora.ALGO_CW, eps, seed,
                                            stats_cap=100000, want_active_round=True)
            off2, col2 = chk.noisy_graph(g.off, g.col, ar)
            assert np.array_equal(lab, ora.kwik(off2, col2, order)), (gi, seed)
            chk.check_partition_invariants(g.off, g.col, lab)
            if g.n:
                _check_bsp_windows(g.off, g.col, order, lab, ar, st, eps, seed)
