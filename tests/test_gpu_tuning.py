"""Schedule settings change no result: every clustering, per-round statistic
and batched job is identical under extreme tunings and equal to the oracle;
the autotuner stores its choice and reuses it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STAT_FIELDS = ("n_alive", "delta", "k", "centers", "removed", "blocked")
EXTREMES = [
    {},
    {"walk_batches": 1, "prefetch_ahead": 0, "inline_heavy": 0, "inline_rebuild": 0, "inline_decide": 0,
     "heavy_shift": 4, "warp_resolve_row": 0},
    {"walk_batches": 8, "prefetch_ahead": 8, "inline_heavy": 65536, "inline_rebuild": 65536,
     "inline_decide": 65536, "heavy_shift": 2, "warp_resolve_row": 1 << 24},
    {"walk_batches": 2, "prefetch_ahead": 1, "inline_heavy": 16, "inline_rebuild": 16, "inline_decide": 1,
     "heavy_shift": 3},
]


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1507_05086_gb300 as cc
    cc.load()
    return cc


def _graphs(gg):
    rng = np.random.default_rng(4)
    n = 120_000
    er = gg.erdos_renyi(n, 5.0 / n, seed=2)
    src = [np.repeat(np.arange(n, dtype=np.int32), np.diff(er.off).astype(np.int64)), np.zeros(30_000, np.int32)]
    leaves = rng.choice(np.arange(1, n, dtype=np.int32), 30_000, replace=False)
    hub = gg.from_edges(n, np.concatenate(src), np.concatenate([er.col, leaves]))
    return [gg.rmat(15, 16, seed=6), gg.chung_lu(60_000, 20.0, seed=8), hub,
            gg.planted_partition(n=40_000, q=100, seed=3, noise=60_000)]


def test_round_kernel_settings_change_no_result(cc, ora, gg):
    for g in _graphs(gg):
        with cc.Graph(g.off, g.col) as graph:
            for algo, a, seed in (("c4", 1, 5), ("cw", 2, 6), ("cw", 2, 7)):
                order = ora.permutation(g.n, seed)
                olab, orr, _, ost = ora.rounds(g.off, g.col, order, a, 0.5, 1, stats_cap=1_000_000)
                for t in EXTREMES:
                    graph.set_tuning(t)
                    assert all(graph.get_tuning()[k] == v for k, v in t.items())
                    lab, r, d, st = graph.cluster(algo, 0.5, seed, stats_cap=100_000)
                    assert np.array_equal(lab, olab) and r == orr, (algo, t)
                    for f in STAT_FIELDS:
                        assert np.array_equal(st[f], ost[f]), (algo, t, f)
            graph.set_tuning({})


def test_batch_settings_change_no_result(cc, gg):
    gs = [gg.chung_lu(n, 10.0, seed=30 + i) for i, n in enumerate((700, 3000, 20_000, 70_000, 150_000))]
    graphs = [cc.Graph(g.off, g.col) for g in gs]
    default = cc.get_batch_tuning()
    try:
        seeds = np.arange(len(gs), dtype=np.uint64) * 11 + 3
        ref = cc.batch_jobs(graphs, "c4", 0.5, seeds, 3)
        for t in ({"batch_small_n": 1024, "batch_team_n": 4096, "batch_team_blocks": 2, "walk_batches": 1,
                   "inline_heavy": 0, "heavy_shift": 3},
                  {"batch_small_n": 1 << 20, "batch_team_n": 1 << 20, "batch_team_blocks": 16},
                  {"batch_small_n": 2048, "batch_team_n": 1 << 24, "batch_team_blocks": 16}):
            cc.set_batch_tuning(dict(default, **t))
            D, R = cc.batch_jobs(graphs, "c4", 0.5, seeds, 3)
            assert np.array_equal(D, ref[0]) and np.array_equal(R, ref[1]), t
    finally:
        cc.set_batch_tuning(default)
        for x in graphs:
            x.close()


def test_autotuner_stores_and_reuses_its_choice(cc, gg, tmp_path):
    from paper_1507_05086_gb300 import autotune
    g = gg.rmat(14, 16, seed=2)
    cache = str(tmp_path / "tuning.json")
    with cc.Graph(g.off, g.col) as graph:
        _, r0, d0 = graph.cluster("cw", 0.5, 9, want_labels=False)
        e1 = autotune.tune_rounds(graph, algos=("cw",), seeds=(9,), cache=cache, budget_s=20.0,
                                  knobs={"walk_batches": (2, 4), "heavy_shift": (1, 2)})
        assert e1["source"] == "tuned now" and e1["evaluations"] >= 2
        assert graph.get_tuning()["walk_batches"] == e1["tuning"]["walk_batches"]
        e2 = autotune.tune_rounds(graph, algos=("cw",), seeds=(9,), cache=cache)
        assert e2["source"] == "cache" and e2["tuning"] == e1["tuning"]
        _, r1, d1 = graph.cluster("cw", 0.5, 9, want_labels=False)
        assert (r1, d1) == (r0, d0)
