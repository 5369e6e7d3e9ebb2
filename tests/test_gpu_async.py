"""GPU parity of the asynchronous C4 (Alg. 3 with attemptCluster, no rounds).

C4 is serializable (Sec. 4): whatever the interleaving of the decisions, the
labels are those of serial KwikCluster under the same pi.  Every comparison
is exact, against the oracle's KwikCluster and objective.
"""
import numpy as np
import pytest

from test_gpu_parity import small_graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1507_05086_gb300 as cc
    cc.load()
    return cc


def check_async(cc, ora, graph, g, seed):
    order = ora.permutation(g.n, seed)
    expect = ora.kwik(g.off, g.col, order)
    lab, rounds, d, st = graph.cluster("c4-async", 0.5, seed, stats_cap=4)
    assert np.array_equal(lab, expect), seed
    assert rounds == 0
    assert d == ora.disagreements(g.off, g.col, expect)
    # one record for the whole run
    assert st["n_alive"].tolist() == [g.n] and st["removed"].tolist() == [g.n] and st["k"].tolist() == [g.n]
    assert st["centers"][0] == np.unique(expect).size
    assert 0 <= st["blocked"][0] <= g.n
    assert 0 <= st["edges"][0] <= g.off[-1]
    return lab, d, st


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_async_c4_equals_kwikcluster_on_small_graphs(cc, ora, gg, seed):
    for g in small_graphs(gg, seed):
        with cc.Graph(g.off, g.col) as graph:
            check_async(cc, ora, graph, g, seed + 11)


def test_async_c4_equals_bsp_c4_under_many_orders(cc, ora, gg):
    g = gg.erdos_renyi(10_000, 20 / 9_999, seed=0)
    with cc.Graph(g.off, g.col) as graph:
        for seed in range(12):
            lab, d, _ = check_async(cc, ora, graph, g, seed)
            lab4, _, d4 = graph.cluster("c4", 0.5, seed)
            assert np.array_equal(lab, lab4) and d == d4


def test_async_c4_hubs_use_the_deferred_pushes(cc, ora, gg):
    """Hubs of degree 66k-80k (rows above the eager-push limit) in a sparse
    background, plus R-MAT and Chung-Lu power laws."""
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
    graphs = [gg.from_edges(n, np.concatenate(src), np.concatenate(dst)), gg.rmat(17, 16, seed=5),
              gg.chung_lu(200_000, 30.0, seed=2)]
    for g in graphs:
        with cc.Graph(g.off, g.col) as graph:
            for seed in (4, 9):
                check_async(cc, ora, graph, g, seed)


def test_async_c4_device_labels_and_repeat(cc, ora, gg):
    import torch
    g = gg.rmat(13, 16, seed=1)
    off = torch.from_numpy(g.off).cuda()
    col = torch.from_numpy(g.col).cuda()
    with cc.Graph(off, col) as graph:
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for _ in range(3):
            graph.cluster("c4-async", 0.5, 3, labels_out=out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), ora.kwik(g.off, g.col, ora.permutation(g.n, 3)))


def test_async_c4_is_not_a_batch_or_server_algorithm(cc, gg):
    g = gg.rmat(8, 4, seed=0)
    with cc.Graph(g.off, g.col) as graph:
        with pytest.raises(cc.CCError) as ei:
            cc.batch_jobs([graph], "c4-async", 0.5, np.array([1], np.uint64), 2)
        assert ei.value.status == -1
        with pytest.raises(cc.CCError) as ei:
            graph.cluster("c4-async", 0.0, 1)              # eps is still checked
        assert ei.value.status == -1
