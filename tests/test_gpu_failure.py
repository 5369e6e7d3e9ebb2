"""Failure detection without a GPU fault: a bounded wait of the round kernel
is made to run out (the coordinator withholds one barrier release through the
test hook), every block unwinds, the call reports CC_ERR_TIMEOUT, and the
graph keeps giving the oracle's results afterwards."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1507_05086_gb300 as cc
    cc.load()
    return cc


def test_withheld_release_times_out_and_the_graph_stays_usable(cc, ora, gg):
    g = gg.rmat(12, 8, seed=3)
    order = ora.permutation(g.n, 7)
    olab, orr, _, _ = ora.rounds(g.off, g.col, order, 2, 0.5)
    assert orr > 2
    with cc.Graph(g.off, g.col) as graph:
        graph.debug_withhold_release(1)
        t0 = time.perf_counter()
        with pytest.raises(cc.CCError) as ei:
            graph.cluster("cw", 0.5, 7)
        waited = time.perf_counter() - t0
        assert ei.value.status == -5                     # CC_ERR_TIMEOUT
        assert waited > 3.0                              # the 4 s bound ran out
        # the hook applied to one call: the next ones are exact again
        for algo, a in (("cw", 2), ("c4", 1)):
            lab, r, d = graph.cluster(algo, 0.5, 7)
            elab, er, _, _ = ora.rounds(g.off, g.col, order, a, 0.5)
            assert np.array_equal(lab, elab) and r == er
        # a hook past the last round changes nothing
        graph.debug_withhold_release(orr + 5)
        lab, r, d = graph.cluster("cw", 0.5, 7)
        assert np.array_equal(lab, olab) and r == orr
        with pytest.raises(cc.CCError):
            graph.debug_withhold_release(-1)
        # a call that fails its argument checks consumes the hook too
        graph.debug_withhold_release(1)
        with pytest.raises(cc.CCError) as ei:
            graph.cluster("cw", 1.5, 7)
        assert ei.value.status == -1
        lab, r, d = graph.cluster("cw", 0.5, 7)
        assert np.array_equal(lab, olab) and r == orr


def test_asynchronous_call_consumes_the_hook(cc, gg):
    g = gg.rmat(10, 8, seed=1)
    with cc.Graph(g.off, g.col) as graph:
        graph.debug_withhold_release(0)
        graph.cluster("c4-async", 0.5, 1)            # consumes the hook without effect
        lab, r, d = graph.cluster("cw", 0.5, 1)      # runs to the end
        assert r > 0
