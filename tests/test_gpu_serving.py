"""Serving loop: continuous batching returns, for every request, exactly the
result of the same standalone clustering, whatever else is in flight."""
import threading
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


def serve_graphs(gg):
    return [gg.chung_lu(n, d, seed=70 + i) for i, (n, d) in
            enumerate([(500, 6.0), (3000, 20.0), (12000, 10.0), (40000, 30.0), (65000, 8.0)])]


def test_results_same_alone_and_in_the_mix(cc, ora, gg):
    import torch
    gs = serve_graphs(gg)
    graphs = [cc.Graph(g.off, g.col) for g in gs]
    rng = np.random.default_rng(5)
    reqs = [(int(rng.integers(len(gs))), ["cw", "c4"][int(rng.integers(2))], int(rng.integers(1 << 40)))
            for _ in range(120)]
    outs = [torch.full((gs[i].n,), -1, dtype=torch.int32, device="cuda") for i, _, _ in reqs]
    try:
        with cc.Server(mem_budget=2 << 30, max_batch=64) as srv:
            tickets = []
            for q, (i, algo, seed) in enumerate(reqs):
                tickets.append(srv.submit(graphs[i], algo, 0.5, seed, labels_out=outs[q]))
                if q % 17 == 0:
                    time.sleep(0.002)           # arrivals while earlier batches run
            res = [srv.wait(t) for t in tickets]
        torch.cuda.synchronize()
        for q, (i, algo, seed) in enumerate(reqs):
            lab, r, d = graphs[i].cluster(algo, 0.5, seed)
            assert (res[q][0], res[q][1]) == (r, d), q
            assert np.array_equal(outs[q].cpu().numpy(), lab), q
            assert res[q][2] >= 0.0
        # and against the oracle for a few
        for q in range(0, len(reqs), 23):
            i, algo, seed = reqs[q]
            g = gs[i]
            olab, orr, _, _ = ora.rounds(g.off, g.col, ora.permutation(g.n, seed), 1 if algo == "c4" else 2, 0.5)
            assert np.array_equal(outs[q].cpu().numpy(), olab) and res[q][0] == orr
    finally:
        for x in graphs:
            x.close()


def test_submissions_from_several_threads(cc, gg):
    gs = serve_graphs(gg)[:3]
    graphs = [cc.Graph(g.off, g.col) for g in gs]
    out = {}
    try:
        with cc.Server(mem_budget=1 << 30, max_batch=16) as srv:
            def client(c):
                for k in range(20):
                    t = srv.submit(graphs[(c + k) % len(gs)], "cw", 0.9, 1000 * c + k)
                    out[(c, k)] = srv.wait(t)
            th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
            for x in th:
                x.start()
            for x in th:
                x.join()
        for (c, k), (r, d, _) in out.items():
            _, r2, d2 = graphs[(c + k) % len(gs)].cluster("cw", 0.9, 1000 * c + k, want_labels=False)
            assert (r, d) == (r2, d2)
        assert len(out) == 80
    finally:
        for x in graphs:
            x.close()


def test_admission_by_memory(cc, gg):
    g = gg.chung_lu(60000, 16.0, seed=3)
    graph = cc.Graph(g.off, g.col)
    try:
        # room for one job's scratch at a time: still every request completes
        with cc.Server(mem_budget=12 << 20, max_batch=8) as srv:
            ts = [srv.submit(graph, "cw", 0.5, s) for s in range(6)]
            res = [srv.wait(t) for t in ts]
        for s, (r, d, _) in enumerate(res):
            _, r2, d2 = graph.cluster("cw", 0.5, s, want_labels=False)
            assert (r, d) == (r2, d2)
        # a budget below one job's scratch can never admit it
        with cc.Server(mem_budget=1 << 16, max_batch=8) as srv:
            t = srv.submit(graph, "cw", 0.5, 0)
            with pytest.raises(cc.CCError) as ei:
                srv.wait(t)
            assert ei.value.status == -3
    finally:
        graph.close()
