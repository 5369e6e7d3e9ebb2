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


def test_batches_overlap_on_the_device_across_size_classes(cc, ora, gg):
    """Continuous batching: requests that arrive while an earlier batch runs
    start on the device before that batch ends (device clock stamps of every
    job), medium graphs run as teams of blocks and a graph above 2^21 vertices
    on the whole GPU at the same time, and every result equals the standalone
    clustering (and the oracle for a sample)."""
    import torch
    small = [gg.chung_lu(n, 16.0, seed=90 + i) for i, n in enumerate((30000, 45000, 60000))]
    medium = gg.chung_lu(300_000, 12.0, seed=95)
    large = gg.rmat(22, 8, seed=96)
    assert large.n > 1 << 21 and (1 << 16) < medium.n <= (1 << 21)
    graphs = [cc.Graph(g.off, g.col) for g in small + [medium, large]]
    gsets = small + [medium, large]
    reqs = []
    try:
        with cc.Server(mem_budget=16 << 30, max_batch=128) as srv:
            srv.wait(srv.submit(graphs[0], "cw", 0.1, 1))          # warm-up
            wave1, wave2 = [], []
            # wave 1: long jobs (a small eps means many rounds); wave 2 (another
            # algorithm, so never the same launch) arrives right behind it
            for q in range(96):
                i = q % 3
                reqs.append((i, "cw", 0.02, 1000 + q))
                wave1.append(srv.submit(graphs[i], "cw", 0.02, 1000 + q))
            for q in range(48):
                i = q % 3
                reqs.append((i, "c4", 0.5, 5000 + q))
                wave2.append(srv.submit(graphs[i], "c4", 0.5, 5000 + q))
            t_mid = srv.submit(graphs[3], "c4", 0.5, 7)              # a team job
            t_big = srv.submit(graphs[4], "cw", 0.5, 8)              # the whole GPU
            res = [srv.wait(t) for t in wave1 + wave2]
            r_mid, r_big = srv.wait(t_mid), srv.wait(t_big)
            times1 = [srv.device_times(t) for t in wave1]
            times2 = [srv.device_times(t) for t in wave2]
            tm = srv.device_times(t_mid)
            assert srv.device_times(t_big) == (-1, -1)
        assert all(a > 0 and b >= a for a, b in times1 + times2 + [tm])
        end1 = max(b for _, b in times1)
        start2 = min(a for a, _ in times2)
        assert start2 < end1, ("the second wave must start on the device while the first still runs",
                               (end1 - min(a for a, _ in times1)) / 1e6, (start2 - end1) / 1e6)
        for (i, algo, eps, seed), (r, d, _) in zip(reqs, res):
            _, r2, d2 = graphs[i].cluster(algo, eps, seed, want_labels=False)
            assert (r, d) == (r2, d2), (i, algo, seed)
        _, r2, d2 = graphs[3].cluster("c4", 0.5, 7, want_labels=False)
        assert (r_mid[0], r_mid[1]) == (r2, d2)
        _, r2, d2 = graphs[4].cluster("cw", 0.5, 8, want_labels=False)
        assert (r_big[0], r_big[1]) == (r2, d2)
        g = medium
        kc = ora.kwik(g.off, g.col, ora.permutation(g.n, 7))
        assert r_mid[1] == ora.disagreements(g.off, g.col, kc)
        for k in (0, 50, 100, 140):
            i, algo, eps, seed = reqs[k]
            g = gsets[i]
            olab, orr, _, _ = ora.rounds(g.off, g.col, ora.permutation(g.n, seed), 1 if algo == "c4" else 2, eps)
            assert res[k][0] == orr and res[k][1] == ora.disagreements(g.off, g.col, olab)
    finally:
        for x in graphs:
            x.close()


def test_a_failed_batch_does_not_stop_the_server(cc, gg):
    """A request whose scratch can never fit fails alone; later requests are
    served normally."""
    g_small = gg.chung_lu(2000, 8.0, seed=1)
    g_big = gg.chung_lu(60000, 16.0, seed=2)
    a, b = cc.Graph(g_small.off, g_small.col), cc.Graph(g_big.off, g_big.col)
    try:
        with cc.Server(mem_budget=4 << 20, max_batch=8) as srv:
            t_bad = srv.submit(b, "cw", 0.5, 3)
            with pytest.raises(cc.CCError) as ei:
                srv.wait(t_bad)
            assert ei.value.status == -3
            ts = [srv.submit(a, "cw", 0.5, s) for s in range(5)]
            res = [srv.wait(t) for t in ts]
        for s, (r, d, _) in enumerate(res):
            _, r2, d2 = a.cluster("cw", 0.5, s, want_labels=False)
            assert (r, d) == (r2, d2)
    finally:
        a.close()
        b.close()
