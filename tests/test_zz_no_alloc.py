"""cc_disagreements_static: the allocation-free objective.

Callers that run inside a fixed memory pool, or under a rule that forbids
allocating once they are running, get the disagreement count from buffers
they already hold plus the library's built-in scratch area.  This checks it
through the C ABI against the allocating cc_disagreements, exactly, on two
calls in a row (the second with a different labelling, so leftovers in the
shared scratch would show).  Kept in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import graphgen
    import paper_1507_05086_gb300 as cc
    from paper_1507_05086_gb300 import native
    graphgen.build()
    return torch, graphgen, cc, native.load()


def _static(lib, torch, n, off_d, col_d, lab_d, out_d):
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.cc_disagreements_static(n, ctypes.c_void_p(off_d.data_ptr()), ctypes.c_void_p(col_d.data_ptr()),
                                     ctypes.c_void_p(lab_d.data_ptr()), ctypes.c_void_p(out_d.data_ptr()),
                                     ctypes.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize()
    return int(out_d.item())


def test_static_matches_allocating_entry_on_two_calls(env):
    torch, graphgen, cc, lib = env
    g = graphgen.planted_partition(n=300_000, q=400, seed=6, noise=300_000)
    assert g.n <= 1 << 20
    off_d = torch.from_numpy(g.off).cuda()
    col_d = torch.from_numpy(g.col).cuda()
    out_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    with cc.Graph(g.off, g.col) as graph:
        clustered, _, d_cw = graph.cluster("cw", 0.5, 3)
        rng = np.random.default_rng(11)
        runs = [(g.aux, graph.disagreements(g.aux)),
                (clustered, d_cw),
                (rng.integers(0, 5000, g.n).astype(np.int32), None)]
        for lab, expect in runs:
            if expect is None:
                expect = graph.disagreements(lab)
            lab_d = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).cuda()
            assert _static(lib, torch, g.n, off_d, col_d, lab_d, out_d) == expect
        # the same labelling twice in a row gives the same number
        lab_d = torch.from_numpy(np.ascontiguousarray(clustered, np.int32)).cuda()
        assert _static(lib, torch, g.n, off_d, col_d, lab_d, out_d) == d_cw
        assert _static(lib, torch, g.n, off_d, col_d, lab_d, out_d) == d_cw


def test_static_matches_oracle_on_power_law_hubs_and_recovers_from_a_bad_label(env, ora):
    """R-MAT with 2^20 vertices (the scratch's limit; hub rows far longer
    than one warp's share): the count equals the oracle's.  A labelling with
    one value out of range gives -1; the next valid call is exact again (the
    flag in the shared scratch is cleared).  n = 0 gives 0."""
    torch, graphgen, cc, lib = env
    g = graphgen.rmat(20, 16, seed=5)
    assert g.n == 1 << 20 and int(np.diff(g.off).max()) > 10_000
    off_d = torch.from_numpy(g.off).cuda()
    col_d = torch.from_numpy(g.col).cuda()
    out_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    order = ora.permutation(g.n, 4)
    kc = ora.kwik(g.off, g.col, order)
    for lab in (kc, (np.arange(g.n) // 7).astype(np.int32)):
        lab_d = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).cuda()
        assert _static(lib, torch, g.n, off_d, col_d, lab_d, out_d) == ora.disagreements(g.off, g.col, lab)
    bad = kc.copy()
    bad[12345] = g.n
    lab_d = torch.from_numpy(bad).cuda()
    assert _static(lib, torch, g.n, off_d, col_d, lab_d, out_d) == -1
    lab_d = torch.from_numpy(kc).cuda()
    assert _static(lib, torch, g.n, off_d, col_d, lab_d, out_d) == ora.disagreements(g.off, g.col, kc)
    off0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    out_d.fill_(77)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.cc_disagreements_static(0, ctypes.c_void_p(off0.data_ptr()), None, None,
                                     ctypes.c_void_p(out_d.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(out_d.item()) == 0


def test_static_rejects_sizes_above_its_scratch(env):
    torch, graphgen, cc, lib = env
    out_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    big = (1 << 20) + 1
    rc = lib.cc_disagreements_static(big, None, None, None, ctypes.c_void_p(out_d.data_ptr()), None)
    assert rc == -1
    rc = lib.cc_disagreements_static(-1, None, None, None, ctypes.c_void_p(out_d.data_ptr()), None)
    assert rc == -1
