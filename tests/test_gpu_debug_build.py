"""The bounds-checked build (nvcc -DCC_DEBUG): every list append, heavy-list
entry, member count and neighbour index of the round kernel is checked
against its array before the access.  On valid graphs no check fires and the
results are the oracle's; the checks run in a separate process that loads
the debug library (CC_DEBUG_BUILD=1)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, sys
sys.path.insert(0, {root!r})
import graphgen, oracle
import paper_1507_05086_gb300 as cc
from paper_1507_05086_gb300 import native
assert native.lib_path().endswith("_build_debug/libcc.so")
graphgen.build(); oracle.build()
graphs = [graphgen.rmat(14, 16, seed=3), graphgen.chung_lu(40_000, 20.0, seed=5),
          graphgen.planted_partition(n=30_000, q=80, seed=1, noise=50_000)]
for g in graphs:
    with cc.Graph(g.off, g.col) as graph:
        for algo, a in (("c4", 1), ("cw", 2)):
            for eps, seed in ((0.1, 4), (0.9, 5)):
                order = oracle.permutation(g.n, seed)
                olab, orr, _, _ = oracle.rounds(g.off, g.col, order, a, eps)
                lab, r, d = graph.cluster(algo, eps, seed)
                assert np.array_equal(lab, olab) and r == orr, (algo, eps)
        seeds = np.array([7], np.uint64)
        D, R = cc.batch_jobs([graph], "c4", 0.5, seeds, 2)
        for j in range(2):
            olab, orr, _, _ = oracle.rounds(g.off, g.col, oracle.permutation(g.n, 7 + j), 1, 0.5)
            assert R[0, j] == orr and D[0, j] == oracle.disagreements(g.off, g.col, olab)
print("DEBUG BUILD OK")
"""


def test_bounds_checked_build_gives_the_oracle_results():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, CC_DEBUG_BUILD="1")
    p = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=1200)
    assert p.returncode == 0 and "DEBUG BUILD OK" in p.stdout, p.stdout[-2000:] + p.stderr[-4000:]
