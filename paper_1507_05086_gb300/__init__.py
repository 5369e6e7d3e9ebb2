"""GB300-native parallel correlation clustering (C4 and ClusterWild!).

The bulk-synchronous rounds of "Parallel Correlation Clustering on Big Graphs"
(Pan et al., 2015; Alg. 2) and the disagreement objective, as hand-written
sm_103a CUDA kernels behind the C ABI of ``include/cc.h``.  This package is a
thin ctypes binding over that library.
"""
from .native import (ALGOS, C4, CLUSTERWILD, CCError, Graph, ROUND_STAT_FIELDS, Server, Tuning, batch_jobs,
                     batch_run, default_tuning, get_batch_tuning, lib_path, load, release_memory,
                     set_batch_tuning)

__all__ = ["ALGOS", "C4", "CLUSTERWILD", "CCError", "Graph", "ROUND_STAT_FIELDS", "Server", "Tuning", "batch_jobs",
           "batch_run", "default_tuning", "get_batch_tuning", "lib_path", "load", "release_memory",
           "set_batch_tuning"]
