"""CPU oracle for parallel correlation clustering -- TEST INFRASTRUCTURE ONLY.

Plain serial C (``cc_oracle.c``) behind ctypes.  It computes, slowly and
literally, what the paper "Parallel Correlation Clustering on Big Graphs"
defines: the permutation pi, KwikCluster (Alg. 1), the C4 and ClusterWild!
rounds (Alg. 2), the disagreement objective (Sec. 2 definition), the exhaustive
optimum for tiny graphs and the KwikCluster cost summed over every permutation.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  The CUDA library never links it and
this package never imports the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcc_oracle.so")
_lock = threading.Lock()
_lib = None

ALGO_C4 = 1
ALGO_CW = 2

ROUND_STAT_FIELDS = ("n_alive", "delta", "k", "centers", "removed", "blocked")


class _RoundStat(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ROUND_STAT_FIELDS]


def build(force: bool = False) -> str:
    """Compile ``cc_oracle.c`` into ``_build/libcc_oracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared",
                           "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, u64, i32p, i64p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p
        lib.orc_splitmix64.restype = u64
        lib.orc_splitmix64.argtypes = [u64]
        lib.orc_perm_key.restype = u64
        lib.orc_perm_key.argtypes = [u64, i64]
        lib.orc_permutation.restype = ctypes.c_int
        lib.orc_permutation.argtypes = [i64, u64, i32p]
        lib.orc_kwik.restype = ctypes.c_int
        lib.orc_kwik.argtypes = [i64, i64p, i32p, i32p, i32p]
        lib.orc_batch_size.restype = i64
        lib.orc_batch_size.argtypes = [i64, i64, i64]
        lib.orc_rounds.restype = ctypes.c_int
        lib.orc_rounds.argtypes = [i64, i64p, i32p, i32p, ctypes.c_int, i64, ctypes.c_int,
                                   i32p, i64p, i32p, ctypes.c_void_p, i64]
        lib.orc_rounds_bsp.restype = ctypes.c_int
        lib.orc_rounds_bsp.argtypes = [i64, i64p, i32p, i32p, ctypes.c_int, i64, u64,
                                       i32p, i64p, i32p, ctypes.c_void_p, i64]
        lib.orc_bsp_period.restype = i64
        lib.orc_bsp_period.argtypes = [i64, i64, i64]
        lib.orc_bsp_delta_hat.restype = i64
        lib.orc_bsp_delta_hat.argtypes = [i64, i64, i64]
        lib.orc_bsp_threshold.restype = u64
        lib.orc_bsp_threshold.argtypes = [i64, i64, ctypes.POINTER(ctypes.c_int)]
        lib.orc_bsp_batch.restype = i64
        lib.orc_bsp_batch.argtypes = [u64, i64, i64, u64, ctypes.c_int]
        lib.orc_disagreements_pairs.restype = i64
        lib.orc_disagreements_pairs.argtypes = [i64, i64p, i32p, i32p]
        lib.orc_disagreements.restype = i64
        lib.orc_disagreements.argtypes = [i64, i64p, i32p, i32p]
        lib.orc_opt_bruteforce.restype = i64
        lib.orc_opt_bruteforce.argtypes = [ctypes.c_int, ctypes.c_void_p, i64p, i32p]
        lib.orc_kwik_all_perms_total.restype = i64
        lib.orc_kwik_all_perms_total.argtypes = [ctypes.c_int, ctypes.c_void_p, i64p, i64p, i64p]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _csr(off, col):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
    return off, col


def eps_to_ppm(eps: float) -> int:
    """Reading R4: eps in parts per million, rounded to nearest."""
    return int(round(float(eps) * 1_000_000))


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(ctypes.c_uint64(x & (2**64 - 1))))


def perm_key(seed: int, v: int) -> int:
    return int(_load().orc_perm_key(ctypes.c_uint64(seed & (2**64 - 1)), v))


def permutation(n: int, seed: int) -> np.ndarray:
    """order[r] = vertex of rank r under ascending (splitmix64(seed ^ v), v)."""
    order = np.empty(max(n, 1), np.int32)
    rc = _load().orc_permutation(n, ctypes.c_uint64(seed & (2**64 - 1)), _p(order))
    if rc != 0:
        raise RuntimeError(f"orc_permutation failed: {rc}")
    return order[:n]


def kwik(off, col, order) -> np.ndarray:
    """KwikCluster with pi (Alg. 1); label = center vertex id."""
    off, col = _csr(off, col)
    n = off.size - 1
    order = np.ascontiguousarray(order, dtype=np.int32)
    lab = np.empty(max(n, 1), np.int32)
    rc = _load().orc_kwik(n, _p(off), _p(col), _p(order), _p(lab))
    if rc != 0:
        raise RuntimeError(f"orc_kwik failed: {rc}")
    return lab[:n]


def batch_size(eps_ppm: int, n_i: int, delta_i: int) -> int:
    return int(_load().orc_batch_size(eps_ppm, n_i, delta_i))


def rounds(off, col, order, algo: int, eps: float, delta_mode: int = 1,
           stats_cap: int = 0, want_active_round: bool = False):
    """C4 / ClusterWild! rounds (Alg. 2), serial.

    Returns (labels, rounds, active_round or None, stats dict of arrays or None).
    """
    off, col = _csr(off, col)
    n = off.size - 1
    order = np.ascontiguousarray(order, dtype=np.int32)
    lab = np.empty(max(n, 1), np.int32)
    nr = np.zeros(1, np.int64)
    ar = np.empty(max(n, 1), np.int32) if want_active_round else None
    st = (_RoundStat * stats_cap)() if stats_cap > 0 else None
    rc = _load().orc_rounds(n, _p(off), _p(col), _p(order), algo, eps_to_ppm(eps), delta_mode,
                            _p(lab), _p(nr), _p(ar) if ar is not None else ctypes.c_void_p(0),
                            ctypes.cast(st, ctypes.c_void_p) if st is not None else ctypes.c_void_p(0),
                            stats_cap)
    if rc != 0:
        raise RuntimeError(f"orc_rounds failed: {rc}")
    r = int(nr[0])
    stats = None
    if st is not None:
        cnt = min(r, stats_cap)
        stats = {f: np.array([getattr(st[i], f) for i in range(cnt)], np.int64)
                 for f in ROUND_STAT_FIELDS}
    return lab[:n], r, (ar[:n] if ar is not None else None), stats



def bsp_period(n: int, max_deg: int, eps: float) -> int:
    """Rounds between two halvings of Delta-hat (Sec. 5, reading R13)."""
    return int(_load().orc_bsp_period(n, max_deg, eps_to_ppm(eps)))


def bsp_delta_hat(max_deg: int, period: int, round_: int) -> int:
    return int(_load().orc_bsp_delta_hat(max_deg, period, round_))


def bsp_threshold(eps: float, delta_hat: int):
    """(T, all): a trial succeeds when its draw is below T, or always (R14)."""
    a = ctypes.c_int(0)
    t = int(_load().orc_bsp_threshold(eps_to_ppm(eps), delta_hat, ctypes.byref(a)))
    return t, bool(a.value)


def bsp_batch(seed: int, round_: int, trials: int, thr: int, all_: bool) -> int:
    """B_i: successes among `trials` Bernoulli trials of round `round_` (R14)."""
    return int(_load().orc_bsp_batch(ctypes.c_uint64(seed & (2**64 - 1)), round_, trials,
                                      ctypes.c_uint64(thr), 1 if all_ else 0))


def rounds_bsp(off, col, order, algo: int, eps: float, seed: int, stats_cap: int = 0,
               want_active_round: bool = False):
    """C4 / ClusterWild! rounds with the practical schedule of Sec. 5 (Delta-hat
    halving, binomial batches over the unprocessed suffix of pi; seed = the
    seed of pi).  Returns (labels, rounds, active_round or None, stats or None)."""
    off, col = _csr(off, col)
    n = off.size - 1
    order = np.ascontiguousarray(order, dtype=np.int32)
    lab = np.empty(max(n, 1), np.int32)
    nr = np.zeros(1, np.int64)
    ar = np.empty(max(n, 1), np.int32) if want_active_round else None
    st = (_RoundStat * stats_cap)() if stats_cap > 0 else None
    rc = _load().orc_rounds_bsp(n, _p(off), _p(col), _p(order), algo, eps_to_ppm(eps),
                                ctypes.c_uint64(seed & (2**64 - 1)), _p(lab), _p(nr),
                                _p(ar) if ar is not None else ctypes.c_void_p(0),
                                ctypes.cast(st, ctypes.c_void_p) if st is not None else ctypes.c_void_p(0),
                                stats_cap)
    if rc != 0:
        raise RuntimeError(f"orc_rounds_bsp failed: {rc}")
    r = int(nr[0])
    stats = None
    if st is not None:
        cnt = min(r, stats_cap)
        stats = {f: np.array([getattr(st[i], f) for i in range(cnt)], np.int64)
                 for f in ROUND_STAT_FIELDS}
    return lab[:n], r, (ar[:n] if ar is not None else None), stats

def disagreements_pairs(off, col, labels) -> int:
    """O(n^2) recount over all unordered pairs (Sec. 2 definition)."""
    off, col = _csr(off, col)
    n = off.size - 1
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    return int(_load().orc_disagreements_pairs(n, _p(off), _p(col), _p(lab)))


def disagreements(off, col, labels) -> int:
    """m - 2*intra + sum_c C(s_c, 2) (Sec. 2 definition, counted)."""
    off, col = _csr(off, col)
    n = off.size - 1
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    if n == 0:
        return 0
    return int(_load().orc_disagreements(n, _p(off), _p(col), _p(lab)))


def opt_bruteforce(adj: np.ndarray):
    """Exhaustive OPT over all set partitions; returns (OPT, #partitions, labels)."""
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    n = adj.shape[0]
    cnt = np.zeros(1, np.int64)
    lab = np.empty(n, np.int32)
    best = _load().orc_opt_bruteforce(n, _p(adj), _p(cnt), _p(lab))
    if best < 0:
        raise RuntimeError("orc_opt_bruteforce: n out of range")
    return int(best), int(cnt[0]), lab


def kwik_all_perms_total(adj: np.ndarray):
    """Sum of KwikCluster cost over all n! orders; returns (total, n!, worst, best)."""
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    n = adj.shape[0]
    perms = np.zeros(1, np.int64)
    worst = np.zeros(1, np.int64)
    bestc = np.zeros(1, np.int64)
    tot = _load().orc_kwik_all_perms_total(n, _p(adj), _p(perms), _p(worst), _p(bestc))
    if tot < 0:
        raise RuntimeError("orc_kwik_all_perms_total: n out of range")
    return int(tot), int(perms[0]), int(worst[0]), int(bestc[0])
