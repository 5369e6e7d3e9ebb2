"""ctypes binding of ``libcc.so`` (the C ABI in ``include/cc.h``).

Argument marshalling only: every step of the clustering runs in the
library's CUDA kernels.  Arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA); torch is used for device memory and streams only.
If the library is missing or fails to load, every call raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

C4 = 1
CLUSTERWILD = 2
C4_EST = 3              # the same with the practical schedule of Sec. 5
CLUSTERWILD_EST = 4
C4_ASYNC = 5            # C4 without rounds (Alg. 3); cluster() only
ALGOS = {"c4": C4, "cw": CLUSTERWILD, "clusterwild": CLUSTERWILD, "c4-est": C4_EST, "cw-est": CLUSTERWILD_EST,
         "c4-async": C4_ASYNC,
         C4: C4, CLUSTERWILD: CLUSTERWILD, C4_EST: C4_EST, CLUSTERWILD_EST: CLUSTERWILD_EST, C4_ASYNC: C4_ASYNC}

CC_DEVICE_PTRS = 2
CC_OFFSETS_I32 = 4
CC_VALIDATE_EXACT = 8

STATUS = {
    0: "ok", -1: "invalid argument", -2: "invalid graph", -3: "out of memory", -4: "CUDA error",
    -5: "device wait timed out", -6: "busy", -7: "internal consistency check failed",
}

ROUND_STAT_FIELDS = ("n_alive", "delta", "k", "centers", "removed", "blocked", "edges", "ns")


class RoundStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ROUND_STAT_FIELDS]


TUNING_FIELDS = (("walk_batches", ctypes.c_int32), ("prefetch_ahead", ctypes.c_int32),
                 ("inline_heavy", ctypes.c_int32), ("inline_decide", ctypes.c_int32),
                 ("inline_rebuild", ctypes.c_int32), ("heavy_shift", ctypes.c_int32),
                 ("batch_small_n", ctypes.c_int64), ("batch_team_n", ctypes.c_int64),
                 ("batch_team_blocks", ctypes.c_int32), ("warp_resolve_row", ctypes.c_int32))


class Tuning(ctypes.Structure):
    """cc_tuning: schedule settings, none of which changes a result."""
    _fields_ = list(TUNING_FIELDS)

    def to_dict(self):
        return {f: int(getattr(self, f)) for f, _ in TUNING_FIELDS}

    @classmethod
    def from_dict(cls, d):
        t = default_tuning()
        for k, v in d.items():
            setattr(t, k, int(v))
        return t


class CCError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {STATUS.get(status, 'unknown')} ({status})")
        self.status = status


_lock = threading.Lock()
_lib = None


def debug_build_requested() -> bool:
    """CC_DEBUG_BUILD=1 in the environment selects the bounds-checked library."""
    return os.environ.get("CC_DEBUG_BUILD", "") not in ("", "0")


def lib_path() -> str:
    return _build.LIB_DEBUG if debug_build_requested() else _build.LIB


def load(build_if_missing: bool = True):
    """Load libcc.so (building it first if it is missing or stale); the
    bounds-checked variant when CC_DEBUG_BUILD=1."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        debug = debug_build_requested()
        path = _build.LIB_DEBUG if debug else _build.LIB
        if build_if_missing and not _build.up_to_date(debug):
            _build.build(debug=debug)
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_1507_05086_gb300.build)")
        lib = ctypes.CDLL(path)
        vp, i64, i32, u32, u64, ci = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_int)
        lib.cc_status_string.restype = ctypes.c_char_p
        lib.cc_release_memory.restype = ci
        lib.cc_release_memory.argtypes = []
        lib.cc_status_string.argtypes = [ci]
        lib.cc_graph_create.restype = ci
        lib.cc_graph_create.argtypes = [i64, vp, vp, u32, vp, ctypes.POINTER(vp)]
        lib.cc_graph_destroy.restype = ci
        lib.cc_graph_destroy.argtypes = [vp]
        lib.cc_graph_info.restype = ci
        lib.cc_graph_info.argtypes = [vp, vp, vp, vp]
        lib.cc_permutation.restype = ci
        lib.cc_permutation.argtypes = [vp, u64, vp]
        lib.cc_cluster.restype = ci
        lib.cc_cluster.argtypes = [vp, ci, ctypes.c_double, u64, vp, vp, vp]
        lib.cc_cluster_ex.restype = ci
        lib.cc_cluster_ex.argtypes = [vp, ci, ctypes.c_double, u64, vp, vp, vp, vp, i32, vp]
        lib.cc_disagreements.restype = ci
        lib.cc_disagreements.argtypes = [vp, vp, vp]
        lib.cc_graph_set_timing.restype = ci
        lib.cc_graph_set_timing.argtypes = [vp, ci]
        lib.cc_last_timings.restype = ci
        lib.cc_last_timings.argtypes = [vp, vp]
        lib.cc_last_phase_times.restype = ci
        lib.cc_last_phase_times.argtypes = [vp, vp, i32]
        lib.cc_debug_withhold_release.restype = ci
        lib.cc_debug_withhold_release.argtypes = [vp, i32]
        lib.cc_disagreements_static.restype = ci
        lib.cc_disagreements_static.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.cc_batch_jobs.restype = ci
        lib.cc_batch_jobs.argtypes = [vp, i32, ci, ctypes.c_double, vp, i32, vp, vp]
        lib.cc_server_create.restype = ci
        lib.cc_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
        lib.cc_server_submit.restype = ci
        lib.cc_server_submit.argtypes = [vp, vp, ci, ctypes.c_double, u64, vp, vp]
        lib.cc_server_poll.restype = ci
        lib.cc_server_poll.argtypes = [vp, i64, vp, vp, vp]
        lib.cc_server_wait.restype = ci
        lib.cc_server_wait.argtypes = [vp, i64, vp, vp, vp]
        lib.cc_server_device_times.restype = ci
        lib.cc_server_device_times.argtypes = [vp, i64, vp, vp]
        lib.cc_server_destroy.restype = ci
        lib.cc_server_destroy.argtypes = [vp]
        for f in ("cc_tuning_default", "cc_get_batch_tuning", "cc_set_batch_tuning"):
            getattr(lib, f).restype = ci
            getattr(lib, f).argtypes = [vp]
        for f in ("cc_graph_set_tuning", "cc_graph_get_tuning"):
            getattr(lib, f).restype = ci
            getattr(lib, f).argtypes = [vp, vp]
        lib.cc_batch_run.restype = ci
        lib.cc_batch_run.argtypes = [vp, i32, ci, ctypes.c_double, vp, i32, vp, vp, vp, vp]
        _lib = lib
        return lib


def _check(fn: str, rc: int):
    if rc != 0:
        raise CCError(fn, rc)


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data if a.size else None
    return a.data_ptr() if a.numel() else None


def _is_cuda(a) -> bool:
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def current_stream_handle():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:   # torch without CUDA: legacy stream
        pass
    return None


class Graph:
    """A graph resident on the GPU (``cc_graph``).

    ``off``/``col``: int64[n+1] / int32[nnz] CSR of the positive edges, as numpy
    arrays (copied to the device) or CUDA torch tensors (adopted by reference;
    keep them alive).
    """

    def __init__(self, off, col, stream=None, exact_symmetry: bool = False):
        lib = load()
        self._lib = lib
        n = int(off.shape[0] - 1)
        flags = CC_VALIDATE_EXACT if exact_symmetry else 0
        self._keep = None
        if _is_cuda(off) or _is_cuda(col):
            import torch
            off = off.to(torch.int64).contiguous()
            col = col.to(torch.int32).contiguous()
            flags |= CC_DEVICE_PTRS
            self._keep = (off, col)
        else:
            off = np.ascontiguousarray(off, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
        if stream is None:
            stream = current_stream_handle()
        h = ctypes.c_void_p()
        _check("cc_graph_create", lib.cc_graph_create(n, _ptr(off), _ptr(col), flags, stream, ctypes.byref(h)))
        self._h = h
        nn, nnz, md = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check("cc_graph_info", lib.cc_graph_info(h, ctypes.byref(nn), ctypes.byref(nnz), ctypes.byref(md)))
        self.n, self.nnz, self.max_degree = nn.value, nnz.value, md.value

    @property
    def m(self) -> int:
        return self.nnz // 2

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def permutation(self, seed: int, out=None):
        out = np.empty(self.n, np.int32) if out is None else out
        _check("cc_permutation", self._lib.cc_permutation(self._h, seed & (2**64 - 1), _ptr(out)))
        return out

    def cluster(self, algo="cw", eps: float = 0.5, seed: int = 0, labels_out=None, want_labels=True,
                stats_cap: int = 0):
        """Run one clustering.  Returns (labels, rounds, disagreements[, stats])."""
        a = ALGOS[algo]
        if labels_out is None and want_labels:
            labels_out = np.empty(self.n, np.int32)
        rounds = ctypes.c_int32()
        d = ctypes.c_int64()
        if stats_cap > 0:
            st = (RoundStats * stats_cap)()
            ln = ctypes.c_int32()
            _check("cc_cluster_ex", self._lib.cc_cluster_ex(
                self._h, a, float(eps), seed & (2**64 - 1), _ptr(labels_out), ctypes.byref(rounds),
                ctypes.byref(d), ctypes.cast(st, ctypes.c_void_p), stats_cap, ctypes.byref(ln)))
            cnt = min(ln.value, stats_cap)
            stats = {f: np.array([getattr(st[i], f) for i in range(cnt)], np.int64) for f in ROUND_STAT_FIELDS}
            return labels_out, rounds.value, d.value, stats
        _check("cc_cluster", self._lib.cc_cluster(self._h, a, float(eps), seed & (2**64 - 1), _ptr(labels_out),
                                                  ctypes.byref(rounds), ctypes.byref(d)))
        return labels_out, rounds.value, d.value

    def set_tuning(self, tuning):
        """Schedule settings of this graph's clusterings (a Tuning or a dict of
        its fields; missing fields keep their defaults)."""
        t = tuning if isinstance(tuning, Tuning) else Tuning.from_dict(tuning)
        _check("cc_graph_set_tuning", self._lib.cc_graph_set_tuning(self._h, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = Tuning()
        _check("cc_graph_get_tuning", self._lib.cc_graph_get_tuning(self._h, ctypes.byref(t)))
        return t.to_dict()

    def set_timing(self, enable: bool = True):
        _check("cc_graph_set_timing", self._lib.cc_graph_set_timing(self._h, 1 if enable else 0))

    def last_timings(self):
        """(permutation, rounds kernel, labels) milliseconds of the last clustering."""
        ms = (ctypes.c_float * 3)()
        _check("cc_last_timings", self._lib.cc_last_timings(self._h, ctypes.cast(ms, ctypes.c_void_p)))
        return tuple(float(x) for x in ms)

    PHASES = ("delta_scan", "delta_rebuild", "sec5_draws", "select", "centers_attach",
              "c4_fixpoint", "removal_decrement")

    def debug_withhold_release(self, round_: int):
        """Test hook: the next clustering withholds its barrier release after
        round `round_`; the other blocks' bounded waits run out and the call
        raises CCError with CC_ERR_TIMEOUT."""
        _check("cc_debug_withhold_release", self._lib.cc_debug_withhold_release(self._h, int(round_)))

    def last_phase_times(self):
        """Milliseconds per phase of the last clustering's round kernel."""
        ms = (ctypes.c_double * 7)()
        _check("cc_last_phase_times", self._lib.cc_last_phase_times(self._h, ctypes.cast(ms, ctypes.c_void_p), 7))
        return dict(zip(self.PHASES, (float(x) for x in ms)))

    def disagreements(self, labels) -> int:
        if isinstance(labels, np.ndarray):
            labels = np.ascontiguousarray(labels, dtype=np.int32)
        d = ctypes.c_int64()
        _check("cc_disagreements", self._lib.cc_disagreements(self._h, _ptr(labels), ctypes.byref(d)))
        return d.value


def default_tuning() -> Tuning:
    t = Tuning()
    _check("cc_tuning_default", load().cc_tuning_default(ctypes.byref(t)))
    return t


def set_batch_tuning(tuning):
    """Process-wide settings of batched jobs and servers created later."""
    t = tuning if isinstance(tuning, Tuning) else Tuning.from_dict(tuning)
    _check("cc_set_batch_tuning", load().cc_set_batch_tuning(ctypes.byref(t)))


def get_batch_tuning() -> dict:
    t = Tuning()
    _check("cc_get_batch_tuning", load().cc_get_batch_tuning(ctypes.byref(t)))
    return t.to_dict()


def release_memory():
    """Return the unused device memory the library's pools keep reserved."""
    _check("cc_release_memory", load().cc_release_memory())


def batch_jobs(graphs, algo="cw", eps=0.5, seeds=None, k_perms=8):
    """Every (graph, permutation) job of a batch: (D, rounds), each shaped
    (len(graphs), k_perms); job (i, j) uses seed seeds[i] + j."""
    lib = load()
    cnt = len(graphs)
    seeds = np.asarray(seeds if seeds is not None else np.zeros(cnt), dtype=np.uint64)
    hs = (ctypes.c_void_p * max(cnt, 1))(*[g._h.value for g in graphs])
    d = np.zeros(max(cnt * k_perms, 1), np.int64)
    r = np.zeros(max(cnt * k_perms, 1), np.int32)
    _check("cc_batch_jobs", lib.cc_batch_jobs(hs, cnt, ALGOS[algo], float(eps), seeds.ctypes.data, k_perms,
                                              d.ctypes.data, r.ctypes.data))
    return d[:cnt * k_perms].reshape(cnt, k_perms), r[:cnt * k_perms].reshape(cnt, k_perms)


def batch_run(graphs, algo="cw", eps=0.5, seeds=None, k_perms=8, want_labels=False):
    """Best-of-k over several graphs (``cc_batch_run``).

    Returns (best_j, best_D, rounds, labels list or None)."""
    lib = load()
    cnt = len(graphs)
    seeds = np.asarray(seeds if seeds is not None else np.zeros(cnt), dtype=np.uint64)
    hs = (ctypes.c_void_p * cnt)(*[g._h.value for g in graphs])
    best_j = np.zeros(cnt, np.int32)
    best_d = np.zeros(cnt, np.int64)
    rounds = np.zeros(cnt, np.int32)
    labels = None
    lab_arr = None
    if want_labels:
        labels = [np.empty(g.n, np.int32) for g in graphs]
        lab_arr = (ctypes.c_void_p * cnt)(*[l.ctypes.data if l.size else None for l in labels])
    _check("cc_batch_run", lib.cc_batch_run(hs, cnt, ALGOS[algo], float(eps), seeds.ctypes.data, k_perms,
                                            lab_arr, best_j.ctypes.data, best_d.ctypes.data, rounds.ctypes.data))
    return best_j, best_d, rounds, labels


class Server:
    """Serving loop with continuous batching (``cc_server_*``).

    ``submit`` returns a ticket at once; requests waiting when a stream frees
    up run together as one batched launch (per size class), overlapping on
    the device with earlier batches, within a device-memory budget for their
    scratch.
    """

    def __init__(self, mem_budget: int = 4 << 30, max_batch: int = 1024):
        self._lib = load()
        h = ctypes.c_void_p()
        _check("cc_server_create", self._lib.cc_server_create(int(mem_budget), int(max_batch), ctypes.byref(h)))
        self._h = h

    def submit(self, graph: Graph, algo="cw", eps: float = 0.5, seed: int = 0, labels_out=None) -> int:
        t = ctypes.c_int64()
        _check("cc_server_submit", self._lib.cc_server_submit(self._h, graph._h, ALGOS[algo], float(eps),
                                                              seed & (2**64 - 1), _ptr(labels_out),
                                                              ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (rounds, disagreements, latency_ms)."""
        r, d, ms = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double()
        rc = self._lib.cc_server_poll(self._h, ticket, ctypes.byref(r), ctypes.byref(d), ctypes.byref(ms))
        if rc == -6:
            return None
        _check("cc_server_poll", rc)
        return r.value, d.value, ms.value

    def wait(self, ticket: int):
        """(rounds, disagreements, latency_ms) of a request, blocking."""
        r, d, ms = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double()
        _check("cc_server_wait", self._lib.cc_server_wait(self._h, ticket, ctypes.byref(r), ctypes.byref(d),
                                                          ctypes.byref(ms)))
        return r.value, d.value, ms.value

    def device_times(self, ticket: int):
        """(start_ns, end_ns) of a finished request's job on the device clock
        (-1, -1 for requests that ran on the whole GPU)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check("cc_server_device_times", self._lib.cc_server_device_times(self._h, ticket, ctypes.byref(a),
                                                                           ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cc_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
