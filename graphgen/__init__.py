"""Seeded synthetic graph generators (shared input module).

Stand-ins for the paper's WebGraph datasets (Table 1), which are not
available: Erdos-Renyi, planted partition, R-MAT and Chung-Lu graphs, each
returned as a symmetric simple CSR ``(off int64[n+1], col int32[nnz])``.

This module contains none of the clustering method.  The oracle and the CUDA
library both consume its graphs; it imports neither.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O3", "-std=c++17", "-pthread", "-Wall", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, i64, u64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.gg_er.argtypes = [i64, dbl, u64, ci, pp]
        lib.gg_planted.argtypes = [i64, i64, i64, dbl, dbl, dbl, dbl, i64, u64, ci, pp]
        lib.gg_rmat.argtypes = [ci, i64, dbl, dbl, dbl, u64, ci, pp]
        lib.gg_chung_lu.argtypes = [i64, dbl, dbl, u64, ci, pp]
        lib.gg_from_edges.argtypes = [i64, vp, vp, i64, ci, pp]
        for f in ("gg_er", "gg_planted", "gg_rmat", "gg_chung_lu", "gg_from_edges"):
            getattr(lib, f).restype = ci
        for f in ("gg_n", "gg_nnz", "gg_aux_len"):
            getattr(lib, f).restype = i64
            getattr(lib, f).argtypes = [vp]
        lib.gg_copy.restype = ci
        lib.gg_copy.argtypes = [vp, vp, vp, vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        _lib = lib
        return lib


@dataclass
class Graph:
    """Symmetric simple CSR of the positive edges."""
    off: np.ndarray          # int64[n+1]
    col: np.ndarray          # int32[nnz], nnz = 2m
    aux: np.ndarray | None = None   # planted labels, when the generator has them
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.off.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.off[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def digest(self) -> str:
        h = hashlib.blake2b(digest_size=16)
        h.update(np.int64(self.n).tobytes())
        h.update(memoryview(self.off))
        h.update(memoryview(self.col[: self.nnz]))
        return h.hexdigest()


def _take(handle: ctypes.c_void_p, name: str) -> Graph:
    lib = _load()
    try:
        n = lib.gg_n(handle)
        nnz = lib.gg_nnz(handle)
        naux = lib.gg_aux_len(handle)
        off = np.empty(n + 1, np.int64)
        col = np.empty(max(nnz, 1), np.int32)
        aux = np.empty(naux, np.int32) if naux else None
        lib.gg_copy(handle, off.ctypes.data, col.ctypes.data, aux.ctypes.data if aux is not None else None)
    finally:
        lib.gg_free(handle)
    return Graph(off, col[:nnz], aux, name)


def _call(fn, *args, name=""):
    h = ctypes.c_void_p()
    rc = fn(*args, ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"graph generator failed ({rc})")
    return _take(h, name)


def erdos_renyi(n: int, p: float, seed: int = 0, threads: int = 0) -> Graph:
    return _call(_load().gg_er, n, p, seed, threads, name=f"er_n{n}_p{p:g}_s{seed}")


def planted_partition(n: int = 1_000_000, q: int = 2000, min_size: int = 5, zipf: float = 1.5,
                      p_max: float = 0.3, mean_intra: float = 30.0, drop: float = 0.1,
                      noise: int = 4_000_000, seed: int = 0, threads: int = 0) -> Graph:
    return _call(_load().gg_planted, n, q, min_size, zipf, p_max, mean_intra, drop, noise, seed,
                 threads, name=f"planted_n{n}_q{q}_s{seed}")


def rmat(scale: int, ef: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, threads: int = 0) -> Graph:
    return _call(_load().gg_rmat, scale, ef, a, b, c, seed, threads,
                 name=f"rmat_s{scale}_ef{ef}_seed{seed}")


def chung_lu(n: int, d: float, beta: float = 2.1, seed: int = 0, threads: int = 0) -> Graph:
    return _call(_load().gg_chung_lu, n, d, beta, seed, threads, name=f"chunglu_n{n}_d{d:g}_s{seed}")


def from_edges(n: int, u, v, threads: int = 0) -> Graph:
    u = np.ascontiguousarray(u, np.int32)
    v = np.ascontiguousarray(v, np.int32)
    return _call(_load().gg_from_edges, n, u.ctypes.data if u.size else None,
                 v.ctypes.data if v.size else None, int(u.size), threads, name=f"edges_n{n}")


def random_small(n: int, p: float, rng: np.random.Generator) -> Graph:
    """Tiny G(n,p) from a numpy generator (test fixtures)."""
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    return from_edges(n, iu[keep].astype(np.int32), ju[keep].astype(np.int32), threads=1)


def adjacency_matrix(g: Graph) -> np.ndarray:
    a = np.zeros((g.n, g.n), np.uint8)
    for u in range(g.n):
        a[u, g.col[g.off[u]:g.off[u + 1]]] = 1
    return a


# Named workloads: the synthetic stand-ins at the sizes the benchmark uses.
def chung_lu_batch_params(count: int = 4096, base_seed: int = 0):
    """(n_g, d_g, seed_g) of the Chung-Lu batch: n log-uniform in [1e3, 1e6],
    mean degree uniform in [8, 64], seed base + g."""
    out = []
    for g in range(count):
        s = np.random.default_rng(base_seed + g)
        u1, u2 = s.random(), s.random()
        out.append((int(round(10 ** (3 + 3 * u1))), 8.0 + 56.0 * u2, base_seed + g))
    return out


def chung_lu_device(n: int, d: float, beta: float = 2.1, seed: int = 0, device="cuda"):
    """Chung-Lu graph generated on a GPU with torch (for batches of thousands
    of graphs, where the host generator would take minutes): the same weights
    as chung_lu (w_i proportional to (i+1)^(-1/(beta-1)), scaled to mean degree
    d, capped at sqrt(n d)), round(n d / 2) endpoint pairs drawn by inverse
    CDF from torch's seeded uniforms, self loops dropped, both directions
    kept, duplicates merged.  Returns (off int64[n+1], col int32[nnz]) as
    device tensors; to_host() turns them into a Graph.  The graph depends on
    the seed and on torch's generator, so it is reproducible on one torch
    version; the oracle reads the same arrays through to_host()."""
    import torch
    dev = torch.device(device)
    i = torch.arange(1, n + 1, dtype=torch.float64, device=dev)
    w = i.pow(-1.0 / (beta - 1.0))
    w = torch.clamp(w * (d * n / float(w.sum())), max=float(np.sqrt(n * d)))
    cdf = torch.cumsum(w, 0)
    acc = float(cdf[-1])
    m = int(round(n * d / 2.0))
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) & (2**63 - 1))
    ends = []
    for _ in range(2):
        x = torch.rand(m, dtype=torch.float64, device=dev, generator=gen) * acc
        ends.append(torch.clamp(torch.searchsorted(cdf, x, right=True), max=n - 1))
    u, v = ends
    keep = u != v
    u, v = u[keep], v[keep]
    keys = torch.cat([u * n + v, v * n + u])
    del u, v, keep, ends
    keys = torch.unique(keys, sorted=True)
    rows = keys // n
    col = (keys - rows * n).to(torch.int32)
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(torch.bincount(rows, minlength=n), 0)
    return off, col


def to_host(off, col, name: str = "") -> Graph:
    """Host Graph from device CSR tensors (chung_lu_device)."""
    return Graph(off.cpu().numpy(), col.cpu().numpy(), None, name)


def workload(name: str, threads: int = 0) -> Graph:
    """'er10k' | 'planted1m' | 'rmat24' | 'rmat26' | 'rmat<scale>'."""
    if name == "er10k":
        return erdos_renyi(10_000, 20.0 / 9_999.0, seed=0, threads=threads)
    if name == "planted1m":
        return planted_partition(seed=0, threads=threads)
    if name.startswith("rmat"):
        return rmat(int(name[4:]), 16, seed=0, threads=threads)
    raise KeyError(name)
