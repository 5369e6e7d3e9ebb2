#!/usr/bin/env python
"""Benchmark: C4 and ClusterWild! clustering of a ~1B-edge graph on GB300.

Workload: R-MAT scale 26, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05),
symmetrised, deduplicated, self loops removed (1.052e9 undirected edges,
2.10e9 CSR entries), seeded synthetic stand-in for the billion-edge web crawls
of the paper's experiments.  One step = one C4 and one ClusterWild!
clustering at eps = 0.5, each on a fresh permutation: permutation, all Alg. 2
rounds, fused objective, labels written to device memory.  The CSR (8.6 GB)
and the state arrays (0.5 GB) are far larger than L2, so no flush is needed
between steps.

Metric: undirected edges clustered per second (m * clusterings / time).
Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same generator (R-MAT scale 22).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s clustered (C4 + ClusterWild!, eps=0.5) at 1B edges"
SAMPLE_SCALE = 22          # CPU sample: same R-MAT generator, 1/16 of the vertices
KERNELS_PER_CLUSTERING = 10  # 7 permutation kernels + state init + rounds + labels


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="rmat26")
    p.add_argument("--eps", type=float, default=0.5)
    p.add_argument("--algos", default="cw,c4")
    p.add_argument("--e2e-steps", type=int, default=4)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tune", type=int, default=1,
                   help="pick the schedule settings with the autotuner (cached per device and graph class)")
    p.add_argument("--configs", type=int, default=1,
                   help="also time the other workload configurations once each (0 = skip)")
    p.add_argument("--parity", type=int, default=1,
                   help="check the last timed step's labels against the oracle on the full graph (CPU leg)")
    p.add_argument("--batch-graphs", type=int, default=4096,
                   help="Chung-Lu graphs of the batched and served workload (0 = skip the batch leg)")
    p.add_argument("--sec5", type=int, default=1, help="also time the Sec. 5 schedule once per algorithm (0 = skip)")
    p.add_argument("--async-c4", type=int, default=1, help="also time C4 without rounds (Alg. 3) once (0 = skip)")
    p.add_argument("--serve-seconds", type=float, default=2.0,
                   help="length of the Poisson arrival stream for the serving measurement (0 = skip)")
    return p.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def step_seeds(rank: int, step: int, n_algos: int, base: int = 1000):
    """Seeds of one step on one rank: every (rank, step, algo) gets its own pi."""
    return [base + ((rank * 1_000_003 + step) * n_algos + i) for i in range(n_algos)]


def aggregate(edges_per_rank, ms_per_rank):
    """Whole-job throughput: all ranks' work over the slowest rank's time."""
    t = max(ms_per_rank)
    return sum(edges_per_rank) / (t / 1e3), t


def reduce_across_ranks(elapsed_ms: float, edges: int, world: int, device):
    """Whole-job throughput over all ranks: total edges over the slowest
    rank's time.  Every rank gets the same (value, max_ms)."""
    if world <= 1:
        return aggregate([edges], [elapsed_ms])
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    e = torch.tensor([float(edges)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return e.item() / (t.item() / 1e3), t.item()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_graph(workload: str):
    import graphgen
    graphgen.build()
    return graphgen.workload(workload)


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# DRAM traffic of the round kernel per algorithmic byte, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, a one-pass metric set, of the
# four k_rounds launches of `bench.py --steps 1 --warmup 1` on the
# default workload, R-MAT scale 26, eps 0.5: ClusterWild! 46.01 and 46.00 GB against
# 18.19 GB algorithmic, C4 46.03 and 46.05 GB against 18.79 GB), keyed by a digest of the
# kernel's code (comments and blank lines left out): a changed kernel reports
# traffic null until it is captured again.
ROUNDS_SOURCES = ("paper_1507_05086_gb300/csrc/cc_rounds.cu", "paper_1507_05086_gb300/csrc/cc_device.cuh",
                  "paper_1507_05086_gb300/csrc/cc_internal.h")
ROUNDS_TRAFFIC_PER_BYTE = {"23e42cca60e96365": (46.01e9 + 46.03e9 + 46.00e9 + 46.05e9) / (2 * (18.19e9 + 18.79e9))}


def rounds_sources_digest() -> str:
    """Digest of the round kernel's code: its sources without comments and
    blank lines (a comment edit leaves the compiled kernel unchanged)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ROUNDS_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measure_gather_ceiling(torch, device, table_words: int = 1 << 23, reads: int = 1 << 28) -> float:
    """Random 4-byte reads per second of a library gather (torch.index_select
    with int32 indices) from a table of `table_words` words (32 MiB: the size
    of the round kernel's removal-tag array at 2^26 vertices, held in L2),
    indices streamed from memory: the access pattern of the round kernel's
    adjacency passes, one random neighbour read per streamed column id."""
    g = torch.Generator(device=device)
    g.manual_seed(7)
    table = torch.randint(0, 1 << 30, (table_words,), dtype=torch.int32, device=device, generator=g)
    idx = torch.randint(0, table_words, (reads,), dtype=torch.int32, device=device, generator=g)
    out = torch.empty(reads, dtype=torch.int32, device=device)
    for _ in range(3):
        torch.index_select(table, 0, idx, out=out)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    s.record()
    for _ in range(reps):
        torch.index_select(table, 0, idx, out=out)
    e.record()
    torch.cuda.synchronize()
    return reads * reps / (s.elapsed_time(e) / 1e3)


def rounds_algorithmic_bytes(edges_scanned: int, n: int) -> int:
    """Bytes the round kernel must move for one clustering: every scanned
    adjacency entry reads its 4-byte column id and the neighbour's 4-byte state
    word; every vertex costs its two row offsets (16), its own state read and
    write (8) and its alive-list entry (8)."""
    return 8 * edges_scanned + 32 * n


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"host_cores": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def oracle_parity(g, checks, eps):
    """The oracle on the full workload for the last timed step's permutations:
    C4 against serial KwikCluster (Alg. 1; C4 returns exactly its clustering),
    ClusterWild! against the oracle's literal rounds (Alg. 2).  checks: algo ->
    (seed, labels, rounds, D) of the GPU.  Each check runs serially on its own
    host core; the two run side by side."""
    import concurrent.futures

    import numpy as np

    import oracle
    oracle.build()

    def one(a):
        seed, lab, r, d = checks[a]
        t0 = time.perf_counter()
        order = oracle.permutation(g.n, seed)
        if a == "c4":
            olab = oracle.kwik(g.off, g.col, order)
            orr = None
        else:
            olab, orr, _, _ = oracle.rounds(g.off, g.col, order, 2, eps)
        dt = time.perf_counter() - t0
        od = oracle.disagreements(g.off, g.col, olab)
        ok = bool(np.array_equal(lab, olab)) and od == d and (orr is None or orr == r)
        return a, {"seed": seed, "labels_equal": bool(np.array_equal(lab, olab)), "disagreements_equal": od == d,
                   "rounds_equal": None if orr is None else orr == r, "ok": ok, "oracle_s": dt,
                   "oracle": "KwikCluster (Alg. 1)" if a == "c4" else "literal Alg. 2 rounds"}

    with concurrent.futures.ThreadPoolExecutor(len(checks)) as ex:
        return dict(ex.map(one, list(checks)))


def cpu_sample_run(algos, eps, seed_base=7):
    """One pass of the oracle (permutation + Alg. 2 rounds) per algorithm on
    the R-MAT scale-22 sample; returns (edges, seconds)."""
    import graphgen
    import oracle
    oracle.build()
    g = graphgen.rmat(SAMPLE_SCALE, 16, seed=0)
    t0 = time.perf_counter()
    for i, a in enumerate(algos):
        order = oracle.permutation(g.n, seed_base + i)
        oracle.rounds(g.off, g.col, order, 1 if a == "c4" else 2, eps, 1)
    dt = time.perf_counter() - t0
    return g.m * len(algos), dt


class BatchWorkload:
    """The batched and served workload: Chung-Lu graphs (exponent 2.1), n
    log-uniform in [1e3, 1e6], mean degree uniform in [8, 64], seed = g
    (graphgen.chung_lu_batch_params), generated on the GPU
    (graphgen.chung_lu_device) and adopted by the library as device CSR.
    The graphs are admitted in waves of at most `wave_bytes` of CSR; on one
    GB300 every wave stays resident (about 90 GB for 4,096 graphs)."""

    def __init__(self, cc, torch, count: int, wave_bytes: int = 48 << 30):
        import graphgen
        self.params = graphgen.chung_lu_batch_params(count)
        self.graphs, self.tensors, self.waves = [], [], []
        t0 = time.perf_counter()
        wave, wbytes = 0, 0
        for (n, d, seed) in self.params:
            off, col = graphgen.chung_lu_device(n, d, seed=seed)
            if wbytes + 4 * col.numel() > wave_bytes and wbytes > 0:
                self.waves.append(wave)
                wave, wbytes = 0, 0
            wave += 1
            wbytes += 4 * col.numel() + 8 * off.numel()
            self.tensors.append((off, col))
            self.graphs.append(cc.Graph(off, col))
        self.waves.append(wave)
        torch.cuda.synchronize()
        self.gen_s = time.perf_counter() - t0
        self.sum_n = sum(g.n for g in self.graphs)
        self.sum_m = sum(g.m for g in self.graphs)

    def describe(self):
        return (f"{len(self.graphs)} Chung-Lu graphs (exponent 2.1), n log-uniform in [1e3, 1e6], mean degree "
                f"U[8, 64], seed = index; sum n = {self.sum_n}, sum m = {self.sum_m}; generated on the GPU in "
                f"{self.gen_s:.1f} s, admitted in {len(self.waves)} wave(s) of <= 48 GB of CSR, all resident")

    def host_graph(self, i):
        import graphgen
        off, col = self.tensors[i]
        return graphgen.to_host(off, col)

    def close(self):
        for g in self.graphs:
            g.close()
        self.graphs, self.tensors = [], []


def measure_batch(cc, torch, wl: "BatchWorkload", k_perms: int, eps: float, algos=("cw", "c4")):
    """Jobs/s of the batched engine (every (graph, permutation) job of the
    workload, best-of-k per graph) against one launch per job, per algorithm.
    Also returns the jobs kept for the oracle check of the CPU leg."""
    import numpy as np
    seeds = np.arange(len(wl.graphs), dtype=np.uint64) * 1000
    out = {"workload": wl.describe(), "graphs": len(wl.graphs), "k_perms": k_perms, "eps": eps,
           "sum_n": wl.sum_n, "sum_m": wl.sum_m}
    cc.batch_jobs(wl.graphs[:8], "cw", eps, seeds[:8], 2)           # warm-up
    torch.cuda.synchronize()
    # one launch per job on a stratified sample (graphs spread over the size range)
    order = sorted(range(len(wl.graphs)), key=lambda i: wl.graphs[i].n)
    sample = order[:: max(1, len(order) // 48)]
    check = {}
    for a in algos:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D, R = cc.batch_jobs(wl.graphs, a, eps, seeds, k_perms)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        jobs = len(wl.graphs) * k_perms
        t0 = time.perf_counter()
        for i in sample:
            _, r, d = wl.graphs[i].cluster(a, eps, int(seeds[i]) + 1, want_labels=False)
            assert (r, d) == (R[i, 1], D[i, 1])
        t_single = (time.perf_counter() - t0) / len(sample)
        # one-launch-per-job time of the whole workload, from the sample's
        # per-size rate (edges per second of the sampled jobs)
        sample_m = sum(wl.graphs[i].m for i in sample)
        t_single_all = t_single * len(sample) / sample_m * wl.sum_m * k_perms
        out[a] = {"jobs": jobs, "ms": t_batch * 1e3, "jobs_per_s": jobs / t_batch,
                  "edges_per_s": wl.sum_m * k_perms / t_batch,
                  "one_launch_per_job_jobs_per_s": jobs / t_single_all,
                  "speedup_vs_one_launch_per_job": t_single_all / t_batch,
                  "best_of_k_mean_D_gain": float(np.mean(D.min(1) / np.maximum(D[:, 0], 1))),
                  "one_launch_sample": f"{len(sample)} graphs across the size range, permutation 1 of each"}
        pick = [order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]]
        check[a] = [(i, int(seeds[i]) + j, int(R[i, j]), int(D[i, j])) for i in pick for j in (0, k_perms - 1)]
    return out, check


def measure_serving(cc, torch, wl: "BatchWorkload", seconds: float, rate: float = 2000.0, eps: float = 0.5):
    """Poisson arrivals at `rate` jobs/s through the serving loop, each request
    a random graph of the workload, ClusterWild! or C4 with equal odds:
    latency percentiles, throughput and how many jobs ran at once on the
    device, against serving each request with its own launch as it arrives."""
    import numpy as np
    graphs = wl.graphs
    rng = np.random.default_rng(2000)
    nreq = max(1, int(rate * seconds))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    which = rng.integers(0, len(graphs), nreq)
    algo = np.where(rng.random(nreq) < 0.5, "cw", "c4")
    with cc.Server(mem_budget=48 << 30, max_batch=512) as srv:
        srv.wait(srv.submit(graphs[0], "cw", eps, 1))            # warm-up
        t0 = time.perf_counter()
        tickets = []
        for q in range(nreq):
            while time.perf_counter() - t0 < arrivals[q]:
                pass
            tickets.append(srv.submit(graphs[int(which[q])], str(algo[q]), eps, 77 + q))
        res = [srv.wait(t) for t in tickets]
        t_total = time.perf_counter() - t0
        times = [srv.device_times(t) for t in tickets]
    lat = np.array([r[2] for r in res])
    # jobs running at once on the device (from the device clock stamps)
    ev = sorted([(a, 1) for a, b in times if a > 0] + [(b, -1) for a, b in times if a > 0])
    cur = peak = 0
    for _, s in ev:
        cur += s
        peak = max(peak, cur)
    # one launch per request, served in arrival order
    t0 = time.perf_counter()
    lat1 = []
    for q in range(min(nreq, 400)):
        while time.perf_counter() - t0 < arrivals[q]:
            pass
        graphs[int(which[q])].cluster(str(algo[q]), eps, 77 + q, want_labels=False)
        lat1.append((time.perf_counter() - t0 - arrivals[q]) * 1e3)
    lat1 = np.array(lat1)
    small = np.array([graphs[int(i)].n <= 1 << 16 for i in which])
    return {"workload": wl.describe(), "rate_jobs_per_s": rate, "requests": nreq,
            "throughput_jobs_per_s": nreq / t_total,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_ms_small_graphs": float(np.percentile(lat[small], 50)) if small.any() else None,
            "p50_ms_large_graphs": float(np.percentile(lat[~small], 50)) if (~small).any() else None,
            "peak_jobs_in_flight_on_device": peak,
            "one_launch_per_job": {"requests": int(lat1.size), "p50_ms": float(np.percentile(lat1, 50)),
                                   "p99_ms": float(np.percentile(lat1, 99))},
            "algos": "cw and c4, equal odds", "eps": eps}


def batch_oracle_check(wl: "BatchWorkload", check, eps):
    """Sampled batch jobs (smallest, two middle and the largest graph; first
    and last permutation) against the oracle: rounds and disagreements."""
    import oracle
    oracle.build()
    out = []
    for a, items in check.items():
        for i, seed, r, d in items:
            g = wl.host_graph(i)
            order = oracle.permutation(g.n, seed)
            lab, orr, _, _ = oracle.rounds(g.off, g.col, order, 1 if a == "c4" else 2, eps)
            od = oracle.disagreements(g.off, g.col, lab)
            out.append({"algo": a, "graph": i, "n": g.n, "seed": seed, "ok": (orr, od) == (r, d)})
    return {"jobs_checked": len(out), "all_equal": all(x["ok"] for x in out), "jobs": out}


def measure_e2e(cc, torch, g, algos, eps, steps, rank):
    """End to end through the C ABI with host buffers.  Every step uploads the
    graph from pinned host memory (cc_graph_create: copy and validation),
    runs one clustering per algorithm with labels returned to pinned host
    memory, and destroys the graph.  Timed two ways, after one untimed step
    (the library's pool grows to the graph's size once):
    * pipelined (the value): the next step's graph is created by a second
      host thread on its own stream while this step's clusterings run, the
      way a caller processing a stream of graphs would overlap them; the
      first step's upload is inside the timed region and not overlapped;
    * serial: create, cluster, destroy one step after the other.
    Wall clock around device-wide synchronisation (several streams)."""
    import concurrent.futures
    off_h = torch.from_numpy(g.off).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    lab_h = {a: torch.empty(max(g.n, 1), dtype=torch.int32).pin_memory() for a in algos}
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    dev = torch.cuda.current_device()

    def create(i):
        torch.cuda.set_device(dev)                        # the device is per host thread
        return cc.Graph(off_h.numpy(), col_h.numpy(), stream=streams[i % 2].cuda_stream)

    def cluster_all(gh, step):
        for a, seed in zip(algos, step_seeds(rank, step, len(algos))):
            gh.cluster(a, eps, seed, labels_out=lab_h[a].numpy())

    with create(0) as gh:                                  # untimed: pool growth
        cluster_all(gh, 9_999)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        with create(s) as gh:
            cluster_all(gh, 10_000 + s)
    torch.cuda.synchronize()
    serial_ms = (time.perf_counter() - t0) * 1e3 / steps
    with concurrent.futures.ThreadPoolExecutor(1) as ex:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt = ex.submit(create, 0)
        for s in range(steps):
            gh = nxt.result()
            if s + 1 < steps:
                nxt = ex.submit(create, s + 1)
            cluster_all(gh, 20_000 + s)
            gh.close()
        torch.cuda.synchronize()
        pipe_ms = (time.perf_counter() - t0) * 1e3 / steps
    m = g.m
    return {"value": m * len(algos) / (pipe_ms / 1e3), "unit": "edges/s",
            "h2d_bytes_per_step": 8 * (g.n + 1) + 4 * g.nnz,
            "d2h_bytes_per_step": (4 * g.n + 16) * len(algos),
            "ms_per_step": pipe_ms, "steps": steps,
            "serial": {"value": m * len(algos) / (serial_ms / 1e3), "ms_per_step": serial_ms},
            "what": "per step: cc_graph_create from pinned host CSR (copy + validation), one C4 and one "
                    "ClusterWild! cc_cluster with labels to pinned host memory, cc_graph_destroy; the next "
                    "step's upload overlapped with this step's clusterings by a second host thread "
                    "(serial: no overlap); after one untimed step; measured before the device-resident steps"}


def _time_clusterings(graph, algo, eps, seeds, labels):
    """Device time (permutation + rounds + labels, CUDA events) of one
    clustering per seed after one warm-up; returns the means and the last
    run's statistics."""
    graph.cluster(algo, eps, 99, labels_out=labels)
    ms, rk, rs, ds, st = [], [], [], [], None
    for s in seeds:
        _, r, d, st = graph.cluster(algo, eps, s, labels_out=labels, stats_cap=100_000)
        pm, rm, lm = graph.last_timings()
        ms.append(pm + rm + lm)
        rk.append(rm)
        rs.append(r)
        ds.append(d)
    return statistics.mean(ms), statistics.mean(rk), rs, ds, st


def per_round_bandwidth(st, peak):
    """Algorithmic GB/s of every round of the round kernel (8 B per scanned
    adjacency entry, 32 B per vertex removed in the round, over the round's
    device time): median, 10th and 90th percentiles, and the byte-weighted
    mean (total bytes over total time)."""
    import numpy as np
    b = 8.0 * st["edges"] + 32.0 * st["removed"]
    t = np.maximum(st["ns"], 1) / 1e9
    gbs = b / t / 1e9
    return {"rounds": int(b.size), "median_gbs": float(np.median(gbs)), "p10_gbs": float(np.percentile(gbs, 10)),
            "p90_gbs": float(np.percentile(gbs, 90)), "weighted_gbs": float(b.sum() / t.sum() / 1e9),
            "weighted_frac": float(b.sum() / t.sum() / 1e9 / peak)}


def measure_configs(cc, torch, graph26, labels26, peak):
    """The other workload configurations, each timed on its own (not part of
    a step): ClusterWild! at eps 0.1 and 0.9 on R-MAT scale 26; R-MAT scale 24
    with per-round bandwidth; the planted-partition graph at three eps over
    ten orders; the 10^4-vertex Erdos-Renyi graph (L2-resident, so latency per
    round is its measure) over ten orders."""
    import statistics
    import graphgen
    out = {}
    g = graphgen.workload("er10k")
    with cc.Graph(g.off, g.col) as gr:
        gr.set_timing(True)
        lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for a in ("cw", "c4"):
            ms, rk, rs, ds, st = _time_clusterings(gr, a, 0.5, tuple(range(10)), lab)
            out[f"er10k_{a}_eps0.5"] = {"ms_per_clustering": ms, "rounds_kernel_ms": rk, "rounds": rs,
                                        "us_per_round": rk * 1e3 / statistics.mean(rs), "disagreements": ds,
                                        "edges_per_s": gr.m / (ms / 1e3)}
        del lab
    del g
    for eps in (0.1, 0.9):
        ms, rk, rs, ds, st = _time_clusterings(graph26, "cw", eps, (5001, 5002), labels26)
        out[f"rmat26_cw_eps{eps}"] = {"ms_per_clustering": ms, "rounds_kernel_ms": rk, "rounds": rs,
                                      "disagreements": ds, "edges_per_s": graph26.m / (ms / 1e3)}
    g = graphgen.workload("rmat24")
    with cc.Graph(g.off, g.col) as gr:
        gr.set_timing(True)
        lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for a in ("cw", "c4"):
            ms, rk, rs, ds, st = _time_clusterings(gr, a, 0.5, (6001, 6002), lab)
            out[f"rmat24_{a}_eps0.5"] = {"ms_per_clustering": ms, "rounds_kernel_ms": rk, "rounds": rs,
                                         "disagreements": ds, "edges_per_s": gr.m / (ms / 1e3),
                                         "per_round": per_round_bandwidth(st, peak)}
        del lab
    del g
    g = graphgen.workload("planted1m")
    with cc.Graph(g.off, g.col) as gr:
        gr.set_timing(True)
        lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
        planted = gr.disagreements(g.aux)
        for a in ("cw", "c4"):
            for eps in (0.1, 0.5, 0.9):
                ms, rk, rs, ds, st = _time_clusterings(gr, a, eps, tuple(range(7001, 7011)), lab)
                out[f"planted1m_{a}_eps{eps}"] = {"ms_per_clustering": ms, "rounds": rs, "disagreements": ds,
                                                   "planted_labels_disagreements": planted,
                                                   "edges_per_s": gr.m / (ms / 1e3)}
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if world > 1 and rank != 0:
        return
    algos = args.algos.split(",")
    for _ in range(args.warmup):
        cpu_sample_run(algos, args.eps)
    edges = 0
    secs = 0.0
    for s in range(args.steps):
        e, dt = cpu_sample_run(algos, args.eps, seed_base=100 + s)
        edges += e
        secs += dt
    value = edges / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"rmat{SAMPLE_SCALE} (sample of the rmat26 workload's generator)",
                   "algos": algos, "eps": args.eps},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": f"serial C oracle: permutation + Alg. 2 rounds, R-MAT scale {SAMPLE_SCALE}"},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1507_05086_gb300 as cc

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    algos = args.algos.split(",")
    g = load_graph(args.workload)
    m = g.m
    # end to end through the public API with host buffers, measured first
    # (run after the device-resident steps and the random-read ceiling below,
    # the same steps were measured 30-40 % slower; a second resident graph
    # alone does not slow them, and the cause was not identified)
    e2e = None
    if args.e2e_steps > 0:
        e2e = measure_e2e(cc, torch, g, algos, args.eps, args.e2e_steps, rank)

    graph = cc.Graph(g.off, g.col)
    graph.set_timing(True)
    # schedule settings for this graph class on this device: from the
    # autotuner's cache, else tuned now (no setting changes a result)
    tuning = {}
    if args.tune:
        from paper_1507_05086_gb300 import autotune
        tuning["rounds"] = autotune.tune_rounds(graph, tuple(algos), args.eps, budget_s=30.0)
    # one label buffer per algorithm, so that the last timed step's labels of
    # both can be checked against the oracle after the timed region
    labels_of = {a: torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda") for a in algos}
    labels = labels_of[algos[0]]

    for s in range(args.warmup):
        for a, seed in zip(algos, step_seeds(rank, -1 - s, len(algos))):
            graph.cluster(a, args.eps, seed, labels_out=labels_of[a])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    per = {a: {"ms": [], "rounds_ms": [], "perm_ms": [], "rounds": [], "D": [], "edges": [], "phases": []}
           for a in algos}
    with ClockSampler(local_rank) as clocks:
        barrier()
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record()
        for s in range(args.steps):
            for a, seed in zip(algos, step_seeds(rank, s, len(algos))):
                _, r, d, st = graph.cluster(a, args.eps, seed, labels_out=labels_of[a], stats_cap=100_000)
                pm, rm, lm = graph.last_timings()
                per[a]["ms"].append(pm + rm + lm)
                per[a]["perm_ms"].append(pm)
                per[a]["rounds_ms"].append(rm)
                per[a]["rounds"].append(r)
                per[a]["D"].append(d)
                per[a]["edges"].append(int(st["edges"].sum()))
                per[a]["phases"].append(graph.last_phase_times())
        end.record()
        torch.cuda.synchronize()
        barrier()
    elapsed = start.elapsed_time(end)
    # the last timed step's outputs, for the oracle check of the CPU leg
    last_step = {a: (seed, labels_of[a][:g.n].cpu().numpy(), per[a]["rounds"][-1], per[a]["D"][-1])
                 for a, seed in zip(algos, step_seeds(rank, args.steps - 1, len(algos)))}
    clusterings = args.steps * len(algos)
    edges_done = m * clusterings
    value, tmax = reduce_across_ranks(elapsed, edges_done, world, torch.device("cuda", local_rank))

    # roofline of the dominant kernel (the persistent round kernel)
    peak, peak_kind = measured_hbm_peak()
    rk_ms = [x for a in algos for x in per[a]["rounds_ms"]]
    rk_bytes = [rounds_algorithmic_bytes(e, g.n) for a in algos for e in per[a]["edges"]]
    achieved = (sum(rk_bytes) / 1e9) / (sum(rk_ms) / 1e3)
    ratio = ROUNDS_TRAFFIC_PER_BYTE.get(rounds_sources_digest())
    traffic = ratio * sum(rk_bytes) / len(rk_bytes) if ratio is not None else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k_rounds", "peak_kind": peak_kind,
                "bytes_per_launch": sum(rk_bytes) / len(rk_bytes), "ms_per_launch": sum(rk_ms) / len(rk_ms),
                # the same figure against HBM3e's nominal 8.0 TB/s
                "frac_of_nominal_8000_gbs": achieved / 8000.0}
    # the same kernel against the random-read rate a library gather reaches
    # on this GPU: every scanned adjacency entry costs one random 4-byte read
    ceiling = measure_gather_ceiling(torch, torch.device("cuda", local_rank))
    rk_edges = sum(e for a in algos for e in per[a]["edges"])
    random_access = {"achieved": rk_edges / (sum(rk_ms) / 1e3), "ceiling": ceiling, "unit": "random reads/s",
                     "frac": rk_edges / (sum(rk_ms) / 1e3) / ceiling, "kernel": "k_rounds",
                     "ceiling_kind": "measured: torch.index_select, int32 indices, 2^28 reads from a 32 MiB table"}

    # the practical schedule of Sec. 5 (Delta-hat halving, binomial batches) on
    # the same graph, one clustering each: a comparison, not part of a step
    sec5 = None
    if rank == 0 and args.sec5:
        sec5 = {}
        for a in algos:
            graph.cluster(a + "-est", args.eps, 4242, labels_out=labels)
            pm, rm, lm = graph.last_timings()
            _, r, d = graph.cluster(a + "-est", args.eps, 4243, labels_out=labels)
            pm, rm, lm = graph.last_timings()
            sec5[a + "-est"] = {"ms_per_clustering": pm + rm + lm, "rounds_kernel_ms": rm, "rounds": r,
                                "disagreements": d, "edges_per_s": m / ((pm + rm + lm) / 1e3)}

    # C4 without rounds (Alg. 3) on the same graph: same labels as C4 (and
    # KwikCluster), one clustering after one warm-up; a comparison, not part
    # of a step
    async_c4 = None
    if rank == 0 and args.async_c4 and "c4" in algos:
        graph.cluster("c4-async", args.eps, 4244, labels_out=labels)
        _, _, d, st = graph.cluster("c4-async", args.eps, 4245, labels_out=labels, stats_cap=1)
        pm, km, om = graph.last_timings()
        async_c4 = {"ms_per_clustering": pm + km + om, "permutation_ms": pm, "decide_push_ms": km,
                    "labels_objective_ms": om, "disagreements": d, "blocked": int(st["blocked"][0]),
                    "centers": int(st["centers"][0]), "edges_read": int(st["edges"][0]),
                    "edges_per_s": m / ((pm + km + om) / 1e3),
                    "what": "permutation; k_async_init, k_async_decide (one cooperative launch), "
                            "k_async_push_long, k_async_labels; objective from the labels"}

    configs = None
    if rank == 0 and args.configs:
        configs = measure_configs(cc, torch, graph, labels, peak)

    batch = serve = batch_check = wl = None
    if rank == 0 and (args.batch_graphs > 0 or args.serve_seconds > 0):
        del labels_of, labels
        graph.close()                         # room for the batch workload
        wl = BatchWorkload(cc, torch, max(args.batch_graphs, 64))
        if args.tune:
            from paper_1507_05086_gb300 import autotune
            # size classes and team size, timed on every eighth graph of the batch
            # with the batch's own 8 permutations per graph (with 2 the sample's
            # time is set by its largest graphs' jobs, not by throughput: team
            # sizes 4 and 8 timed within 2 % there, 15 % apart on the batch)
            tuning["batch"] = autotune.tune_batch(wl.graphs[::8], "cw", args.eps, k_perms=8, budget_s=60.0)
        if args.batch_graphs > 0:
            batch, batch_check = measure_batch(cc, torch, wl, 8, args.eps)
        if args.serve_seconds > 0:
            # the batch tuning optimises throughput; the server keeps the
            # default size classes (a latency objective)
            cc.set_batch_tuning(cc.default_tuning())
            serve = measure_serving(cc, torch, wl, args.serve_seconds)

    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        e, dt = cpu_sample_run(algos, args.eps)
        cpu = {"value": e / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": f"serial C oracle (permutation + Alg. 2 rounds, C4 and ClusterWild!, eps={args.eps}) "
                         f"on R-MAT scale {SAMPLE_SCALE} from the same generator, {e // len(algos)} edges, "
                         f"{dt:.1f} s",
               **host_cpu()}
        # the timed step's output on the full workload against the oracle
        if args.parity:
            parity = oracle_parity(g, last_step, args.eps)
            if batch_check:
                parity["batch"] = batch_oracle_check(wl, batch_check, args.eps)
    if wl is not None:
        wl.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: R-MAT scale 26, ef 16, (0.57,0.19,0.19,0.05), seed 0"
                       if args.workload == "rmat26" else args.workload,
                       "n": g.n, "m": m, "nnz": g.nnz, "max_degree": graph.max_degree, "algos": algos,
                       "eps": args.eps, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (CSR and state far above 129 MB); no flush"},
            "per_algo": {a: {"ms_per_clustering": statistics.mean(per[a]["ms"]),
                             "rounds_kernel_ms": statistics.mean(per[a]["rounds_ms"]),
                             "permutation_ms": statistics.mean(per[a]["perm_ms"]),
                             "rounds": per[a]["rounds"][0], "disagreements": per[a]["D"],
                             "edges_scanned": per[a]["edges"][0],
                             "phase_ms": {k: statistics.mean(p[k] for p in per[a]["phases"])
                                          for k in per[a]["phases"][0]},
                             "edges_per_s": m / (statistics.mean(per[a]["ms"]) / 1e3)} for a in algos},
            "clocks": clocks.summary(),
            "e2e": e2e,
            "gpu_launches": KERNELS_PER_CLUSTERING * clusterings,
            "roofline": roofline,
            "random_access": random_access,
            "cpu_baseline": cpu,
            "parity": parity,
            "tuning": tuning,
            "configs": configs,
            "batch": batch,
            "serve": serve,
            "sec5_schedule": sec5,
            "async_c4": async_c4,
        }
        print(json.dumps(line), flush=True)
    graph.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
