"""Multi-rank logic of bench.py on CPU (gloo, world size 2): independent
replicas get distinct permutations, and the reported throughput is the sum
of all ranks' work over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [100.0, 250.0][rank]
    edges = [1_000_000, 3_000_000][rank]
    value, tmax = bench.reduce_across_ranks(elapsed, edges, world, torch.device("cpu"))
    seeds = [s for step in range(3) for s in bench.step_seeds(rank, step, 2)]
    q.put((rank, value, tmax, seeds))
    dist.destroy_process_group()


def test_two_rank_aggregation_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, value, tmax, _ in out:
        assert tmax == 250.0
        assert value == pytest.approx(4_000_000 / 0.25)
    s0, s1 = set(out[0][3]), set(out[1][3])
    assert len(s0) == 6 and len(s1) == 6 and not (s0 & s1)


def test_single_rank_aggregate():
    import bench
    v, t = bench.reduce_across_ranks(200.0, 1_000_000, 1, None)
    assert t == 200.0 and v == pytest.approx(5e6)
