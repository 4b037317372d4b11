"""The multi-rank logic of bench.py on CPU with two gloo ranks: each rank
reports its own timings, the job time is the slowest rank's, and the value
counts the work of every rank (Q replicas, weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks([1.0 + rank, 10.0 - rank], "cpu", world)
    v = bench.weak_scaling_value(world, 2.0e12, t[0])
    out.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == [2.0, 10.0]                 # maxima over the ranks
        assert abs(v - 2 * 2.0e12 / 2e-3 / 1e12) < 1e-9   # both ranks' flops / slowest time


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], "cpu", 1) == [3.0, 4.0]
    assert bench.weak_scaling_value(1, 1e12, 1000.0) == 1.0     # 1e12 flops in 1 s
