"""Multi-process bench logic on CPU (gloo, world size 2).

The sort does not shard across GPUs ("replicas only"): under torchrun every rank
sorts its own arrays and bench.py reports all ranks' keys over the slowest rank's
time.  These tests run that aggregation with two gloo processes on the host.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 * (rank + 1)                      # rank 1 is the slowest
    worst = bench.max_over_ranks(ms)
    value = bench.replica_throughput(1000, worst, dist.get_world_size())
    q.put((rank, worst, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_with_two_gloo_ranks():
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
    assert [r[1] for r in res] == [20.0, 20.0]            # both see the slowest time
    assert all(abs(r[2] - 2 * 1000 / 0.020) < 1e-6 for r in res)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(100, 1000.0, 1) == 100.0
