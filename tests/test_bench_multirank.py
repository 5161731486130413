"""bench.py's multi-rank aggregation on two gloo ranks (CPU): the whole-job value is the units
of all ranks over the slowest rank's time; every rank is an independent replica."""
from __future__ import annotations

import multiprocessing as mp
import os
import socket


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rmax, rsum = bench.make_reducers(dist)
    value, slowest = bench.aggregate(1.0 + rank, 100.0 * (rank + 1), world, rmax, rsum)
    dist.barrier()
    q.put((rank, value, slowest))
    dist.destroy_process_group()


def test_two_rank_aggregation():
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
    for rank, value, slowest in res:
        assert slowest == 2.0  # the max over ranks
        assert value == 150.0  # (100 + 200) units / 2.0 s


def test_single_rank_aggregation():
    import bench
    value, slowest = bench.aggregate(2.0, 10.0, 1)
    assert (value, slowest) == (5.0, 2.0)
