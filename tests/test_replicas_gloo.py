"""The multi-process path of bench.py (independent replicas, one per GPU):
the whole-job time is the slowest rank's and the items are summed.  Runs as
two gloo ranks on the CPU."""
from __future__ import annotations

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


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, items = bench.replica_aggregate(10.0 + 5.0 * rank, 1000 * (rank + 1), dist, "cpu")
    q.put((rank, ms, items))
    dist.destroy_process_group()


def test_replica_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 15.0, 3000), (1, 15.0, 3000)]


def test_replica_aggregate_single():
    import bench
    assert bench.replica_aggregate(3.5, 7) == (3.5, 7)
