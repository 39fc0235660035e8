"""The replica path of bench.py with two processes (gloo on CPU): the job time is the slowest rank's time and the
units are summed over ranks."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [1.5, 2.25][rank]
    units = [1000.0, 3000.0][rank]
    q.put((rank, bench.aggregate(seconds, units, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_on_gloo():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == (2.25, 4000.0)


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(3.0, 7.0, 1) == (3.0, 7.0)
