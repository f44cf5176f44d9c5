"""The multi-GPU form is replicas only (the ILUT triangular solves do not shard):
each rank solves its own problems and only the timing is combined.  This runs
that combination with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.reduce_step_time(1.0 + rank, dist, "cpu")   # rank 1 is the slow one
        q.put((rank, t, bench.job_value(2.0e6, world, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 2.0                      # both ranks see the slowest rank's time
        assert v == pytest.approx(2.0)       # 2e6 units x 2 ranks / 2 s = 2 M units/s
