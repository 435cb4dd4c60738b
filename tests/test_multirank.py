"""Host logic of the multi-process bench (replicas, one per rank): two gloo
ranks on CPU.  The method has no exchange step, so ranks share nothing but
the timing reduction: the slowest rank's time, and each rank's own seeded
object."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2208_12964_gb300 import synth

        t = bench.max_over_ranks([10.0 + rank, 3.0 * (world - rank)])
        spec = synth.parallel_workload(8, 6, 17)
        spec["seed"] = bench.replica_seed(spec["seed"], rank)
        p = synth.projections(spec)
        out.put((rank, t, float(p.sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_objects():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1] == [11.0, 6.0]  # max over ranks, element-wise
    assert res[0][2] != res[1][2]  # replicas reconstruct different seeded objects


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.replica_seed(7, 0) == 7
