"""Multi-rank logic of bench.py on CPU: two gloo ranks (replicas), the time is the
maximum over ranks and the whole-job value counts every rank's units."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port,
                            rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, world)
    out[rank] = (ms, bench.whole_job_mlups(world, 1000, 10, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, value = out[r]
        assert ms == pytest.approx(150.0)
        # 2 replicas x 1000 nodes x 10 steps in 0.15 s
        assert value == pytest.approx(2 * 1000 * 10 / 0.150 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_mlups(1, 2048, 100, 1000.0) == pytest.approx(2048 * 100 / 1.0 / 1e6)
