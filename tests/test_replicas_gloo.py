"""The multi-GPU form is replicas only (every rank runs its own copy of the
workload); bench.py's one collective is the max of the step time over ranks.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], world, device="cpu")
    out[rank] = (ms, bench.job_value(1000.0, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_time_and_job_value_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    times = [40.0, 50.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == pytest.approx(50.0)
        assert value == pytest.approx(world * 1000.0 / 0.050)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_value(10.0, 1, 1000.0) == pytest.approx(10.0)
