"""The multi-GPU bench path is replicas only (one independent solve per GPU,
no data-path collective): its host logic -- the slowest rank's time as the
job's time and the job's rate over all ranks' work -- on two gloo ranks on
the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 25.0 * rank            # rank 1 is the slower one
        job_ms = bench.max_over_ranks(my_ms, dist, "cpu")
        rate = bench.whole_job_rate(world, 3.6e6 * 3 * 10, job_ms)
        dist.barrier()
        out[rank] = (job_ms, rate)
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_all_ranks_work():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        job_ms, rate = out[r]
        assert job_ms == 125.0
        assert rate == pytest.approx(world * 3.6e6 * 3 * 10 / 0.125)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.whole_job_rate(1, 1000, 500.0) == 2000.0
