"""The multi-rank plumbing of bench.py on CPU (gloo, world size 2): the job's
time is the slowest rank's (max over ranks) and the reported throughput is
the whole job's (every rank runs its own replica: weak scaling).  The GPU
path uses the same helpers over NCCL."""
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


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = 10.0 + 7.5 * rank                       # this rank's total time (ms)
    total = bench.max_over_ranks(mine, dist, "cpu")
    dist.barrier()
    out[rank] = total
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    import bench
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert dict(out) == {0: 17.5, 1: 17.5}
    # 2 replicas of 1000 DOF, 4 steps each, in the slowest rank's 17.5 ms
    assert bench.job_throughput(world, 1000, 4, 17.5) == pytest.approx(2 * 1000 * 4 / 17.5e-3 / 1e9)
