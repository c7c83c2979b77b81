"""The N > 1 host logic of bench.py (replicas, one per rank) on two gloo
ranks on the CPU: the slowest rank's time is what every rank sees, and the
whole-job value counts every rank's units."""

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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        # rank r took 10 + 5 r ms for 3 steps, and 2 + r s end to end
        ms, e2e = bench.max_over_ranks([10.0 + 5 * rank, 2.0 + rank], "cpu")
        value = bench.replica_throughput(world, 3, ms * 1e-3)
        out[rank] = (ms, e2e, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_bench():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        ms, e2e, value = out[r]
        assert ms == 15.0 and e2e == 3.0            # the slowest rank's times
        assert value == pytest.approx(2 * 3 / 15e-3)  # every rank's steps over that time


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([4.0, 7.5], "cpu") == [4.0, 7.5]
    assert bench.replica_throughput(1, 5, 2.0) == 2.5
