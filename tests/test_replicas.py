"""The multi-GPU path of bench.py is replicas only (the method has no exchange step): each
rank times its own replica, the job's time is the slowest rank's, and batched instances are
split across ranks without any collective on the data. The host logic runs here as two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 1.5 if rank == 0 else 2.25  # seconds each replica took
        dist.barrier()
        slowest = bench.slowest_rank_seconds(local, dist, "cpu")
        value = bench.job_throughput(30, world, slowest)
        mine = bench.shard(256, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = (slowest, value, gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_shard():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        slowest, value, gathered = res[rank]
        assert slowest == 2.25                       # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 30 / 2.25)  # units of all ranks over that time
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(256))              # every instance exactly once
        assert abs(len(gathered[0]) - len(gathered[1])) <= 1


@pytest.mark.parametrize("count,world", [(256, 1), (256, 3), (5, 8), (0, 2)])
def test_shard_partitions(count, world):
    parts = [bench.shard(count, r, world) for r in range(world)]
    assert sorted(i for p in parts for i in p) == list(range(count))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1


def test_single_rank_needs_no_process_group():
    assert bench.slowest_rank_seconds(3.0) == 3.0
    assert bench.job_throughput(30, 1, 3.0) == 10.0
