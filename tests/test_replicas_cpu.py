"""Multi-GPU runs are replicas only: every rank solves its own system and the
job's throughput is the points of all ranks over the slowest rank's time.
The host-side reduction is exercised here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r is slower by r milliseconds in solve and 2r in eval
        t = bench.max_over_ranks([50.0 + rank, 40.0 + 2 * rank], world, "cpu")
        out[rank] = (t, bench.replica_throughput(1_000_000, world, t[0]))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == [51.0, 42.0]
        assert v == pytest.approx(2 * 1_000_000 / 0.051 / 1e6)


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks([3.0, 4.5], 1, "cpu") == [3.0, 4.5]
    assert bench.replica_throughput(2_000_000, 1, 50.0) == pytest.approx(40.0)
