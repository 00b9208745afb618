"""bench.py's multi-GPU path is replicas only: the ranks share nothing but the
timing collectives (a barrier and a max over ranks), and the job's frame rate
is every rank's frames over the slowest rank's step time.  Checked here with
two gloo ranks on the CPU."""
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
        bench.ranks_barrier(world)
        ms = [1.5, 2.5][rank]  # the second rank is the slower one
        m = bench.max_over_ranks(ms, world, torch.device("cpu"))
        out[rank] = (m, bench.replica_fps(m, world))
        bench.ranks_barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step_and_sum_the_frames():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    m, fps = res[0]
    assert m == 2.5
    assert fps == pytest.approx(2 * 1000.0 / 2.5)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, 1, torch.device("cpu")) == 3.0
    bench.ranks_barrier(1)
    assert bench.replica_fps(2.0, 1) == pytest.approx(500.0)
