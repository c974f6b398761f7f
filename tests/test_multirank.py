"""The multi-rank path of the benchmark on the CPU (gloo, two processes):
every rank runs its own scene, the job's time is the slowest rank's, and the
whole-job rate counts every rank's frames.  No data-path collective exists."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import argparse
        import bench
        args = argparse.Namespace(scene="tiny", seed=None)
        sc = bench.scene_for_rank(args, rank)
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_ms, torch.device("cpu"), world)
        out[rank] = (slowest, bench.job_rate(20, world, slowest), float(sc.frames[5].Z.sum()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_by_the_slowest_and_count_all_frames():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # 20 frames on each of two ranks in 150 ms
    assert res[0][1] == pytest.approx(40 / 0.150)
    # each rank runs its own scene
    assert res[0][2] != res[1][2]


def test_one_rank_is_the_plain_value():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu"), 1) == 3.5
    assert bench.job_rate(100, 1, 50.0) == pytest.approx(2000.0)
