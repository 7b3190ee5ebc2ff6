"""The multi-process path of bench.py on CPU: two gloo ranks, each timing
its own replica, agree on the slowest rank's time, and the whole-job value
counts the cells of both replicas over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        t = bench.max_over_ranks(mine, world, "cpu")
        out[rank] = (t, bench.whole_job_mlups(1_000_000, 100, t, world))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # 2 replicas x 1e6 cells x 100 steps in 15 ms each step -> 1.0e12 / 1.5 cell updates/s
    assert abs(res[0][1] - 2 * 1e6 * 100 / (15.0e-3) / 1e6) < 1e-6
    assert res[0][1] == res[1][1]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_mlups(10, 2, 4.0, 1) == 10 * 2 / 4e-3 / 1e6
