"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1).

Every rank runs an independent replica (no collective on the data path);
the only collective is the max over ranks of the timed interval, and the
whole-job rate counts every rank's solves over that slowest time.
"""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        t = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.whole_job_rate(3, world, t)
        out[rank] = (t, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == 150.0
        assert rate == pytest.approx(3 * world / 0.150)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.whole_job_rate(2, 1, 500.0) == pytest.approx(4.0)
