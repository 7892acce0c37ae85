"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): the
job time is the slowest rank's, every rank sees it, and the whole-job rate
counts the work of all replicas.  The data path has no collective (replicas
only), so this is the only cross-rank logic there is."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_info()
        assert (ws, r, local) == (world, rank, rank)
        mine = 100.0 + 50.0 * rank          # rank 1 is the slower one
        job = bench.max_over_ranks(mine, torch.device("cpu"))
        rate = bench.whole_job_rate(1e12, 10, ws, job)
        results[rank] = (job, rate)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        got = dict(results)
    assert got[0][0] == got[1][0] == 150.0     # the slowest rank's time, on every rank
    # 10 steps of 1e12 units on each of 2 replicas in 150 ms
    assert got[0][1] == pytest.approx(2 * 10 * 1e12 / 0.150 / 1e12)


def test_single_rank_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, torch.device("cpu")) == 42.0
    assert bench.whole_job_rate(2e12, 5, 1, 1000.0) == pytest.approx(10.0)
