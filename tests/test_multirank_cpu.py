"""The multi-GPU path of bench.py on CPU ranks (gloo, world size 2): the
work is sharded into disjoint, complete shares with no exchange between
ranks, and the job's figures are the slowest rank's time and the sum of
the ranks' work (max-over-ranks timing)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        items = list(range(10))
        mine = bench.shard(items, r, ws)
        # a rank's local time and work; the job takes the max time and the sum of work
        t_local = 1.0 + r  # rank 1 is the slow one
        work_local = 100.0 * len(mine)
        out[r] = (ws, r, local, mine, bench.job_max(t_local, "cpu"),
                  bench.job_sum(work_local, "cpu"))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(worker, args=(world, free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    shares = [out[r][3] for r in range(world)]
    assert sorted(shares[0] + shares[1]) == list(range(10))  # disjoint and complete
    assert not set(shares[0]) & set(shares[1])
    for r in range(world):
        ws, rank, local, _, t_max, work = out[r]
        assert (ws, rank, local) == (world, r, r)
        assert t_max == 2.0  # the slowest rank's time on every rank
        assert work == 1000.0  # all ranks' work


def test_one_process_job_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_max(3.5, "cpu") == 3.5 and bench.job_sum(2.0, "cpu") == 2.0
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
