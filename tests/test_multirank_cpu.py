"""The multi-GPU path of bench.py on CPU: world size 2 over gloo.

Every rank is an independent replica of the workload (no data-path
collective); the job's time is the slowest rank's (a MAX all-reduce) and its
throughput counts every rank's units.  This checks that host logic with two
gloo processes on 127.0.0.1; no GPU is involved."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1.5 + r seconds for 1000 units
        secs = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        out[rank] = (secs, bench.job_throughput(world, 1000, secs))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    secs, thr = res[0]
    assert secs == pytest.approx(2.5)
    assert thr == pytest.approx(2 * 1000 / 2.5)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_throughput(1, 500, 2.0) == 250.0
