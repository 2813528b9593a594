"""The bench's N > 1 path on CPU ranks (gloo, world size 2): every rank runs
its own replica (distinct Philox streams), the job value is all ranks' flips
over the slowest rank's time, and no collective touches the lattice data."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slower one
        value, t_max = bench.job_value(local_ms, 1e9, dist)
        # the rank's own lattice: replica id = rank, first two sweeps on L = 16
        s = oracle.init(16, 1, bench.replica_of_rank(rank))
        oracle.sweep(s, 0.44, 1, 2, replica=bench.replica_of_rank(rank))
        out[rank] = (value, t_max, s.tobytes())
    finally:
        dist.destroy_process_group()


def test_two_rank_job_value_and_distinct_replicas():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29500 + (os.getpid() % 2000)
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    (v0, t0, s0), (v1, t1, s1) = res[0], res[1]
    assert t0 == t1 == 150.0
    assert v0 == v1 == pytest.approx(2e9 / (150.0 * 1e6))
    assert s0 != s1  # independent replicas


def test_single_rank_job_value():
    v, t = bench.job_value(200.0, 4e9)
    assert t == 200.0 and v == pytest.approx(4e9 / 2e8)
