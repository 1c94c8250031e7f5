"""The multi-rank host logic of bench.py on CPU processes (gloo, world size 2).

Queries are independent, so ranks run replicas of the index on their own
query batches (weak scaling) and share only a max-reduce of their step times;
these tests run that reduce, the whole-job rate and the per-rank query seeds
over a real two-process group."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1707_00143_gb300 import datagen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank measured its own times; the job's step time is the slowest rank's
        mine = [1.0 + rank, 10.0 - rank, 3.5]
        got = bench.max_over_ranks(mine, "cpu")
        seed = bench.rank_query_seed(rank, datagen.SEED_QUERY)
        _, q = datagen.workload("tiny", n=10, nq=8, seed_query=seed)
        qs = [torch.zeros(8, 32) for _ in range(world)]
        dist.all_gather(qs, torch.from_numpy(q))
        out[rank] = (got, [x.numpy().copy() for x in qs])
    finally:
        dist.destroy_process_group()


def test_max_reduce_and_query_batches_over_two_ranks():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        got, qs = out[r]
        assert got == [2.0, 10.0, 3.5]  # element-wise max over ranks
        assert not np.array_equal(qs[0], qs[1])  # distinct query batches per rank
    assert np.array_equal(out[0][1][0], out[1][1][0])  # every rank sees the same batches


def test_single_process_values_pass_through_and_job_rate():
    assert bench.max_over_ranks([4.0, 5.0], "cpu") == [4.0, 5.0]
    # 2 ranks x 10,000 queries in 4 ms (the slowest rank) -> 5 M queries/s for the job
    assert bench.job_qps(2, 10000, 4.0) == pytest.approx(5e6)
    assert bench.rank_query_seed(0, 2) == 2 and bench.rank_query_seed(3, 2) == 3002
