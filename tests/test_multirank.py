"""Host logic of the N > 1 bench path on CPU: two gloo ranks.

Queries are independent, so bench.py gives every rank its own block of the
batch (weak scaling, no collective on the data path) and takes the job's
time as the slowest rank's (a MAX all-reduce).  Checked here with
world_size 2 on the gloo backend: the shards are disjoint and cover the
batch, and every rank sees the same maximum.
"""
import os
import socket

import numpy as np
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Qall = np.arange(world * 5 * 3, dtype=np.float32).reshape(world * 5, 3)
        Q = bench.shard_queries(Qall, rank, 5)
        mine = 10.0 + 7.0 * rank                   # rank 1 is the slower one
        worst = bench.max_over_ranks(mine, dist)
        dist.barrier()
        out[rank] = (Q[:, 0].tolist(), worst)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_queries_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    firsts = sorted(v for q, _ in res.values() for v in q)
    assert firsts == [float(3 * i) for i in range(world * 5)]        # disjoint blocks covering the batch
    assert res[0][0] == [0.0, 3.0, 6.0, 9.0, 12.0]
    assert all(w == 17.0 for _, w in res.values())                    # every rank sees the maximum


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(3.25) == 3.25
    Q = np.zeros((8, 2))
    assert bench.shard_queries(Q, 0, 8).shape == (8, 2)
