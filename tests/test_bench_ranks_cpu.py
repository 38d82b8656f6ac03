"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) time
different amounts, and the whole-job throughput uses the slowest rank."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [2.0, 5.0][rank]
    t, v = bench.aggregate_ranks(torch, dist, seconds, world, 100, "cpu")
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == pytest.approx(5.0)
        assert v == pytest.approx(2 * 100 / 5.0)


def test_single_rank_is_unchanged():
    t, v = bench.aggregate_ranks(torch, None, 4.0, 1, 100, "cpu")
    assert (t, v) == (4.0, 25.0)
