"""Host logic of multi-GPU runs, on CPU with two `gloo` ranks: the EMD solves of
different shots are independent, so ranks share shots and reduce only the step time."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_shard_shots_is_a_balanced_partition():
    sizes = [((s * 7919) % 97 + 1) * 1000 for s in range(48)]
    for world in (1, 2, 3, 4, 8):
        parts = bench.shard_shots(sizes, world)
        assert len(parts) == world
        flat = sorted(s for p in parts for s in p)
        assert flat == list(range(48))
        loads = [sum(sizes[s] for s in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)  # greedy bound


def test_max_over_ranks_without_a_group():
    assert bench.max_over_ranks(3.5) == 3.5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [10, 40, 20, 30, 50]
        mine = bench.shard_shots(sizes, world)[rank]
        t = bench.max_over_ranks(1.0 + rank)
        out[rank] = (mine, t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_shots_and_agree_on_the_max():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    shards = [res[r][0] for r in range(world)]
    assert sorted(shards[0] + shards[1]) == [0, 1, 2, 3, 4]
    assert not set(shards[0]) & set(shards[1])
    assert res[0][1] == res[1][1] == 2.0  # every rank sees the slowest rank's time
