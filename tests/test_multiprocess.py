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


def _shots():
    """Five small shot pairs of uneven sizes (seeded)."""
    import numpy as np
    rng = np.random.default_rng(21)
    shapes = [(2, 5), (4, 10), (3, 7), (3, 10), (5, 10)]
    return [(np.maximum(rng.standard_normal(s), 0), np.maximum(rng.standard_normal(s), 0)) for s in shapes]


def _solve(pair):
    from oracle import emd_oracle as O
    return O.pdhg(pair[0], pair[1], 0.1, 0.2, max_iter=60)["dist"]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shots = _shots()
        mine = bench.shard_shots([o.size for o, _ in shots], world)[rank]
        dists = {s: _solve(shots[s]) for s in mine}  # this rank's share, solved independently
        t = bench.max_over_ranks(1.0 + rank)
        out[rank] = (mine, t, dists)
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
    # the union of the ranks' results is the single-process result, shot by shot
    merged = {**res[0][2], **res[1][2]}
    assert sorted(merged) == [0, 1, 2, 3, 4]
    for s, pair in enumerate(_shots()):
        assert merged[s] == _solve(pair)
