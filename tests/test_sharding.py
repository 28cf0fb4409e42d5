"""Multi-rank path on CPU: world_size 2 gloo ranks shard spectra disjointly
and agree on the max-over-ranks time (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2604_03271_b300.sharding import max_over_ranks, shard_seeds, sum_over_ranks


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    seeds = [shard_seeds(step, world, rank, 3) for step in range(4)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    t = max_over_ranks(1.5 + rank, dist)
    n = sum_over_ranks(len(seeds) * 3, dist)
    dist.barrier()
    if rank == 0:
        q.put((gathered, t, n))
    dist.destroy_process_group()


def test_two_rank_sharding_is_disjoint_and_max_time_agrees():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, t, n = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == pytest.approx(2.5)
    assert n == 24
    for step in range(4):
        a, b = gathered[0][step], gathered[1][step]
        assert not set(a) & set(b)
        assert sorted(a + b) == list(range(1 + step * 6, 1 + (step + 1) * 6))


def test_single_process_defaults():
    assert shard_seeds(0, 1, 0, 2) == [1, 2]
    assert shard_seeds(3, 1, 0, 2) == [7, 8]
    assert max_over_ranks(4.0) == 4.0
