"""Job sharding across ranks (one process per GPU).

The sampler's jobs -- one per (spectrum, K) -- are independent, so N GPUs
process disjoint sets of spectra with no collective on the data path; the
only cross-rank operations are a barrier and a max over the ranks' elapsed
times for reporting (weak scaling: each rank keeps the same work per step).
"""
from __future__ import annotations

from typing import List


def shard_seeds(step: int, world: int, rank: int, batch: int, base: int = 1) -> List[int]:
    """Data seeds of the `batch` spectra that `rank` processes at `step`.

    Seeds of all ranks at one step form the contiguous block
    base + step*world*batch ... base + (step+1)*world*batch - 1, rank r taking
    the r-th sub-block, so shards are disjoint and independent of world size
    per rank."""
    first = base + (step * world + rank) * batch
    return list(range(first, first + batch))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
