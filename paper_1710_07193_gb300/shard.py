"""Splitting independent work across ranks (one process per GPU).

Blocks never read one another (every block is padded on its own, Sec. II.B-C),
so images and block ranges shard across GPUs with no exchange: each rank
filters its own share and the only collective is the timing reduction of
the benchmark.  These helpers are plain host logic.
"""
from __future__ import annotations


def shard_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """Balanced contiguous [begin, end) share of `total` units for `rank`."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    return total * rank // world, total * (rank + 1) // world


def shard_items(sizes: list[int], rank: int, world: int) -> list[int]:
    """Indices of the items (e.g. images of a grouped batch, by block count)
    given to `rank`: greedy longest-first onto the least-loaded rank, so
    uneven images still balance by blocks.  Deterministic on every rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad shard arguments")
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def max_over_ranks(value: float, dist=None) -> float:
    """The largest `value` over all ranks (the job ends with its slowest rank)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
