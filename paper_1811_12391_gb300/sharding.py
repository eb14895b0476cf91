"""Batch-axis sharding across ranks (one process per GPU).

The path shards naturally on independent instances (the views of an axial
scan, or separate phantoms): each rank solves a contiguous block of them, and
the only exchange is one FP64 sum of the per-rank dose at the end.  Timing
uses the maximum over ranks.  These helpers take a torch.distributed process
group (nccl on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import List, Sequence


def block(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def my_items(items: Sequence, rank: int, world: int) -> List:
    return [items[i] for i in block(len(items), rank, world)]


def sum_dose(dose, group=None):
    """All-reduce (sum) of a per-rank FP64 dose tensor in place; returns it."""
    import torch
    import torch.distributed as dist
    if dose.dtype != torch.float64:
        raise TypeError("dose must be float64")
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(dose, op=dist.ReduceOp.SUM, group=group)
    return dose


def max_time(ms: float, device=None, group=None) -> float:
    """Maximum over ranks of a per-rank duration."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
