"""Shot sharding across ranks (one process per GPU).

Shots are independent problems until the gradient sum, so a multi-GPU
gradient gives each rank a contiguous block of shots and exchanges one
gradient-sized buffer and the misfit per FWI iteration.
"""
from __future__ import annotations


def shard(nshot: int, rank: int, world: int) -> list[int]:
    """Contiguous, balanced block of shot indices owned by `rank`."""
    if world < 1 or not (0 <= rank < world) or nshot < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(nshot, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return list(range(lo, hi))


def allreduce_gradient(grad, misfit: float, group=None):
    """Sum the per-rank gradients (in place) and misfits over the process
    group; returns the total misfit."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    t = torch.tensor([misfit], dtype=torch.float64, device=grad.device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
