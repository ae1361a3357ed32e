"""Shot sharding across ranks (one process per GPU).

Shots are independent problems until the gradient sum (Section 3.1: the
misfit and its gradient are sums over shots), so a multi-GPU gradient gives
each rank a contiguous block of shots and exchanges one gradient-sized
buffer and the misfit per FWI iteration.
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
    if not grad.is_cuda and dist.get_backend(group) == "nccl":
        # NCCL reduces device memory only: reduce a device copy of a host gradient
        g = grad.to(torch.device("cuda", torch.cuda.current_device()))
        total = allreduce_gradient(g, misfit, group)
        grad.copy_(g.cpu())
        return total
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    t = torch.tensor([misfit], dtype=torch.float64, device=grad.device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def sharded_adjoint_gradient(mesh, shot_ids, d_obs, grad, group=None, ckpt_every=-1, compute=None):
    """Misfit and gradient of all `shot_ids`, with the shots partitioned over
    the ranks of `group`: this rank runs the adjoint-state gradient on its
    contiguous block of shots, then one sum-allreduce of the gradient and one
    of the misfit give every rank the totals.

    d_obs: observed data [len(shot_ids)][nrec][2][nt] of all shots, or of
    this rank's block only (the block is taken when the leading dimension is
    the full shot count).  grad: [3][nz][nx], overwritten with the total.
    compute(ids, d_obs_block, grad) -> misfit runs one rank's share; the
    default is ``mesh.adjoint_gradient`` (the CUDA library).  A rank with no
    shots contributes zeros.  Returns the total misfit."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = shard(len(shot_ids), rank, world)
    if compute is None:
        def compute(ids, d_blk, g):
            return mesh.adjoint_gradient(ids, d_blk, g, ckpt_every)
    if mine:
        blk = d_obs[mine[0]:mine[-1] + 1] if d_obs.shape[0] == len(shot_ids) else d_obs
        if blk.shape[0] != len(mine):
            raise ValueError("d_obs holds neither every shot nor this rank's block")
        if hasattr(blk, "is_contiguous") and not blk.is_contiguous():
            blk = blk.contiguous()
        f = compute([shot_ids[i] for i in mine], blk, grad)
    else:
        grad.zero_()
        f = 0.0
    return allreduce_gradient(grad, f, group)
