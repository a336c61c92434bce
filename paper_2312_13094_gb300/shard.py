"""Shot-parallel runs over several processes (one per GPU).

Shots are independent problems (Sec. IV-B models one shot per run; the
gradient of a multi-shot misfit is the sum of the per-shot gradients), so the
forward path shards with no exchange at all: rank r takes a contiguous,
balanced share of the shot list.  The one collective is the sum of the
per-rank gradient partial sums (plus the max of the per-rank times when a run
is timed).  torch.distributed carries both (NCCL on GPUs, gloo on CPU ranks).
"""
from __future__ import annotations


def shot_range(nshots: int, world: int, rank: int) -> range:
    """Shots of `rank`: [rank*n/world, (rank+1)*n/world) -- every shot exactly
    once over the ranks, shares differing by at most one."""
    if world < 1 or not 0 <= rank < world or nshots < 0:
        raise ValueError(f"bad split: nshots={nshots} world={world} rank={rank}")
    return range(nshots * rank // world, nshots * (rank + 1) // world)


def sum_over_ranks(t, dist=None):
    """In-place sum of a tensor over all ranks (no-op without a process group)."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def max_over_ranks(t, dist=None):
    """In-place max of a tensor over all ranks (no-op without a process group)."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t


def shot_parallel_gradient(nshots: int, grad_of_shot, like, dist=None):
    """Sum over all shots of grad_of_shot(s) (a tensor shaped like `like`),
    each rank evaluating only its share, then one sum over ranks.  Returns the
    full sum on every rank, and the per-rank loss sum likewise reduced."""
    import torch
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    rank = dist.get_rank() if dist is not None and dist.is_initialized() else 0
    acc = torch.zeros_like(like)
    loss = torch.zeros(1, dtype=torch.float64, device=like.device)
    for s in shot_range(nshots, world, rank):
        g, l_s = grad_of_shot(s)
        acc += g
        loss += l_s
    sum_over_ranks(acc, dist)
    sum_over_ranks(loss, dist)
    return acc, float(loss)
