"""Data parallelism over views (one process per GPU).

Each rank renders its own subset of the views -- their images, losses and 2D
gradients are independent -- and the only exchange is the sum of the
raw-parameter gradients, N * 4 (15 + 6M) bytes per step, as one all-reduce
(NCCL on GPUs; any torch.distributed backend works).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> tuple[int, int]:
    """(rank, world size); (0, 1) without an initialised process group."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard_views(cameras, rank: int, world_size: int):
    """Round-robin split of the views: rank r renders views r, r + N, ..."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("invalid rank / world size")
    return list(cameras)[rank::world_size]


def reduce_gradients(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Sums the per-rank parameter gradients in place (identity on one rank)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks (the step time of a weak-scaling run)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
