"""Data parallelism over views (one process per GPU).

Each rank renders its own subset of the views -- their images, losses and 2D
gradients are independent -- and the only exchange is the sum of the
raw-parameter gradients, N * 4 (15 + 6M) bytes per step, as one all-reduce
(NCCL on GPUs; any torch.distributed backend works), or as one asynchronous
all-reduce per chunk of primitives, each started as soon as the projection
backward has written that chunk.
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


def chunk_ranges(n: int, chunk: int):
    """[c0, c1) primitive ranges of at most `chunk` primitives; every c0 is a
    multiple of 4 (the C ABI wants 16-byte aligned parameter planes)."""
    chunk = max(4, (int(chunk) + 3) // 4 * 4)
    return [(c0, min(c0 + chunk, n)) for c0 in range(0, n, chunk)]


def reduce_gradients_chunked(grad: torch.Tensor, produce, n: int, chunk: int, group=None) -> torch.Tensor:
    """Sums the per-rank gradients like reduce_gradients, overlapped with
    their production: produce(c0, c1) writes the gradient columns [c0, c1)
    (the projection backward over those primitives), and each chunk's
    all-reduce is started asynchronously as soon as it is written, so it runs
    while the next chunks are computed.  Columns beyond n are left alone."""
    multi = dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1
    pending = []
    for c0, c1 in chunk_ranges(n, chunk):
        produce(c0, c1)
        if multi:
            buf = grad[:, c0:c1].contiguous()          # staging copy, ordered after produce()
            pending.append((c0, c1, buf, dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group,
                                                          async_op=True)))
    for c0, c1, buf, work in pending:
        work.wait()
        grad[:, c0:c1].copy_(buf)
    return grad


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks (the step time of a weak-scaling run)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
