"""Multi-GPU sharding of a render: one process per GPU.

Paths are independent and every random number is keyed by the global path
id, so rank r of W traces the ids [r * N, (r + 1) * N) (weak scaling, N paths
per rank) and the per-rank histogram estimates are averaged with one FP64
sum all-reduce -- the only exchange the method has.  The result equals a
single render of W * N paths up to FP64 summation order.
"""
from __future__ import annotations


def path_offset(rank: int, paths_per_rank: int) -> int:
    """First global path id of `rank`."""
    return int(rank) * int(paths_per_rank)


def combine(hist, world_size: int, group=None):
    """Average per-rank histogram estimates in place (sum all-reduce / W)."""
    if world_size > 1:
        import torch.distributed as dist
        dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
        hist.div_(world_size)
    return hist
