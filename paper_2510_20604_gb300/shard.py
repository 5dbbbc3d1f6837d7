"""Sharding of the trees across ranks (one process per GPU).

Every successor draw is keyed by the global tree id, so rank r sampling the
ids [tree0 + r T, tree0 + (r + 1) T) and the ranks adding their per-vertex
visit sums give exactly the trees and sums of one process sampling all
N T ids (weak scaling: T trees per rank).  The sums are integers below 2^53
held in FP64, so the all-reduce is exact in any order.  No other step of the
path exchanges data: the pivot solve and the recovery run on the reduced
sums, on every rank or on one.
"""
from __future__ import annotations


def tree_range(rank: int, world: int, trees_per_rank: int, tree0: int = 0) -> tuple[int, int]:
    """(first global tree id, count) of rank ``rank`` of ``world``."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside [0, {world})")
    if trees_per_rank < 0 or tree0 < 0:
        raise ValueError("tree counts and offsets must be non-negative")
    first = tree0 + rank * trees_per_rank
    if first + trees_per_rank > (1 << 32):
        raise ValueError("global tree ids must lie in [0, 2^32)")
    return first, trees_per_rank


def all_reduce_sums(sums, group=None):
    """Add the per-vertex visit sums of all ranks in place (torch.distributed)."""
    import torch.distributed as dist
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums
