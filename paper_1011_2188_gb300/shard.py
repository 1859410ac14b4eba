"""Host-side partition of the history index space across ranks.

Histories are independent (Sec. 2.3: each thread re-traces its own history)
and the integer energy tally is additive, so N processes can each replay a
contiguous range of history indices and the tallies add up bitwise to the
single-process result; the paper's two-GPU card split its histories the same
way and summed the doses at the end.
"""
from __future__ import annotations


def shard_range(total: int, rank: int, world: int):
    """Contiguous [lo, hi) of ``total`` histories for ``rank`` of ``world``
    (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard request")
    lo = total * rank // world
    hi = total * (rank + 1) // world
    return lo, hi


def weak_shard(per_rank: int, rank: int):
    """Weak scaling: every rank replays ``per_rank`` histories of a beam
    holding world * per_rank, at offset rank * per_rank."""
    return rank * per_rank, (rank + 1) * per_rank


def all_reduce_tally(tally, group=None):
    """Sum an int64 (or float64) tally tensor over the process group in place."""
    import torch.distributed as dist
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally
