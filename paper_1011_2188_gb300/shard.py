"""Multi-process split of a run over the history index space.

Histories are independent (Sec. 2.3: each thread re-traces its own history)
and the energy tally is an int64 sum, so N processes can each replay a
contiguous range of history indices and add their tallies: the sum equals
the tally of one process replaying every history, bit for bit, whatever the
split.  The paper's two-GPU card did the same -- one host thread per GPU,
each on its own histories, doses summed at the end (Sec. 2.3).  Here the sum
is one all-reduce of the int64 tally (NCCL between GPUs; gloo stages it
through host memory), followed by a single conversion to dose.
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
    """Sum an int64 (or float64) tally tensor over the process group, in
    place.  With the gloo backend a CUDA tensor is summed through a host copy;
    NCCL reduces device memory directly.  Integer sums are exact and do not
    depend on the order in which the ranks' tallies are added."""
    import torch.distributed as dist
    if tally.is_cuda and dist.get_backend(group) == "gloo":
        host = tally.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
        tally.copy_(host)
    else:
        dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally


def run_sharded(eng, spots, n_histories, seed, rank, world, group=None, tally=None, dose=None,
                history_offset=0, **run_opts):
    """This rank's share of a run of ``n_histories`` histories starting at
    ``history_offset``: replay the rank's contiguous range through
    ``eng.run_ex`` into an int64 tally, all-reduce the tally over the group
    and convert the sum to dose once (``fdc_dose_from_tally``).  Every rank
    returns (tally, dose) of the whole run; ``run_opts`` are passed to
    ``run_ex`` (track_group, fp64_geometry, schedule, ...)."""
    import torch
    lo, hi = shard_range(n_histories, rank, world)
    dev = f"cuda:{eng.device}"
    if tally is None:
        tally = torch.empty(eng.shape, dtype=torch.int64, device=dev)
    if hi > lo:
        eng.run_ex(spots, hi - lo, seed, history_offset=history_offset + lo, tally=tally, **run_opts)
    else:
        tally.zero_()
    eng.sync()
    if world > 1:
        all_reduce_tally(tally, group)
    dose = eng.dose_from_tally(tally, dose)
    return tally, dose
