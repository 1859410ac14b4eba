"""Uncertainty-driven run lengths (Sec. 2.4): how many histories, and how much
device time, the plain method needs to reach a target mean relative
uncertainty, using the batch method of eq. (1) on the device."""
from __future__ import annotations


def time_to_sigma(eng, beam, shape, seed, target=0.02, frac=0.5, n_batches=10, n0=200_000, device=0,
                  max_rounds=5, track_group=1):
    """Device seconds and histories for the mean eq. (1) uncertainty over
    voxels above frac * max to fall to ``target``.  The history count is
    predicted from sigma ~ N^-1/2 and re-measured until reached (or the beam
    runs out of histories)."""
    import torch
    dev = f"cuda:{device}"
    s1 = torch.zeros(shape, dtype=torch.float64, device=dev)
    s2 = torch.zeros_like(s1)
    total = int(beam["n_histories"].sum())

    def measure(n):
        n = min(total, max(n_batches, (n // n_batches) * n_batches))
        kw = dict(n_batches=n_batches, batch_sum=s1, batch_sumsq=s2, track_group=track_group)
        eng.run_ex(beam, n, seed, **kw)  # capture / warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        eng.run_ex(beam, n, seed, **kw)
        e1.record()
        e1.synchronize()
        _, _, rel = eng.batch_stats(s1, s2, n_batches, frac)
        return n, e0.elapsed_time(e1) * 1e-3, rel

    n, sec, rel = measure(n0)
    for _ in range(max_rounds):
        if rel <= target or n >= total:
            break
        n, sec, rel = measure(int(n * (rel / target) ** 2 * 1.05) + n_batches)
    return {"histories": n, "seconds": sec, "mean_rel_sigma": rel, "target": target, "frac": frac,
            "n_batches": n_batches, "track_group": track_group, "reached": bool(rel <= target)}
