"""Gamma index (Low, Harms, Mutic & Purdy 1998), global dose difference,
voxel-centre sampling: test infrastructure only.

gamma(v) = min over evaluated voxels u with |u - v| within the search radius
of sqrt(|u - v|^2 / dta^2 + (eval(u) - ref(v))^2 / (dose_frac * max(ref))^2),
for reference voxels with ref(v) > threshold * max(ref).  Pass rate: share of
those voxels with gamma <= 1.
"""
from __future__ import annotations

import math

import numpy as np


def gamma(ref, ev, spacing, dose_frac=0.02, dta=0.2, threshold=0.1, radius=None):
    ref = np.asarray(ref, np.float64)
    ev = np.asarray(ev, np.float64)
    sx, sy, sz = spacing
    if radius is None:
        radius = min(8, int(math.ceil(1.5 * dta / min(spacing))))
    mx = ref.max()
    dmax = dose_frac * mx
    nz, ny, nx = ref.shape
    best = np.full(ref.shape, np.inf)
    for a in range(-radius, radius + 1):
        for b in range(-radius, radius + 1):
            for c in range(-radius, radius + 1):
                dist2 = (a * sz) ** 2 + (b * sy) ** 2 + (c * sx) ** 2
                # evaluated value at v + (a, b, c), inf outside the grid
                sh = np.full(ref.shape, np.nan)
                zs = slice(max(0, -a), nz - max(0, a))
                ys = slice(max(0, -b), ny - max(0, b))
                xs = slice(max(0, -c), nx - max(0, c))
                zd = slice(max(0, a), nz - max(0, -a))
                yd = slice(max(0, b), ny - max(0, -b))
                xd = slice(max(0, c), nx - max(0, -c))
                sh[zs, ys, xs] = ev[zd, yd, xd]
                g2 = dist2 / dta ** 2 + (sh - ref) ** 2 / dmax ** 2
                g2 = np.where(np.isnan(g2), np.inf, g2)
                best = np.minimum(best, g2)
    g = np.sqrt(best)
    mask = ref > threshold * mx
    out = np.where(mask, g, -1.0)
    return out, float(np.mean(g[mask] <= 1.0)) if mask.any() else 0.0
