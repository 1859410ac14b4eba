"""FP64 statistics of Sec. 2.4 (test infrastructure only).

Eq. (1), batch method: with n independent batches of dose D_i and mean
D_bar, sigma_Dbar = sqrt( sum_i (D_i - D_bar)^2 / (n (n - 1)) ).

Eq. (2), history-by-history method: with N primary histories contributing
D_i each, sigma_D = sqrt( (sum D_i^2 / N - (sum D_i / N)^2) / (N - 1) ).
The printed equation runs its sums to n; they run over the N histories.
This estimates the uncertainty of the mean per-history dose; multiplying by
N gives the uncertainty of the summed dose.

Mean dose uncertainty: average of sigma_D / D over voxels whose dose is above
half the maximum dose.
"""
from __future__ import annotations

import numpy as np


def batch_sigma(batches):
    """Eq. (1) from an explicit stack of batch doses [n, ...]."""
    d = np.asarray(batches, dtype=np.float64)
    n = d.shape[0]
    if n < 2:
        raise ValueError("eq. (1) needs at least two batches")
    mean = d.mean(axis=0)
    return mean, np.sqrt(((d - mean) ** 2).sum(axis=0) / (n * (n - 1)))


def batch_sigma_from_sums(s, s2, n):
    """Eq. (1) from per-voxel sum and sum of squares over n batches."""
    s = np.asarray(s, np.float64)
    s2 = np.asarray(s2, np.float64)
    mean = s / n
    ss = np.maximum(s2 - s * s / n, 0.0)
    return mean, np.sqrt(ss / (n * (n - 1)))


def history_sigma(s, s2, N):
    """Eq. (2): per-voxel sigma of the mean per-history dose."""
    s = np.asarray(s, np.float64)
    s2 = np.asarray(s2, np.float64)
    var = np.maximum(s2 / N - (s / N) ** 2, 0.0) / (N - 1)
    return np.sqrt(var)


def mean_relative_uncertainty(dose, sigma, frac=0.5):
    """Average of sigma/D over voxels with D > frac * max(D)."""
    dose = np.asarray(dose, np.float64)
    sigma = np.asarray(sigma, np.float64)
    m = dose > frac * dose.max()
    if not np.any(m):
        return float("nan")
    return float(np.mean(sigma[m] / dose[m]))
