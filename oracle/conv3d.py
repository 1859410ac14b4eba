"""FP64 reference of the denoiser's convolutions (test infrastructure only).

Definitions (channels-last x[b][d][h][w][c], weights w[co][kd][kh][kw][ci]):

  forward  y[b, o, co]  = bias[co] + sum_{t, ci} x[b, o*s - p + t, ci] w[co, t, ci]
  data     dx[b, i, ci] = sum_{(o, t): o*s - p + t = i} sum_co dy[b, o, co] w[co, t, ci]
  weights  dw[co, t, ci] = sum_{b, o} dy[b, o, co] x[b, o*s - p + t, ci]
  bias     db[co]        = sum_{b, o} dy[b, o, co]

(out-of-range input positions are zero padding; t runs over the k^3 taps).
Written as sums over taps of shifted slices, in the order of the definition.
"""
from __future__ import annotations

import numpy as np


def out_size(n, k, s, p):
    return (n + 2 * p - k) // s + 1


def _pad(x, p):
    return np.pad(x, ((0, 0), (p, p), (p, p), (p, p), (0, 0)))


def _taps(k):
    return [(a, b, c) for a in range(k) for b in range(k) for c in range(k)]


def forward(x, w, bias=None, stride=1, pad=1, relu=False):
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, D, H, W, Ci = x.shape
    Co, k = w.shape[0], w.shape[1]
    Do, Ho, Wo = (out_size(n, k, stride, pad) for n in (D, H, W))
    xp = _pad(x, pad)
    y = np.zeros((B, Do, Ho, Wo, Co))
    for (a, b, c) in _taps(k):
        sl = xp[:, a:a + stride * (Do - 1) + 1:stride, b:b + stride * (Ho - 1) + 1:stride,
                c:c + stride * (Wo - 1) + 1:stride, :]
        y += sl @ w[:, a, b, c, :].T
    if bias is not None:
        y += np.asarray(bias, np.float64)
    if relu:
        y = np.maximum(y, 0.0)
    return y


def backward_data(dy, w, in_shape, stride=1, pad=1):
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    B, D, H, W, Ci = in_shape
    _, Do, Ho, Wo, Co = dy.shape
    k = w.shape[1]
    dxp = np.zeros((B, D + 2 * pad + stride, H + 2 * pad + stride, W + 2 * pad + stride, Ci))
    for (a, b, c) in _taps(k):
        dxp[:, a:a + stride * (Do - 1) + 1:stride, b:b + stride * (Ho - 1) + 1:stride,
            c:c + stride * (Wo - 1) + 1:stride, :] += dy @ w[:, a, b, c, :]
    return dxp[:, pad:pad + D, pad:pad + H, pad:pad + W, :]


def backward_weights(x, dy, k, stride=1, pad=1):
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    _, Do, Ho, Wo, Co = dy.shape
    Ci = x.shape[-1]
    xp = _pad(x, pad)
    dw = np.zeros((Co, k, k, k, Ci))
    for (a, b, c) in _taps(k):
        sl = xp[:, a:a + stride * (Do - 1) + 1:stride, b:b + stride * (Ho - 1) + 1:stride,
                c:c + stride * (Wo - 1) + 1:stride, :]
        dw[:, a, b, c, :] = np.einsum("bdhwo,bdhwi->oi", dy, sl)
    db = dy.sum(axis=(0, 1, 2, 3))
    return dw, db


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample2_adjoint(dy):
    B, D, H, W, C = dy.shape
    return dy.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))
