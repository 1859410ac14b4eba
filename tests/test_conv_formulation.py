"""The algebra of the kw-stacked tensor-core convolution, checked on the CPU
against the FP64 reference convolution: for an output block of 8 (h) x 14 (w)
voxels at depth d0, with A the input halo rows (row m = 16 h + w' for input
column w0 - 1 + w', one matrix per (kd, kh)) and B the weights of the three kw
taps stacked along N (column kw NT + co),

    D[m][kw NT + co] = sum_{kd, kh} A_{kd,kh}[m] . B_{kd,kh}[kw NT + co]
    y[h][w][co]      = sum_kw D[16 h + w + kw][kw NT + co]    (w < 14).

This is the identity the kernel's MMAs and epilogue implement."""
import numpy as np

from oracle import conv3d as ref


def test_kw_stacked_block_equals_convolution():
    rng = np.random.default_rng(4)
    D_, H_, W_, Ci, NT = 5, 11, 19, 16, 16
    x = rng.normal(size=(1, D_, H_, W_, Ci))
    w = rng.normal(size=(NT, 3, 3, 3, Ci))
    y_ref = ref.forward(x, w)[0]
    for d0, h0, w0 in [(0, 0, 0), (2, 8, 14), (4, 8, 0)]:
        D = np.zeros((128, 3 * NT))
        for kd in range(3):
            for kh in range(3):
                A = np.zeros((128, Ci))
                for m in range(128):
                    h, wp = m // 16, m % 16
                    zi, yi, xi = d0 - 1 + kd, h0 - 1 + h + kh, w0 - 1 + wp
                    if 0 <= zi < D_ and 0 <= yi < H_ and 0 <= xi < W_:
                        A[m] = x[0, zi, yi, xi]
                B = np.concatenate([w[:, kd, kh, kw, :] for kw in range(3)], axis=0)  # (3 NT, Ci)
                D += A @ B.T
        for m in range(128):
            h, wl = m // 16, m % 16
            if wl >= 14 or h0 + h >= H_ or w0 + wl >= W_:
                continue
            y = D[m, 0:NT] + D[m + 1, NT:2 * NT] + D[m + 2, 2 * NT:3 * NT]
            np.testing.assert_allclose(y, y_ref[d0, h0 + h, w0 + wl], rtol=1e-10, atol=1e-10)
