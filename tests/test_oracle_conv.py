"""Pins of the FP64 convolution reference used to check the denoiser kernels."""
import numpy as np
import pytest

from oracle import conv3d


def test_forward_matches_scipy_correlate_single_channel():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 6, 5, 7, 1))
    w = rng.normal(size=(1, 3, 3, 3, 1))
    y = conv3d.forward(x, w, stride=1, pad=1)
    ref = scipy_signal.correlate(x[0, :, :, :, 0], w[0, :, :, :, 0], mode="same")
    np.testing.assert_allclose(y[0, :, :, :, 0], ref, rtol=1e-12, atol=1e-12)


def test_forward_strided_brute_force():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 6, 4, 3))
    w = rng.normal(size=(5, 2, 2, 2, 3))
    b = rng.normal(size=5)
    y = conv3d.forward(x, w, b, stride=2, pad=0)
    assert y.shape == (2, 2, 3, 2, 5)
    ref = np.zeros_like(y)
    for bb in range(2):
        for d in range(2):
            for h in range(3):
                for ww in range(2):
                    patch = x[bb, 2 * d:2 * d + 2, 2 * h:2 * h + 2, 2 * ww:2 * ww + 2, :]
                    ref[bb, d, h, ww] = np.einsum("abci,oabci->o", patch, w) + b
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k,s,p", [(3, 1, 1), (2, 2, 0), (1, 1, 0)])
def test_adjoint_identities(k, s, p):
    """<conv(x), dy> = <x, dgrad(dy)> and = <w, wgrad(x, dy)> for the
    bias-free linear map; pins the two gradients against the forward."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 6, 4, 6, 3))
    w = rng.normal(size=(4, k, k, k, 3))
    y = conv3d.forward(x, w, stride=s, pad=p)
    dy = rng.normal(size=y.shape)
    lhs = np.sum(y * dy)
    dx = conv3d.backward_data(dy, w, x.shape, stride=s, pad=p)
    dw, db = conv3d.backward_weights(x, dy, k, stride=s, pad=p)
    assert abs(lhs - np.sum(x * dx)) < 1e-9 * abs(lhs)
    assert abs(lhs - np.sum(w * dw)) < 1e-9 * abs(lhs)
    np.testing.assert_allclose(db, dy.sum(axis=(0, 1, 2, 3)))


def test_finite_difference_gradient():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(1, 4, 4, 4, 2))
    w = rng.normal(size=(3, 3, 3, 3, 2))
    b = rng.normal(size=3)
    dy = rng.normal(size=(1, 4, 4, 4, 3))

    def loss(xx, ww, bb):
        return np.sum(conv3d.forward(xx, ww, bb, relu=True) * dy)

    y = conv3d.forward(x, w, b, relu=True)
    g = dy * (y > 0)
    dx = conv3d.backward_data(g, w, x.shape)
    dw, db = conv3d.backward_weights(x, g, 3)
    eps = 1e-6
    for idx in [(0, 1, 2, 3, 1), (0, 0, 0, 0, 0), (0, 3, 3, 3, 1)]:
        e = np.zeros_like(x)
        e[idx] = eps
        fd = (loss(x + e, w, b) - loss(x - e, w, b)) / (2 * eps)
        assert abs(fd - dx[idx]) < 1e-5 * max(1.0, abs(fd))
    for idx in [(0, 1, 1, 1, 0), (2, 0, 2, 1, 1)]:
        e = np.zeros_like(w)
        e[idx] = eps
        fd = (loss(x, w + e, b) - loss(x, w - e, b)) / (2 * eps)
        assert abs(fd - dw[idx]) < 1e-5 * max(1.0, abs(fd))
    e = np.zeros(3)
    e[1] = eps
    fd = (loss(x, w, b + e) - loss(x, w, b - e)) / (2 * eps)
    assert abs(fd - db[1]) < 1e-5 * max(1.0, abs(fd))


def test_upsample_adjoint():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(1, 2, 3, 2, 4))
    dy = rng.normal(size=(1, 4, 6, 4, 4))
    assert abs(np.sum(conv3d.upsample2(x) * dy) - np.sum(x * conv3d.upsample2_adjoint(dy))) < 1e-10


def test_gamma_closed_forms():
    from oracle import gamma as G
    sp = (0.2, 0.2, 0.2)
    ref = np.full((6, 5, 4), 3.0)
    g, pr = G.gamma(ref, ref, sp)
    assert np.all(g == 0.0) and pr == 1.0
    # uniform 1 % excess with a 2 % criterion: gamma = 0.5 everywhere
    g, pr = G.gamma(ref, 1.01 * ref, sp)
    np.testing.assert_allclose(g, 0.5, rtol=1e-12)
    # step edge shifted by two voxels (0.4 cm = 2 DTA): gamma = 2 at the voxels
    # that lost the dose, 0 elsewhere
    ref = np.zeros((12, 1, 1))
    ref[:6] = 10.0
    ev = np.zeros_like(ref)
    ev[:4] = 10.0
    g, pr = G.gamma(ref, ev, sp, dta=0.2, threshold=0.1)
    np.testing.assert_allclose(g[:4, 0, 0], 0.0)
    np.testing.assert_allclose(g[4, 0, 0], 1.0)   # one voxel to the nearest matching dose
    np.testing.assert_allclose(g[5, 0, 0], 2.0)
    assert np.all(g[6:] == -1.0)
    assert pr == 5 / 6
