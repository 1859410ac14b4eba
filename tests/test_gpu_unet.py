"""Denoiser kernels through the C ABI against the FP64 references of the
oracle package (GB300 only)."""
import ctypes as C

import numpy as np
import pytest

from oracle import conv3d as ref
from oracle import gamma as gref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def bf16(a):
    """Round to bfloat16 (nearest even) and return (torch bf16 tensor on the
    GPU, the rounded values as float64)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)
    return t.cuda(), t.to(torch.float64).numpy()


def geom(x_shape, cout, k, s, p, relu=0):
    from paper_1011_2188_gb300.denoise import Conv3d
    B, D, H, W, Ci = x_shape
    o = [(n + 2 * p - k) // s + 1 for n in (D, H, W)]
    return Conv3d(B, D, H, W, o[0], o[1], o[2], Ci, cout, k, s, p, relu), (B, *o, cout)


def ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


CASES = [
    # (shape, cout, k, s, p)
    ((1, 7, 6, 9, 16), 16, 3, 1, 1),
    ((2, 5, 6, 7, 32), 64, 3, 1, 1),
    ((1, 8, 6, 10, 16), 32, 2, 2, 0),
    ((1, 6, 4, 8, 64), 128, 2, 2, 0),
    # the network's 32^3 -> 16^3 down-convolution (128 CTAs, K split five
    # ways over 32 K steps: uneven split ranges) and a 16^3 input (16 CTAs,
    # sixteen splits of two K steps)
    ((1, 32, 32, 32, 64), 128, 2, 2, 0),
    ((1, 16, 16, 16, 64), 128, 2, 2, 0),
    ((1, 9, 5, 6, 32), 16, 1, 1, 0),
    ((1, 4, 4, 6, 128), 64, 3, 1, 1),
    ((1, 16, 16, 16, 16), 16, 3, 1, 1),
    ((2, 3, 9, 17, 48), 32, 3, 1, 1),
    ((1, 3, 37, 12, 16), 32, 3, 1, 1),  # three 16-row tiles in h, the last ragged
    ((1, 10, 31, 64, 16), 64, 3, 1, 1),  # enough blocks for the 64-channel tile kernel, ragged h
    # d-walking kernel (input channels <= 32): batch 2 with ragged h and w,
    # two input slices with 32-channel output tiles, a single plane
    ((2, 9, 17, 29, 32), 16, 3, 1, 1),
    ((1, 12, 9, 30, 32), 32, 3, 1, 1),
    ((1, 1, 8, 14, 16), 16, 3, 1, 1),
    # stride-2 down-convolution on odd sizes: the last input plane of each
    # axis reaches no output (zero data gradient), parity classes of unequal size
    ((2, 7, 5, 9, 16), 32, 2, 2, 0),
    # weight gradient with several 16-plane chunks along d, the last ragged
    ((1, 37, 5, 9, 16), 16, 3, 1, 1),
    ((1, 21, 3, 10, 64), 32, 3, 1, 1),
    # stride-2 down-convolutions on the tensor-core path: 32 -> 64, batch 2 with odd sizes
    ((1, 6, 8, 10, 32), 64, 2, 2, 0),
    ((2, 5, 7, 9, 32), 64, 2, 2, 0),
    # TMA d-walking kernel (input read as stored, h >= 10, w >= 16): the
    # smallest grid its boxes allow; walks of several planes per CTA whose
    # ranges restart at tile columns and wrap the plane ring (16- and 32-channel
    # tiles, one and two input slices); four input slices, one CTA per SM
    ((1, 5, 10, 16, 16), 16, 3, 1, 1),
    ((1, 96, 64, 60, 16), 16, 3, 1, 1),
    ((1, 64, 40, 30, 32), 32, 3, 1, 1),
    ((2, 40, 19, 33, 32), 16, 3, 1, 1),
    ((1, 9, 23, 45, 64), 32, 3, 1, 1),
    # one 16-channel tensor, even w >= 32: ragged last tile, two 16-channel
    # output tiles, batch 2 at the smallest width
    ((1, 12, 21, 70, 16), 32, 3, 1, 1),
    ((2, 7, 10, 32, 16), 16, 3, 1, 1),
    # 128 input channels, forward: the K dimension split into two 64-channel
    # parts over CTAs, FP32 partials combined with bias and ReLU (the 16^3
    # bottleneck shape; a ragged 32^3-level shape with two output tiles)
    ((1, 16, 16, 16, 128), 128, 3, 1, 1),
    ((1, 9, 20, 36, 128), 64, 3, 1, 1),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("relu", [0, 1])
def test_conv_forward(case, relu):
    import torch
    from paper_1011_2188_gb300 import fdc
    shape, cout, k, s, p = case
    rng = np.random.default_rng(hash((shape, cout, relu)) % 2**32)
    xt, x = bf16(rng.normal(size=shape))
    wt, w = bf16(rng.normal(size=(cout, k, k, k, shape[-1])) / np.sqrt(k ** 3 * shape[-1]))
    b = rng.normal(size=cout).astype(np.float32)
    g, oshape = geom(shape, cout, k, s, p, relu)
    y32 = torch.empty(oshape, dtype=torch.float32, device="cuda:0")
    y16 = torch.empty(oshape, dtype=torch.bfloat16, device="cuda:0")
    bt = torch.from_numpy(b).cuda()
    assert fdc.lib().fdc_conv3d_forward(C.byref(g), ptr(xt), ptr(wt), ptr(bt), ptr(y16), ptr(y32), None) == 0
    torch.cuda.synchronize()
    r = ref.forward(x, w, b.astype(np.float64), stride=s, pad=p, relu=bool(relu))
    mx = np.abs(r).max()
    np.testing.assert_allclose(y32.cpu().numpy(), r, rtol=0, atol=2e-5 * mx)
    np.testing.assert_allclose(y16.float().cpu().numpy(), r, rtol=0, atol=8e-3 * mx)


@pytest.mark.parametrize("case", CASES)
def test_conv_backward_data_and_weights(case):
    import torch
    from paper_1011_2188_gb300 import fdc
    shape, cout, k, s, p = case
    rng = np.random.default_rng(7 + len(shape) + cout)
    xt, x = bf16(rng.normal(size=shape))
    wt, w = bf16(rng.normal(size=(cout, k, k, k, shape[-1])) / np.sqrt(k ** 3 * shape[-1]))
    g, oshape = geom(shape, cout, k, s, p)
    dyt, dy = bf16(rng.normal(size=oshape))
    L = fdc.lib()
    w_t = torch.empty((shape[-1], k, k, k, cout), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_transpose_weights(C.byref(g), ptr(wt), ptr(w_t), None) == 0
    # layout of the data-gradient weights: transposed, taps reflected for 3^3 stride 1 padding 1
    wr = np.transpose(w, (4, 1, 2, 3, 0))
    if (k, s, p) == (3, 1, 1):
        wr = wr[:, ::-1, ::-1, ::-1, :]
    np.testing.assert_array_equal(w_t.double().cpu().numpy(), wr)
    dx = torch.empty(shape, dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_backward_data(C.byref(g), ptr(dyt), ptr(w_t), None, ptr(dx), None) == 0
    # the same with the ReLU derivative of the input applied in the epilogue
    dxm = torch.empty(shape, dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_backward_data(C.byref(g), ptr(dyt), ptr(w_t), ptr(xt), ptr(dxm), None) == 0
    dw = torch.zeros(w.shape, dtype=torch.float32, device="cuda:0")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda:0")
    assert L.fdc_conv3d_backward_weights(C.byref(g), ptr(xt), ptr(dyt), ptr(dw), ptr(db), None) == 0
    torch.cuda.synchronize()
    rdx = ref.backward_data(dy, w, shape, stride=s, pad=p)
    rdw, rdb = ref.backward_weights(x, dy, k, stride=s, pad=p)
    np.testing.assert_allclose(dx.float().cpu().numpy(), rdx, rtol=0, atol=8e-3 * np.abs(rdx).max())
    assert torch.equal(dxm, torch.where(xt > 0, dx, torch.zeros_like(dx)))
    # masked data gradient plus a residual gradient, rounded once
    rest, res = bf16(rng.normal(size=shape) * np.abs(rdx).max())
    dxr = torch.empty(shape, dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_backward_data_add(C.byref(g), ptr(dyt), ptr(w_t), ptr(xt), ptr(rest), ptr(dxr), None) == 0
    assert L.fdc_conv3d_backward_data_add(C.byref(g), ptr(dyt), ptr(w_t), ptr(xt), ptr(dxr), ptr(dxr), None) != 0
    torch.cuda.synchronize()
    rr = np.where(x > 0, rdx, 0.0) + res
    np.testing.assert_allclose(dxr.float().cpu().numpy(), rr, rtol=0, atol=8e-3 * np.abs(rr).max())
    np.testing.assert_allclose(dw.cpu().numpy(), rdw, rtol=0, atol=2e-5 * np.abs(rdw).max())
    np.testing.assert_allclose(db.cpu().numpy(), rdb, rtol=0, atol=2e-5 * np.abs(rdb).max())
    # accumulation into a weight gradient that is not 16-byte aligned (scalar atomics)
    store = torch.full((dw.numel() + 1,), 0.5, dtype=torch.float32, device="cuda:0")
    dw_odd = store[1:].view(dw.shape)
    assert L.fdc_conv3d_backward_weights(C.byref(g), ptr(xt), ptr(dyt), ptr(dw_odd), None, None) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(dw_odd.cpu().numpy() - 0.5, rdw, rtol=0, atol=2e-5 * np.abs(rdw).max())
    assert float(store[0]) == 0.5


def test_transpose_weights_batch_equals_single_calls():
    """fdc_conv3d_transpose_weights_batch gives, layer by layer, the same
    bytes as fdc_conv3d_transpose_weights (3^3 reflected, 2^3 and 1^3 plain)."""
    import torch
    from paper_1011_2188_gb300 import fdc
    from paper_1011_2188_gb300.denoise import Conv3d
    L = fdc.lib()
    rng = np.random.default_rng(12)
    shapes = [(16, 16, 3, 1, 1), (32, 64, 3, 1, 1), (16, 32, 2, 2, 0), (64, 128, 2, 2, 0), (16, 16, 1, 1, 0)] * 8
    gs, ws, wts, refs = [], [], [], []
    for ci, co, k, st, pd in shapes:  # 40 layers: two launches of up to 32
        g, _ = geom((1, 8, 8, 8, ci), co, k, st, pd)
        wt_, _ = bf16(rng.normal(size=(co, k, k, k, ci)))
        out = torch.full((ci, k, k, k, co), 7.0, dtype=torch.bfloat16, device="cuda:0")
        ref = torch.empty_like(out)
        assert L.fdc_conv3d_transpose_weights(C.byref(g), ptr(wt_), ptr(ref), None) == 0
        gs.append(g); ws.append(wt_); wts.append(out); refs.append(ref)
    n = len(gs)
    garr = (Conv3d * n)(*gs)
    warr = (C.c_void_p * n)(*[t.data_ptr() for t in ws])
    tarr = (C.c_void_p * n)(*[t.data_ptr() for t in wts])
    assert L.fdc_conv3d_transpose_weights_batch(n, garr, warr, tarr, None) == 0
    torch.cuda.synchronize()
    for a, b in zip(wts, refs):
        assert torch.equal(a, b)
    assert L.fdc_conv3d_transpose_weights_batch(-1, garr, warr, tarr, None) != 0
    assert L.fdc_conv3d_transpose_weights_batch(0, None, None, None, None) == 0


def test_elementwise_kernels():
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    rng = np.random.default_rng(3)
    xt, x = bf16(rng.normal(size=(1, 3, 2, 4, 16)))
    up = torch.empty((1, 6, 4, 8, 16), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_upsample2(ptr(xt), ptr(up), 1, 3, 2, 4, 16, 0, None) == 0
    dyt, dy = bf16(rng.normal(size=(1, 6, 4, 8, 16)))
    back = torch.empty((1, 3, 2, 4, 16), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_upsample2(ptr(dyt), ptr(back), 1, 3, 2, 4, 16, 1, None) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(up.double().cpu().numpy(), ref.upsample2(x))
    np.testing.assert_allclose(back.double().cpu().numpy(), ref.upsample2_adjoint(dy), rtol=8e-3, atol=1e-2)
    # concat / split round trip, add, relu backward
    at, a = bf16(rng.normal(size=(10, 16)))
    bt, b = bf16(rng.normal(size=(10, 32)))
    out = torch.empty((10, 48), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_concat_channels(ptr(at), 16, ptr(bt), 32, ptr(out), 10, 0, None) == 0
    a2, b2 = torch.empty_like(at), torch.empty_like(bt)
    assert L.fdc_concat_channels(ptr(a2), 16, ptr(b2), 32, ptr(out), 10, 1, None) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.double().cpu().numpy(), np.concatenate([a, b], axis=1))
    assert torch.equal(a2, at) and torch.equal(b2, bt)
    s = torch.empty_like(at)
    assert L.fdc_add_bf16(ptr(at), ptr(a2), ptr(s), at.numel(), None) == 0
    dx = torch.empty_like(at)
    assert L.fdc_relu_backward(ptr(at), ptr(a2), ptr(dx), at.numel(), None) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(s.double().cpu().numpy(), 2 * a, rtol=8e-3)
    np.testing.assert_array_equal(dx.double().cpu().numpy(), np.where(a > 0, a, 0.0))


def test_tensor_core_status_clean():
    """No tensor-core convolution gave up waiting for its accumulator in the
    convolutions above (the status is sticky until cleared)."""
    from paper_1011_2188_gb300 import fdc
    assert fdc.lib().fdc_unet_status(1) == 0


def test_tensor_core_wait_timeout_is_reported():
    """The bounded-wait path: a barrier that nothing completes times out, the
    status reads FDC_ERR_TIMEOUT, clearing resets it, and the context stays
    usable (a convolution afterwards still succeeds)."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    L.fdc_unet_status(1)
    assert L.fdc_debug_wait_timeout(0, None) != 0
    assert L.fdc_debug_wait_timeout(2_000_000, None) == 0
    torch.cuda.synchronize()
    assert L.fdc_unet_status(1) == 7
    assert L.fdc_unet_status(0) == 0
    xt, _ = bf16(np.ones((1, 4, 8, 14, 16)))
    wt, _ = bf16(np.zeros((16, 3, 3, 3, 16)))
    g, oshape = geom((1, 4, 8, 14, 16), 16, 3, 1, 1)
    y = torch.empty(oshape, dtype=torch.float32, device="cuda:0")
    assert L.fdc_conv3d_forward(C.byref(g), ptr(xt), ptr(wt), None, None, ptr(y), None) == 0
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0 and L.fdc_unet_status(1) == 0


@pytest.mark.parametrize("code", range(8))
def test_dihedral_augmentation(code):
    """Mirror x (bit 0), mirror y (bit 1), exchange x and y first (bit 2),
    against numpy's own array operations; byte-exact."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    rng = np.random.default_rng(10 + code)
    D, H, W = 3, 6, 6
    xt, x = bf16(rng.normal(size=(1, D, H, W, 16)))
    t = rng.normal(size=(D, H, W)).astype(np.float32)
    tt = torch.from_numpy(t).cuda()
    xo, to = torch.empty_like(xt), torch.empty_like(tt)
    assert L.fdc_unet_dihedral(ptr(xt), ptr(tt), D, H, W, code, ptr(xo), ptr(to), None) == 0
    torch.cuda.synchronize()
    # out[z][y][x] = in[z][y'][x']: (y', x') = (x, y) when exchanged, then
    # x' -> W-1-x' (bit 0) and y' -> H-1-y' (bit 1)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    ys, xs = (xx, yy) if code & 4 else (yy, xx)
    if code & 1:
        xs = W - 1 - xs
    if code & 2:
        ys = H - 1 - ys
    ex, et = x[0][:, ys, xs], t[:, ys, xs]
    np.testing.assert_array_equal(xo.double().cpu().numpy()[0], ex)
    np.testing.assert_array_equal(to.cpu().numpy(), et)
    # refused: exchange on a non-square slice, aliasing, bad code
    assert L.fdc_unet_dihedral(ptr(xt), ptr(tt), D, H, W + 1, 4, ptr(xo), ptr(to), None) != 0
    assert L.fdc_unet_dihedral(ptr(xt), ptr(tt), D, H, W, 1, ptr(xt), ptr(to), None) != 0
    assert L.fdc_unet_dihedral(ptr(xt), ptr(tt), D, H, W, 8, ptr(xo), ptr(to), None) != 0


def test_mse_and_adam():
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    rng = np.random.default_rng(4)
    pred = rng.normal(size=(1000, 16)).astype(np.float32)
    tgt = rng.normal(size=1000).astype(np.float32)
    pt, tt = torch.from_numpy(pred).cuda(), torch.from_numpy(tgt).cuda()
    grad = torch.empty((1000, 16), dtype=torch.bfloat16, device="cuda:0")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    assert L.fdc_mse(ptr(pt), 16, ptr(tt), 1000, ptr(grad), ptr(loss), None) == 0
    torch.cuda.synchronize()
    e = pred[:, 0].astype(np.float64) - tgt
    assert float(loss) == pytest.approx(np.mean(e ** 2), rel=1e-5)
    g = grad.double().cpu().numpy()
    np.testing.assert_allclose(g[:, 0], 2 * e / 1000, rtol=8e-3, atol=1e-9)
    assert np.all(g[:, 1:] == 0)
    # Adam, two steps, against the textbook update
    p = rng.normal(size=100).astype(np.float32)
    gr = [rng.normal(size=100).astype(np.float32) for _ in range(2)]
    tp = torch.from_numpy(p.copy()).cuda()
    m = torch.zeros_like(tp)
    v = torch.zeros_like(tp)
    pb = torch.empty(100, dtype=torch.bfloat16, device="cuda:0")
    pr, mr, vr = p.astype(np.float64), np.zeros(100), np.zeros(100)
    for t, gg in enumerate(gr, start=1):
        tg = torch.from_numpy(gg).cuda()
        assert L.fdc_adam(ptr(tp), ptr(tg), ptr(m), ptr(v), ptr(pb), 100, 1e-3, 0.9, 0.999, 1e-8, t, None) == 0
        mr = 0.9 * mr + 0.1 * gg
        vr = 0.999 * vr + 0.001 * gg.astype(np.float64) ** 2
        pr = pr - 1e-3 * (mr / (1 - 0.9 ** t)) / (np.sqrt(vr / (1 - 0.999 ** t)) + 1e-8)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tp.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(pb.double().cpu().numpy(), pr, rtol=8e-3, atol=1e-6)


@pytest.mark.parametrize("n", [1, 255, 5000 + 37, 300_000])
def test_head_and_head_loss(n):
    """The fused head (output channel 0 of the 1^3 convolution), its loss and
    gradients against FP64 sums of the same BF16 values; ragged voxel counts
    (one voxel, less than a block, several blocks with a ragged tail, more
    voxels than the loss kernel's threads)."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    rng = np.random.default_rng(n)
    xt, x = bf16(np.maximum(rng.normal(size=(n, 16)), 0.0))  # ReLU features: about half exact zeros
    w16, w = bf16(rng.normal(size=(16, 16)) / 4)  # the head's [16][16] weights; row 0 is used
    b = torch.tensor(rng.normal(size=16), dtype=torch.float32, device="cuda:0")
    tgt = rng.normal(size=n).astype(np.float32)
    din = rng.random(n).astype(np.float32)
    tt, dt = torch.from_numpy(tgt).cuda(), torch.from_numpy(din).cuda()
    y_ref = x @ w[0] + float(b[0])
    y = torch.empty(n, dtype=torch.float32, device="cuda:0")
    dose = torch.empty(n, dtype=torch.float64, device="cuda:0")
    assert L.fdc_unet_head(ptr(xt), 16, ptr(w16), ptr(b), n, ptr(dt), 2.5, ptr(y), ptr(dose), None) == 0
    torch.cuda.synchronize()
    mag = np.abs(x) @ np.abs(w[0]) + abs(float(b[0]))
    assert np.all(np.abs(y.double().cpu().numpy() - y_ref) <= 2e-6 * mag + 1e-30)
    d_ref = np.maximum((y.double().cpu().numpy() + din) * 2.5, 0.0)  # FP64 epilogue of the FP32 correction
    np.testing.assert_allclose(dose.cpu().numpy(), d_ref, rtol=1e-15, atol=0)
    # loss and gradients
    loss = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    dx = torch.empty((n, 16), dtype=torch.bfloat16, device="cuda:0")
    dw = torch.full((16,), 0.5, dtype=torch.float32, device="cuda:0")  # accumulated into
    db = torch.full((1,), -0.25, dtype=torch.float32, device="cuda:0")
    assert L.fdc_unet_head_loss(ptr(xt), 16, ptr(w16), ptr(b), ptr(tt), n, ptr(loss), ptr(dx), ptr(dw), ptr(db),
                                None) == 0
    torch.cuda.synchronize()
    e = y_ref - tgt
    assert float(loss) == pytest.approx(np.mean(e ** 2), rel=1e-4)
    g = 2 * e / n
    dx_ref = np.where(x > 0, w[0][None, :] * g[:, None], 0.0)
    got = dx.double().cpu().numpy()
    np.testing.assert_allclose(got, dx_ref, rtol=8e-3, atol=1e-3 * np.abs(dx_ref).max() / 64)
    assert np.all(got[x == 0] == 0)
    scale_w = (np.abs(g)[:, None] * x).sum(0)
    assert np.all(np.abs(dw.double().cpu().numpy() - 0.5 - x.T @ g) <= 1e-4 * scale_w + 1e-7)
    assert abs(float(db[0]) + 0.25 - g.sum()) <= 1e-4 * np.abs(g).sum() + 1e-7
    # loss only (no gradients), accumulated onto the previous value
    assert L.fdc_unet_head_loss(ptr(xt), 16, ptr(w16), ptr(b), ptr(tt), n, ptr(loss), None, None, None, None) == 0
    torch.cuda.synchronize()
    assert float(loss) == pytest.approx(2 * np.mean(e ** 2), rel=1e-4)
    # refused: 8 channels, no output, dx aliasing x, only one of dw and db
    assert L.fdc_unet_head(ptr(xt), 8, ptr(w16), ptr(b), n, None, 0.0, ptr(y), None, None) != 0
    assert L.fdc_unet_head(ptr(xt), 16, ptr(w16), ptr(b), n, None, 0.0, None, None, None) != 0
    assert L.fdc_unet_head_loss(ptr(xt), 16, ptr(w16), ptr(b), ptr(tt), n, ptr(loss), ptr(xt), None, None,
                                None) != 0
    assert L.fdc_unet_head_loss(ptr(xt), 16, ptr(w16), ptr(b), ptr(tt), n, ptr(loss), None, ptr(dw), None,
                                None) != 0


def test_head_matches_convolution_and_mse():
    """The fused head equals channel 0 of the general 1^3 convolution with
    FP32 output, and its loss and gradients equal fdc_mse followed by that
    convolution's weight and data gradients."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    rng = np.random.default_rng(77)
    shape = (1, 6, 9, 10, 16)
    n = 6 * 9 * 10
    xt, x = bf16(np.maximum(rng.normal(size=shape), 0.0))
    w16, w = bf16(rng.normal(size=(16, 1, 1, 1, 16)) / 4)
    b = torch.tensor(rng.normal(size=16), dtype=torch.float32, device="cuda:0")
    g, oshape = geom(shape, 16, 1, 1, 0, 0)
    yc = torch.empty(oshape, dtype=torch.float32, device="cuda:0")
    assert L.fdc_conv3d_forward(C.byref(g), ptr(xt), ptr(w16), ptr(b), None, ptr(yc), None) == 0
    y = torch.empty(n, dtype=torch.float32, device="cuda:0")
    assert L.fdc_unet_head(ptr(xt), 16, ptr(w16), ptr(b), n, None, 0.0, ptr(y), None, None) == 0
    tt = torch.from_numpy(rng.normal(size=n).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    c0 = yc.reshape(n, 16)[:, 0]
    assert torch.allclose(y, c0, rtol=0, atol=2e-6 * float(c0.abs().max()))
    # the unfused chain: mse on channel 0, then the convolution's gradients
    loss_a = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    dy = torch.empty(oshape, dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_mse(ptr(yc), 16, ptr(tt), n, ptr(dy), ptr(loss_a), None) == 0
    dw_a = torch.zeros((16, 1, 1, 1, 16), dtype=torch.float32, device="cuda:0")
    db_a = torch.zeros(16, dtype=torch.float32, device="cuda:0")
    assert L.fdc_conv3d_backward_weights(C.byref(g), ptr(xt), ptr(dy), ptr(dw_a), ptr(db_a), None) == 0
    wt = torch.empty_like(w16)
    assert L.fdc_conv3d_transpose_weights(C.byref(g), ptr(w16), ptr(wt), None) == 0
    dx_a = torch.empty(shape, dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_backward_data(C.byref(g), ptr(dy), ptr(wt), ptr(xt), ptr(dx_a), None) == 0
    loss_b = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    dx_b = torch.empty(shape, dtype=torch.bfloat16, device="cuda:0")
    dw_b = torch.zeros(16, dtype=torch.float32, device="cuda:0")
    db_b = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    assert L.fdc_unet_head_loss(ptr(xt), 16, ptr(w16), ptr(b), ptr(tt), n, ptr(loss_b), ptr(dx_b), ptr(dw_b),
                                ptr(db_b), None) == 0
    torch.cuda.synchronize()
    assert float(loss_b) == pytest.approx(float(loss_a), rel=1e-5)
    # the unfused chain rounds the loss gradient to BF16 first: one BF16 rounding apart
    assert torch.allclose(dx_b.float(), dx_a.float(), rtol=1e-2, atol=1e-3 * float(dx_a.float().abs().max()))
    assert torch.allclose(dw_b, dw_a.reshape(16, 16)[0], rtol=1e-2, atol=1e-3 * float(dw_a.abs().max()))
    assert float(db_b[0]) == pytest.approx(float(db_a[0]), rel=1e-2, abs=1e-3 * float(db_a.abs().max()))
    assert float(db_a[1:].abs().max()) == 0.0 and float(dw_a[1:].abs().max()) == 0.0


def test_gamma_matches_oracle():
    import torch
    from paper_1011_2188_gb300 import denoise
    rng = np.random.default_rng(5)
    z = np.linspace(0, 1, 20)[:, None, None]
    r = np.exp(-((z - 0.6) / 0.2) ** 2) * np.ones((20, 18, 16)) + 0.05 * rng.random((20, 18, 16))
    e = r * (1 + 0.03 * rng.normal(size=r.shape))
    sp = (0.2, 0.2, 0.2)
    gout = torch.empty(r.shape, dtype=torch.float32, device="cuda:0")
    rate = denoise.gamma_pass_rate(torch.from_numpy(r).cuda(), torch.from_numpy(e).cuda(), sp, gamma_out=gout)
    g_ref, rate_ref = gref.gamma(r, e, sp)
    np.testing.assert_allclose(gout.cpu().numpy(), g_ref, rtol=1e-5, atol=1e-6)
    assert rate == pytest.approx(rate_ref, abs=1e-12)


def test_unet_forward_backward_and_training_reduces_loss():
    """A small U-Net on a 32^3 toy problem: the loss decreases under the
    project's forward, backward and Adam kernels."""
    import torch
    from paper_1011_2188_gb300 import denoise
    rng = np.random.default_rng(6)
    n = 32
    zz, yy, xx = np.meshgrid(*[np.linspace(-1, 1, n)] * 3, indexing="ij")
    clean = np.exp(-(xx ** 2 + yy ** 2) / 0.2) * (1 + zz)
    noisy = clean + 0.2 * rng.normal(size=clean.shape) * clean.max() / 3
    dens = np.ones_like(clean, dtype=np.float32)
    s = denoise.Sample(torch.from_numpy(noisy).cuda(), torch.from_numpy(dens).cuda(),
                       torch.from_numpy(clean).cuda())
    net = denoise.UNet(channels=(16, 32, 32, 64), seed=1)
    l0 = float(denoise.evaluate_loss(net, s))
    for _ in range(150):  # weight gradients sum with FP32 atomics: the trajectory varies slightly run to run
        denoise.train_step(net, s, 2e-3)
    l1 = float(denoise.evaluate_loss(net, s))
    assert np.isfinite(l1) and l1 < 0.6 * l0, (l0, l1)
    out = denoise.denoise(net, s)
    assert out.shape == (n, n, n) and bool(torch.isfinite(out).all())


@pytest.mark.parametrize("ca,cb,up,dims", [(32, 0, 1, (6, 8, 10)), (16, 16, 0, (6, 8, 10)), (64, 64, 0, (6, 8, 10)),
                                           (32, 32, 1, (6, 8, 10)), (16, 16, 0, (5, 12, 20)),
                                           (32, 32, 0, (7, 10, 34)), (32, 16, 0, (4, 11, 16)),
                                           (16, 16, 0, (6, 12, 36)), (16, 16, 0, (96, 40, 62)),
                                           (64, 64, 0, (8, 20, 34))])
def test_fused_upsample_concat_forward(ca, cb, up, dims):
    """fdc_conv3d_forward_fused equals fdc_conv3d_forward on the materialised
    [upsample(xa) | xb] input (the larger grids take the two tensor maps of
    the TMA d-walking kernel)."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    rng = np.random.default_rng(ca + cb + up + sum(dims))
    D, H, W = dims
    sa = (1, D // 2, H // 2, W // 2, ca) if up else (1, D, H, W, ca)
    xat, xa = bf16(rng.normal(size=sa))
    xbt, xb = bf16(rng.normal(size=(1, D, H, W, cb))) if cb else (None, None)
    cin, cout = ca + cb, 32
    wt, w = bf16(rng.normal(size=(cout, 3, 3, 3, cin)) / np.sqrt(27 * cin))
    g, oshape = geom((1, D, H, W, cin), cout, 3, 1, 1, 1)
    y = torch.empty(oshape, dtype=torch.float32, device="cuda:0")
    assert L.fdc_conv3d_forward_fused(C.byref(g), ptr(xat), ca, up, ptr(xbt), ptr(wt), None, None, ptr(y), None) == 0
    torch.cuda.synchronize()
    full = ref.upsample2(xa) if up else xa
    if cb:
        full = np.concatenate([full, xb], axis=-1)
    r = ref.forward(full, w, None, relu=True)
    np.testing.assert_allclose(y.cpu().numpy(), r, rtol=0, atol=2e-5 * np.abs(r).max())


def test_unet_inference_matches_training_forward():
    """The fused inference path gives the same output as the training path."""
    import torch
    from paper_1011_2188_gb300 import denoise
    rng = np.random.default_rng(9)
    n = 32
    dose = torch.from_numpy(rng.random((n, n, n))).cuda()
    dens = torch.ones((n, n, n), dtype=torch.float32, device="cuda:0")
    s = denoise.Sample(dose, dens, dose)
    net = denoise.UNet(seed=2)
    a = net.forward(s.x, keep=True).clone()
    for l in net.layers():
        l.x = l.y = None
    b = net.forward(s.x, keep=False)
    torch.cuda.synchronize()
    assert torch.allclose(a, b, rtol=0, atol=1e-3 * float(a.abs().max()))


def test_inference_graph_replays_the_same_dose():
    """InferenceGraph (one captured CUDA graph) gives the denoise() result bit
    for bit, also after the sample's buffers are refilled in place."""
    import torch
    from paper_1011_2188_gb300 import denoise, fdc
    rng = np.random.default_rng(13)
    n = 32
    dens = torch.ones((n, n, n), dtype=torch.float32, device="cuda:0")
    s = denoise.Sample(torch.from_numpy(rng.random((n, n, n))).cuda(), dens)
    net = denoise.UNet(seed=3)
    ig = denoise.InferenceGraph(net, s)
    for k in range(2):  # new doses, same scale (the graph keeps the one it was captured with)
        dose = torch.from_numpy(rng.random((n, n, n)) * (k + 1)).cuda()
        assert fdc.lib().fdc_unet_prepare(denoise._p(dose), denoise._p(dens), None, n ** 3, s.scale, 0.5,
                                          denoise._p(s.x), denoise._p(s.dose_in), None, denoise._s()) == 0
        a = ig.run().clone()
        b = denoise.denoise(net, s)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_denoised_path_graph_equals_denoise():
    """DenoisedPath (dose scale on the device, one CUDA graph from the scale to
    the denoised dose) gives denoise(net, Sample(dose, density)) bit for bit,
    for several doses refilled in place (different scales), and the
    device-scale calls refuse bad arguments."""
    import torch
    from paper_1011_2188_gb300 import denoise, fdc
    rng = np.random.default_rng(17)
    n = 32
    net = denoise.UNet(seed=4)
    path = denoise.DenoisedPath(net, (n, n, n))
    dens = torch.from_numpy(rng.uniform(0.2, 1.9, (n, n, n)).astype(np.float32)).cuda()
    path.set_density(dens)
    for k in range(3):
        dose = torch.from_numpy(rng.random((n, n, n)) * 10.0 ** (k - 1)).cuda()
        path.dose.copy_(dose)
        a = path.denoise().clone()
        b = denoise.denoise(net, denoise.Sample(dose, dens))
        torch.cuda.synchronize()
        assert float(path.scale) == float(dose.max())
        assert torch.equal(a, b)
    L = fdc.lib()
    assert L.fdc_unet_dose_scale(None, 8, ptr(path.scale), None) == 1
    assert L.fdc_unet_prepare_dev(ptr(path.dose), ptr(dens), n ** 3, None, 0.5, ptr(path.x), ptr(path.dose_in),
                                  None) == 1
    assert L.fdc_unet_head_dev(ptr(path.x), 8, ptr(net.head.w16), ptr(net.head.b32), n ** 3, ptr(path.dose_in),
                               ptr(path.scale), ptr(path.dose), None) == 1


@pytest.mark.parametrize("ca,cb,up,cout,dims", [(32, 0, 1, 16, (6, 10, 18)), (16, 16, 0, 16, (6, 10, 18)),
                                                (32, 32, 0, 32, (6, 10, 18)), (64, 0, 1, 32, (6, 10, 18)),
                                                (16, 16, 0, 16, (6, 10, 34)), (32, 0, 1, 16, (4, 12, 64))])
def test_fused_backward_equals_materialised(ca, cb, up, cout, dims):
    """The gradients of the fused forward (input [upsample?(xa) | xb] never
    materialised): the data gradient with the ReLU mask of that input, split
    by channel, equals fdc_conv3d_backward_data on the materialised input bit
    for bit; the weight and bias gradients agree with
    fdc_conv3d_backward_weights to FP32 accumulation order."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    rng = np.random.default_rng(ca + 3 * cb + up + cout + sum(dims))
    D, H, W = dims
    sa = (1, D // 2, H // 2, W // 2, ca) if up else (1, D, H, W, ca)
    xat, _ = bf16(np.maximum(rng.normal(size=sa), 0) * (rng.random(sa) < 0.8))  # ReLU outputs with zeros
    xbt = bf16(np.maximum(rng.normal(size=(1, D, H, W, cb)), 0))[0] if cb else None
    cin = ca + cb
    wt, _ = bf16(rng.normal(size=(cout, 3, 3, 3, cin)) / np.sqrt(27 * cin))
    g, oshape = geom((1, D, H, W, cin), cout, 3, 1, 1, 1)
    dyt, _ = bf16(rng.normal(size=oshape))
    full = torch.empty((1, D, H, W, cin), dtype=torch.bfloat16, device="cuda:0")
    xa_full = xat
    if up:
        xa_full = torch.empty((1, D, H, W, ca), dtype=torch.bfloat16, device="cuda:0")
        assert L.fdc_upsample2(ptr(xat), ptr(xa_full), 1, D // 2, H // 2, W // 2, ca, 0, None) == 0
    if cb:
        assert L.fdc_concat_channels(ptr(xa_full), ca, ptr(xbt), cb, ptr(full), D * H * W, 0, None) == 0
    else:
        full.copy_(xa_full)
    w_t = torch.empty((cin, 3, 3, 3, cout), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_transpose_weights(C.byref(g), ptr(wt), ptr(w_t), None) == 0
    dx = torch.empty((1, D, H, W, cin), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_backward_data(C.byref(g), ptr(dyt), ptr(w_t), ptr(full), ptr(dx), None) == 0
    dxa = torch.empty((1, D, H, W, ca), dtype=torch.bfloat16, device="cuda:0")
    dxb = torch.empty((1, D, H, W, cb), dtype=torch.bfloat16, device="cuda:0") if cb else None
    assert L.fdc_conv3d_backward_data_fused(C.byref(g), ptr(dyt), ptr(w_t), ptr(xat), ca, up, ptr(xbt), ptr(dxa),
                                            ptr(dxb), None) == 0
    dw = torch.zeros((cout, 3, 3, 3, cin), dtype=torch.float32, device="cuda:0")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda:0")
    assert L.fdc_conv3d_backward_weights(C.byref(g), ptr(full), ptr(dyt), ptr(dw), ptr(db), None) == 0
    dwf, dbf = torch.zeros_like(dw), torch.zeros_like(db)
    assert L.fdc_conv3d_backward_weights_fused(C.byref(g), ptr(xat), ca, up, ptr(xbt), ptr(dyt), ptr(dwf), ptr(dbf),
                                               None) == 0
    torch.cuda.synchronize()
    assert torch.equal(dxa, dx[..., :ca])
    if cb:
        assert torch.equal(dxb, dx[..., ca:])
    torch.testing.assert_close(dwf, dw, rtol=0, atol=1e-5 * float(dw.abs().max()))
    torch.testing.assert_close(dbf, db, rtol=0, atol=1e-5 * float(db.abs().max()))
    # the fused data gradient needs the d-walking kernels (at most 32 output channels)
    g2, _ = geom((1, D, H, W, cin), 64, 3, 1, 1, 1)
    assert L.fdc_conv3d_backward_data_fused(C.byref(g2), ptr(dyt), ptr(w_t), ptr(xat), ca, up, ptr(xbt), ptr(dxa),
                                            ptr(dxb), None) == 1


def _collapse_up(w):
    """The collapsed weights of the sub-pixel upsampling convolution from
    their definition (FP64): along each axis, output parity p and coarse
    offset s in {0, 1} take the taps k with floor((p + k - 1) / 2) = p - 1 + s."""
    co, ci = w.shape[0], w.shape[-1]
    sets = {(p, s): [k for k in range(3) if (p + k - 1) // 2 == p - 1 + s] for p in (0, 1) for s in (0, 1)}
    out = np.zeros((co, 64, ci))
    for t in range(64):
        pd, ph, sd, sh, pw, sw = [(t >> b) & 1 for b in (5, 4, 3, 2, 1, 0)]
        for kd in sets[pd, sd]:
            for kh in sets[ph, sh]:
                for kw in sets[pw, sw]:
                    out[:, t, :] += w[:, kd, kh, kw, :]
    return out


@pytest.mark.parametrize("shape,cout", [((1, 8, 20, 32, 32), 16), ((1, 4, 20, 32, 16), 16),
                                        ((2, 12, 26, 40, 64), 32), ((1, 64, 48, 60, 32), 16),
                                        ((1, 8, 20, 32, 128), 64)])
@pytest.mark.parametrize("relu", [0, 1])
def test_forward_up_subpixel(shape, cout, relu):
    """fdc_conv3d_forward_up (the upsampling convolution on the coarse grid
    by output parity class, 8 collapsed taps per output) against the FP64
    convolution of the materialised upsample2(xa).  Its one extra rounding is
    each collapsed weight's (to BF16: relative 2^-8, the unit roundoff of an
    8-bit significand), so per output |y - ref| <= 2^-8 * sum |w| |x| + the
    FP32 accumulation term of the other convolution tests; the collapsed
    weights equal their FP64 definition within that rounding (after the FP32
    sum: 2^-8 + 2^-22 relative)."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    B, D, H, W, ci = shape  # the full-resolution grid
    rng = np.random.default_rng(sum(shape) + cout + relu)
    xat, xa = bf16(rng.normal(size=(B, D // 2, H // 2, W // 2, ci)))
    wt, w = bf16(rng.normal(size=(cout, 3, 3, 3, ci)) / np.sqrt(27 * ci))
    b = rng.normal(size=cout).astype(np.float32)
    bt = torch.from_numpy(b).cuda()
    g, oshape = geom(shape, cout, 3, 1, 1, relu)
    wup = torch.empty((cout, 64, ci), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_collapse_up_weights(C.byref(g), ptr(wt), ptr(wup), None) == 0
    y32 = torch.empty(oshape, dtype=torch.float32, device="cuda:0")
    y16 = torch.empty(oshape, dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_forward_up(C.byref(g), ptr(xat), ptr(wup), ptr(bt), ptr(y16), ptr(y32), None) == 0
    torch.cuda.synchronize()
    exact = _collapse_up(w)
    got = wup.double().cpu().numpy()
    assert np.all(np.abs(got - exact) <= (2.0 ** -8 + 2.0 ** -22) * np.abs(exact))
    up = ref.upsample2(xa)
    r = ref.forward(up, w, b.astype(np.float64), relu=bool(relu))
    bound = 2.0 ** -8 * ref.forward(np.abs(up), np.abs(w), None) + 2e-5 * np.abs(r).max()
    err = np.abs(y32.cpu().numpy() - r)
    assert np.all(err <= bound), float((err / bound).max())
    assert np.all(np.abs(y16.double().cpu().numpy() - r) <= bound + 2.0 ** -8 * np.abs(r))


def test_forward_up_refuses_shapes_without_its_kernel():
    """FDC_ERR_INVALID, nothing launched: a coarse grid narrower than the TMA
    box (16 w), odd sizes, more than 64 input channels that do not split into
    16-channel parts of at most 32."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    x = torch.zeros((1, 8, 16, 32, 128), dtype=torch.bfloat16, device="cuda:0")
    wup = torch.zeros((16, 64, 128), dtype=torch.bfloat16, device="cuda:0")
    y = torch.empty((1, 16, 32, 64, 16), dtype=torch.bfloat16, device="cuda:0")
    for shape in [(1, 6, 20, 30, 16), (1, 7, 20, 32, 16), (1, 16, 32, 64, 80)]:
        g, _ = geom(shape, 16, 3, 1, 1)
        assert L.fdc_conv3d_forward_up(C.byref(g), ptr(x), ptr(wup), None, ptr(y), None, None) == 1
    torch.cuda.synchronize()


def _collapse_up_t(w):
    """Transposed collapsed weights of the coarse data gradient from their
    definition (FP64): [ci][t][co], t = (q_d, q_h, q_w, i_d, i_h, i_w), the
    forward collapse of output parity q and coarse offset s = 1 - i."""
    fw = _collapse_up(w)  # [co][(pd ph)(sd sh)(pw sw)][ci]
    co, ci = w.shape[0], w.shape[-1]
    out = np.zeros((ci, 64, co))
    for t in range(64):
        qd, qh, qw, idd, idh, idw = [(t >> b) & 1 for b in (5, 4, 3, 2, 1, 0)]
        tf = ((qd * 2 + qh) * 4 + (1 - idd) * 2 + (1 - idh)) * 4 + qw * 2 + (1 - idw)
        out[:, t, :] = fw[:, tf, :].T
    return out


@pytest.mark.parametrize("full,cin,cout", [((1, 8, 20, 32), 32, 16), ((1, 6, 20, 34), 16, 16),
                                           ((2, 8, 24, 40), 64, 32), ((1, 4, 20, 32), 128, 64),
                                           ((1, 64, 40, 64), 32, 16)])
def test_backward_data_up_coarse(full, cin, cout):
    """fdc_conv3d_backward_data_up (the data gradient of the sub-pixel
    up-convolution, on the coarse grid) against the FP64 adjoint of the direct
    form: upsample2-adjoint of the full-resolution data gradient, masked where
    xa is not positive.  Bound: the collapsed weights' BF16 rounding (2^-8 of
    the same sums with |w| and |dy|), FP32 accumulation and the output's BF16
    rounding; the transposed collapsed weights within one BF16 rounding of
    their definition."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    B, D, H, W = full
    rng = np.random.default_rng(B + D + H + W + cin + cout)
    coarse = (B, D // 2, H // 2, W // 2, cin)
    xat, xa = bf16(np.maximum(rng.normal(size=coarse), 0) * (rng.random(coarse) < 0.8))
    wt, w = bf16(rng.normal(size=(cout, 3, 3, 3, cin)) / np.sqrt(27 * cin))
    dyt, dy = bf16(rng.normal(size=(B, D, H, W, cout)))
    g, _ = geom((B, D, H, W, cin), cout, 3, 1, 1)
    wupt = torch.empty((cin, 64, cout), dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_collapse_up_weights_t(C.byref(g), ptr(wt), ptr(wupt), None) == 0
    dxa = torch.full(coarse, 7.0, dtype=torch.bfloat16, device="cuda:0")
    assert L.fdc_conv3d_backward_data_up(C.byref(g), ptr(dyt), ptr(wupt), ptr(xat), ptr(dxa), None) == 0
    torch.cuda.synchronize()
    exact = _collapse_up_t(w)
    assert np.all(np.abs(wupt.double().cpu().numpy() - exact) <= (2.0 ** -8 + 2.0 ** -22) * np.abs(exact))
    shape = (B, D, H, W, cin)
    r = ref.upsample2_adjoint(ref.backward_data(dy, w, shape))
    r = np.where(xa > 0, r, 0.0)
    bound = 2.0 ** -8 * ref.upsample2_adjoint(ref.backward_data(np.abs(dy), np.abs(w), shape)) + \
        2e-5 * np.abs(r).max() + 2.0 ** -8 * np.abs(r)
    err = np.abs(dxa.double().cpu().numpy() - r)
    assert np.all(err <= bound), float((err / bound).max())


def test_backward_data_up_refuses_shapes_without_its_kernel():
    """FDC_ERR_INVALID, nothing launched: a full-resolution grid narrower than
    32 columns, odd sizes."""
    import torch
    from paper_1011_2188_gb300 import fdc
    L = fdc.lib()
    dy = torch.zeros((1, 8, 20, 32, 16), dtype=torch.bfloat16, device="cuda:0")
    wupt = torch.zeros((16, 64, 16), dtype=torch.bfloat16, device="cuda:0")
    dxa = torch.zeros((1, 4, 10, 16, 16), dtype=torch.bfloat16, device="cuda:0")
    for shape in [(1, 8, 20, 30, 16), (1, 7, 20, 32, 16)]:
        g, _ = geom(shape, 16, 3, 1, 1)
        assert L.fdc_conv3d_backward_data_up(C.byref(g), ptr(dy), ptr(wupt), None, ptr(dxa), None) == 1
    torch.cuda.synchronize()
