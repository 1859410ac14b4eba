"""Learned denoiser: a 3-D U-Net from a low-history dose (plus density) to a
high-history dose, trained and run with the library's own kernels
(include/fdc_unet.h).  Not part of the paper: the track-repeating engine
generates its training pairs and remains both the fallback and the reference
its error is measured against.

Network (channels-last BF16 activations, FP32 master weights):
  level 1 (full grid, 16 ch): 2 x conv3 -> skip s1
  down (conv 2^3, stride 2) to 32 ch, 2 x conv3 -> s2; to 64 ch -> s3; to 128 ch
  bottleneck: 2 x conv3 (128)
  up: nearest x2, conv3 to half the channels, concatenate the skip, 2 x conv3
  head: conv 1^3 to 16 ch; channel 0 is the correction added to the input dose
  (the only channel computed: a fused kernel takes it, the loss and its
  gradients straight from the last decoder layer's output).
All convolutions but the head apply ReLU.  Loss: mean squared error of the
corrected dose against the high-history dose (both divided by the input
dose's maximum).  Optimiser: Adam.

Torch provides device memory and the stream only; every arithmetic step is a
library kernel.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import fdc


class Conv3d(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("batch", "in_d", "in_h", "in_w", "out_d", "out_h", "out_w", "c_in",
                                           "c_out", "ksize", "stride", "pad", "relu")]


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _s(stream=None):
    import torch
    return C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


def _ok(rc, what):
    if rc:
        raise fdc.FdcError(rc, what)


class ConvLayer:
    """One convolution with its parameters, gradients and Adam moments."""

    def __init__(self, cin, cout, k, stride, pad, relu, rng, device, cin_real=None, f32_out=False):
        import torch
        self.cin, self.cout, self.k, self.stride, self.pad, self.relu = cin, cout, k, stride, pad, relu
        self.f32_out = f32_out
        fan_in = k ** 3 * (cin_real or cin)
        w = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=(cout, k, k, k, cin)).astype(np.float32)
        if cin_real:
            w[..., cin_real:] = 0.0
        if f32_out:
            w *= 0.1
        self.dev = device
        self.w32 = torch.from_numpy(w).to(device)
        self.b32 = torch.zeros(cout, dtype=torch.float32, device=device)
        self.w16 = torch.empty(self.w32.shape, dtype=torch.bfloat16, device=device)
        self.wt16 = torch.empty((cin, k, k, k, cout), dtype=torch.bfloat16, device=device)
        self.gw = torch.zeros_like(self.w32)
        self.gb = torch.zeros_like(self.b32)
        self.mw, self.vw = torch.zeros_like(self.w32), torch.zeros_like(self.w32)
        self.mb, self.vb = torch.zeros_like(self.b32), torch.zeros_like(self.b32)
        self.sync_weights()

    def geom(self, shape):
        B, D, H, W, _ = shape
        o = [(n + 2 * self.pad - self.k) // self.stride + 1 for n in (D, H, W)]
        return Conv3d(B, D, H, W, o[0], o[1], o[2], self.cin, self.cout, self.k, self.stride, self.pad,
                      1 if self.relu else 0), (B, o[0], o[1], o[2], self.cout)

    def sync_weights(self):
        L = fdc.lib()
        n = self.w32.numel()
        _ok(L.fdc_f32_to_bf16(_p(self.w32), _p(self.w16), n, _s()), "f32_to_bf16")
        g, _ = self.geom((1, 8, 8, 8, self.cin))
        _ok(L.fdc_conv3d_transpose_weights(C.byref(g), _p(self.w16), _p(self.wt16), _s()), "transpose")
        self.collapse_up()

    def enable_up(self):
        """This layer convolves an upsampled input: keep the collapsed weights
        of the sub-pixel form (fdc_conv3d_forward_up) next to the others."""
        import torch
        self.wup16 = torch.empty((self.cout, 64, self.cin), dtype=torch.bfloat16, device=self.dev)
        self.wupt16 = torch.empty((self.cin, 64, self.cout), dtype=torch.bfloat16, device=self.dev)
        self.up_ok = None  # whether fdc_conv3d_forward_up takes this layer's shape (learned at first call)
        self.up_dgrad_ok = None  # the same for fdc_conv3d_backward_data_up
        self.collapse_up()

    def collapse_up(self):
        if getattr(self, "wup16", None) is not None:
            g, _ = self.geom((1, 8, 8, 8, self.cin))
            _ok(fdc.lib().fdc_conv3d_collapse_up_weights(C.byref(g), _p(self.w16), _p(self.wup16), _s()),
                "collapse up")
            _ok(fdc.lib().fdc_conv3d_collapse_up_weights_t(C.byref(g), _p(self.w16), _p(self.wupt16), _s()),
                "collapse up (data gradient)")

    def forward(self, x, keep=True):
        import torch
        g, oshape = self.geom(tuple(x.shape))
        if self.f32_out:
            y = torch.empty(oshape, dtype=torch.float32, device=self.dev)
            _ok(fdc.lib().fdc_conv3d_forward(C.byref(g), _p(x), _p(self.w16), _p(self.b32), None, _p(y), _s()),
                "conv forward")
        else:
            y = torch.empty(oshape, dtype=torch.bfloat16, device=self.dev)
            _ok(fdc.lib().fdc_conv3d_forward(C.byref(g), _p(x), _p(self.w16), _p(self.b32), _p(y), None, _s()),
                "conv forward")
        if keep:
            self.x, self.y = x, y
        return y

    def forward_up(self, xa, keep=False):
        """This 3^3 convolution of upsample2(xa): the sub-pixel kernel on xa's
        grid (collapsed weights, see fdc_conv3d_forward_up) where it takes the
        shape, else forward_fused; with keep, xa is kept for the gradients of
        the exact map (backward)."""
        import torch
        if self.up_ok is not False:
            B, D, H, W, ca = xa.shape
            g, oshape = self.geom((B, 2 * D, 2 * H, 2 * W, self.cin))
            y = torch.empty(oshape, dtype=torch.bfloat16, device=self.dev)
            rc = fdc.lib().fdc_conv3d_forward_up(C.byref(g), _p(xa), _p(self.wup16), _p(self.b32), _p(y), None, _s())
            if rc == 0:
                self.up_ok = True
                if keep:
                    self.x, self.y = None, y
                    self.fused_in = (xa, True, None, (B, 2 * D, 2 * H, 2 * W, self.cin))
                return y
            if rc != 1 or self.up_ok:  # only "no kernel for this shape" falls back
                _ok(rc, "conv forward up")
            self.up_ok = False
        return self.forward_fused(xa, upsample=True, keep=keep)

    def forward_fused(self, xa, upsample=False, xb=None, keep=False):
        """This 3^3 convolution applied to [upsample(xa) | xb] without
        materialising the upsampled or concatenated input; with keep, the two
        parts are kept for the fused gradients (backward)."""
        import torch
        B, D, H, W, ca = xa.shape
        if upsample:
            D, H, W = 2 * D, 2 * H, 2 * W
        g, oshape = self.geom((B, D, H, W, self.cin))
        y = torch.empty(oshape, dtype=torch.bfloat16, device=self.dev)
        _ok(fdc.lib().fdc_conv3d_forward_fused(C.byref(g), _p(xa), ca, 1 if upsample else 0, _p(xb),
                                               _p(self.w16), _p(self.b32), _p(y), None, _s()), "conv forward fused")
        if keep:
            self.x, self.y = None, y
            self.fused_in = (xa, bool(upsample), xb, (B, D, H, W, self.cin))
        return y

    def backward(self, dy, need_dx=True, residual=None):
        """dy: gradient with respect to this layer's pre-activation (its own
        ReLU derivative already applied: every layer's input is the output of
        a ReLU layer, and the data gradient below masks dx by x > 0 in its
        epilogue, which is that derivative for the layer before).  Returns
        the gradient with respect to the previous layer's pre-activation; after
        forward_fused(keep=True), the pair (d xa, d xb) for a concatenated input
        (d xa at full resolution when xa was upsampled), or d xa alone; an
        up-convolution with collapsed weights returns d xa on xa's own coarse
        grid where its kernel takes the shape (then self.dx_coarse is True)."""
        import torch
        L = fdc.lib()
        self.dx_coarse = False
        if getattr(self, "fused_in", None) is not None:
            xa, up, xb, shape = self.fused_in
            g, _ = self.geom(shape)
            ca = xa.shape[-1]
            _ok(L.fdc_conv3d_backward_weights_fused(C.byref(g), _p(xa), ca, 1 if up else 0, _p(xb), _p(dy),
                                                    _p(self.gw), _p(self.gb), _s()), "conv wgrad fused")
            out = None
            if need_dx and up and xb is None and getattr(self, "wupt16", None) is not None and \
                    self.up_dgrad_ok is not False:
                # the gradient of xa itself, on its coarse grid (no full-resolution gradient)
                dxa = torch.empty(xa.shape, dtype=torch.bfloat16, device=self.dev)
                rc = L.fdc_conv3d_backward_data_up(C.byref(g), _p(dy), _p(self.wupt16), _p(xa), _p(dxa), _s())
                if rc == 0:
                    self.up_dgrad_ok, self.dx_coarse = True, True
                    self.fused_in = None
                    self.y = None
                    return dxa
                if rc != 1 or self.up_dgrad_ok:
                    _ok(rc, "conv dgrad up")
                self.up_dgrad_ok = False
            if need_dx:
                dxa = torch.empty(shape[:4] + (ca,), dtype=torch.bfloat16, device=self.dev)
                dxb = (torch.empty(shape[:4] + (self.cin - ca,), dtype=torch.bfloat16, device=self.dev)
                       if xb is not None else None)
                _ok(L.fdc_conv3d_backward_data_fused(C.byref(g), _p(dy), _p(self.wt16), _p(xa), ca, 1 if up else 0,
                                                     _p(xb), _p(dxa), _p(dxb), _s()), "conv dgrad fused")
                out = (dxa, dxb) if xb is not None else dxa
            self.fused_in = None
            self.y = None
            return out
        g, _ = self.geom(tuple(self.x.shape))
        _ok(L.fdc_conv3d_backward_weights(C.byref(g), _p(self.x), _p(dy), _p(self.gw), _p(self.gb), _s()),
            "conv wgrad")
        dx = None
        if need_dx:
            dx = torch.empty(self.x.shape, dtype=torch.bfloat16, device=self.dev)
            if residual is not None:  # plus a second gradient of the same activation
                _ok(L.fdc_conv3d_backward_data_add(C.byref(g), _p(dy), _p(self.wt16), _p(self.x), _p(residual),
                                                   _p(dx), _s()), "conv dgrad + residual")
            else:
                _ok(L.fdc_conv3d_backward_data(C.byref(g), _p(dy), _p(self.wt16), _p(self.x), _p(dx), _s()),
                    "conv dgrad")
        self.x = self.y = None
        return dx

    def zero_grad(self):
        self.gw.zero_()
        self.gb.zero_()

    def step(self, lr, t, b1=0.9, b2=0.999, eps=1e-8):
        L = fdc.lib()
        _ok(L.fdc_adam(_p(self.w32), _p(self.gw), _p(self.mw), _p(self.vw), _p(self.w16), self.w32.numel(),
                       lr, b1, b2, eps, t, _s()), "adam")
        _ok(L.fdc_adam(_p(self.b32), _p(self.gb), _p(self.mb), _p(self.vb), None, self.b32.numel(),
                       lr, b1, b2, eps, t, _s()), "adam")
        g, _ = self.geom((1, 8, 8, 8, self.cin))
        _ok(L.fdc_conv3d_transpose_weights(C.byref(g), _p(self.w16), _p(self.wt16), _s()), "transpose")

    def state(self):
        return {"w": self.w32.cpu().numpy(), "b": self.b32.cpu().numpy()}

    def load(self, st):
        import torch
        self.w32.copy_(torch.from_numpy(st["w"]))
        self.b32.copy_(torch.from_numpy(st["b"]))
        self.sync_weights()


def _upsample(x, backward=False):
    import torch
    B, D, H, W, Cc = x.shape
    if backward:
        y = torch.empty((B, D // 2, H // 2, W // 2, Cc), dtype=x.dtype, device=x.device)
        _ok(fdc.lib().fdc_upsample2(_p(x), _p(y), B, D // 2, H // 2, W // 2, Cc, 1, _s()), "upsample bwd")
    else:
        y = torch.empty((B, 2 * D, 2 * H, 2 * W, Cc), dtype=x.dtype, device=x.device)
        _ok(fdc.lib().fdc_upsample2(_p(x), _p(y), B, D, H, W, Cc, 0, _s()), "upsample")
    return y


def _concat(a, b):
    import torch
    out = torch.empty(a.shape[:-1] + (a.shape[-1] + b.shape[-1],), dtype=a.dtype, device=a.device)
    rows = a.numel() // a.shape[-1]
    _ok(fdc.lib().fdc_concat_channels(_p(a), a.shape[-1], _p(b), b.shape[-1], _p(out), rows, 0, _s()), "concat")
    return out


def _split(out, ca, cb):
    import torch
    a = torch.empty(out.shape[:-1] + (ca,), dtype=out.dtype, device=out.device)
    b = torch.empty(out.shape[:-1] + (cb,), dtype=out.dtype, device=out.device)
    rows = out.numel() // out.shape[-1]
    _ok(fdc.lib().fdc_concat_channels(_p(a), ca, _p(b), cb, _p(out), rows, 1, _s()), "split")
    return a, b


def _add(a, b):
    _ok(fdc.lib().fdc_add_bf16(_p(a), _p(b), _p(a), a.numel(), _s()), "add")
    return a


class UNet:
    def __init__(self, channels=(16, 32, 64, 128), seed=0, device="cuda:0"):
        rng = np.random.default_rng(seed)
        c1, c2, c3, c4 = channels

        def L(cin, cout, k=3, s=1, p=1, relu=True, **kw):
            return ConvLayer(cin, cout, k, s, p, relu, rng, device, **kw)

        self.enc1 = [L(16, c1, cin_real=2), L(c1, c1)]
        self.down1 = L(c1, c2, 2, 2, 0)
        self.enc2 = [L(c2, c2), L(c2, c2)]
        self.down2 = L(c2, c3, 2, 2, 0)
        self.enc3 = [L(c3, c3), L(c3, c3)]
        self.down3 = L(c3, c4, 2, 2, 0)
        self.bott = [L(c4, c4), L(c4, c4)]
        self.up3 = L(c4, c3)
        self.dec3 = [L(2 * c3, c3), L(c3, c3)]
        self.up2 = L(c3, c2)
        self.dec2 = [L(2 * c2, c2), L(c2, c2)]
        self.up1 = L(c2, c1)
        self.dec1 = [L(2 * c1, c1), L(c1, c1)]
        self.head = L(c1, 16, 1, 1, 0, relu=False, f32_out=True)
        self.channels = channels
        self.t = 0
        self._flatten()
        for l in (self.up1, self.up2, self.up3):
            l.enable_up()

    def _flatten(self):
        """All layers' FP32 weights and biases, their gradients, Adam moments
        and BF16 copies become views of five flat buffers, so that one fill
        zeroes every gradient and one Adam launch updates every parameter.
        Every tensor holds a multiple of 16 elements, so each view starts on
        a 64-byte (FP32) / 32-byte (BF16) boundary."""
        import torch
        layers = self.layers()
        n = sum(l.w32.numel() + l.b32.numel() for l in layers)
        dev = layers[0].dev
        self.p32 = torch.empty(n, dtype=torch.float32, device=dev)
        self.g32 = torch.zeros(n, dtype=torch.float32, device=dev)
        self.m32 = torch.zeros(n, dtype=torch.float32, device=dev)
        self.v32 = torch.zeros(n, dtype=torch.float32, device=dev)
        self.p16 = torch.empty(n, dtype=torch.bfloat16, device=dev)
        o = 0
        for l in layers:
            for pn, gn, mn, vn in (("w32", "gw", "mw", "vw"), ("b32", "gb", "mb", "vb")):
                t = getattr(l, pn)
                k = t.numel()
                assert k % 16 == 0 and o % 16 == 0
                view = self.p32[o:o + k].view(t.shape)
                view.copy_(t)
                setattr(l, pn, view)
                setattr(l, gn, self.g32[o:o + k].view(t.shape))
                setattr(l, mn, self.m32[o:o + k].view(t.shape))
                setattr(l, vn, self.v32[o:o + k].view(t.shape))
                if pn == "w32":
                    l.w16 = self.p16[o:o + k].view(t.shape)
                o += k
        for l in layers:
            l.sync_weights()

    def layers(self):
        return (self.enc1 + [self.down1] + self.enc2 + [self.down2] + self.enc3 + [self.down3] + self.bott +
                [self.up3] + self.dec3 + [self.up2] + self.dec2 + [self.up1] + self.dec1 + [self.head])

    @staticmethod
    def _seq(layers, x, keep):
        for l in layers:
            x = l.forward(x, keep)
        return x

    def features(self, x, keep=True):
        """Output of the last decoder layer: the head's input, 16 BF16
        channels per voxel (keep: store what the backward pass needs)."""
        e1 = self._seq(self.enc1, x, keep)
        e2 = self._seq(self.enc2, self.down1.forward(e1, keep), keep)
        e3 = self._seq(self.enc3, self.down2.forward(e2, keep), keep)
        b = self._seq(self.bott, self.down3.forward(e3, keep), keep)
        if keep:  # training
            f3 = self._decoder_train(self.up3, self.dec3, b, e3)
            f2 = self._decoder_train(self.up2, self.dec2, f3, e2)
            f1 = self._decoder_train(self.up1, self.dec1, f2, e1)
        else:  # inference: upsampling and skip concatenation fused into the convolutions
            f = b
            for up, dec, skip in ((self.up3, self.dec3, e3), (self.up2, self.dec2, e2), (self.up1, self.dec1, e1)):
                u = up.forward_up(f)
                f = dec[1].forward(dec[0].forward_fused(u, xb=skip), False)
            f1 = f
        return f1

    def forward(self, x, keep=True):
        """Correction predicted for every voxel, FP32 [1, D, H, W]: output
        channel 0 of the 1^3 head (the other 15 feed neither the loss nor
        the dose, so they are not computed)."""
        import torch
        f1 = self.features(x, keep)
        y = torch.empty(f1.shape[:4], dtype=torch.float32, device=f1.device)
        _ok(fdc.lib().fdc_unet_head(_p(f1), f1.shape[-1], _p(self.head.w16), _p(self.head.b32), y.numel(), None,
                                    0.0, _p(y), None, _s()), "head")
        return y

    def head_loss(self, f1, target, loss, df1=None):
        """Adds the mean squared error of the head's correction against the
        target to loss; with df1, also the head's weight and bias gradients
        and, in df1, the gradient with respect to the last decoder layer's
        pre-activation."""
        grad = df1 is not None
        _ok(fdc.lib().fdc_unet_head_loss(_p(f1), f1.shape[-1], _p(self.head.w16), _p(self.head.b32), _p(target),
                                         target.numel(), _p(loss), _p(df1), _p(self.head.gw) if grad else None,
                                         _p(self.head.gb) if grad else None, _s()), "head loss")

    @staticmethod
    def _fuse_level(up):
        """Decoder levels whose up-convolution has at most 32 output channels
        (the 128^3 and 64^3 levels) train on the fused inputs: the fused data
        gradient runs on the d-walking convolution kernels, which need that."""
        return up.cout <= 32

    def _decoder_train(self, up, dec, f, skip):
        if self._fuse_level(up):  # upsampled and concatenated inputs are never materialised
            u = up.forward_up(f, keep=True)
            h = dec[0].forward_fused(u, xb=skip, keep=True)
        else:
            u = up.forward(_upsample(f), True)
            h = dec[0].forward(_concat(u, skip), True)
        return dec[1].forward(h, True)

    def _decoder_back(self, up, dec, d, c):
        """Gradient of one decoder level: returns (d f, d skip)."""
        d = dec[1].backward(d)
        if self._fuse_level(up):
            dc, dskip = dec[0].backward(d)
        else:
            dc, dskip = _split(dec[0].backward(d), c, c)
        dx = up.backward(dc)
        return (dx if getattr(up, "dx_coarse", False) else _upsample(dx, backward=True)), dskip

    @staticmethod
    def _seq_back(layers, dy, need_last=True):
        for i, l in enumerate(reversed(layers)):
            dy = l.backward(dy, need_dx=need_last or i < len(layers) - 1)
        return dy

    def backward(self, df1):
        """Backward pass from the gradient df1 of the head's input (as
        head_loss leaves it), after features(keep=True)."""
        c1, c2, c3, _ = self.channels
        d, de1 = self._decoder_back(self.up1, self.dec1, df1, c1)
        d, de2 = self._decoder_back(self.up2, self.dec2, d, c2)
        d, de3 = self._decoder_back(self.up3, self.dec3, d, c3)
        # each down-convolution's data gradient adds the skip connection's gradient in its epilogue
        d = self.down3.backward(self._seq_back(self.bott, d), residual=de3)
        d = self.down2.backward(self._seq_back(self.enc3, d), residual=de2)
        d = self.down1.backward(self._seq_back(self.enc2, d), residual=de1)
        self._seq_back(self.enc1, d, need_last=False)

    def zero_grad(self):
        self.g32.zero_()

    def step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        """One Adam step over every parameter (one launch on the flat
        buffers, BF16 copies included), then each layer's data-gradient
        weights from its new BF16 weights."""
        self.t += 1
        L = fdc.lib()
        _ok(L.fdc_adam(_p(self.p32), _p(self.g32), _p(self.m32), _p(self.v32), _p(self.p16), self.p32.numel(),
                       lr, b1, b2, eps, self.t, _s()), "adam")
        if getattr(self, "_tr", None) is None:  # geometries and pointers of every layer (buffers are fixed)
            ls = self.layers()
            self._tr = ((Conv3d * len(ls))(*[l.geom((1, 8, 8, 8, l.cin))[0] for l in ls]),
                        (C.c_void_p * len(ls))(*[l.w16.data_ptr() for l in ls]),
                        (C.c_void_p * len(ls))(*[l.wt16.data_ptr() for l in ls]))
        g, w, wt = self._tr
        _ok(L.fdc_conv3d_transpose_weights_batch(len(g), g, w, wt, _s()), "transpose")
        for l in (self.up1, self.up2, self.up3):
            l.collapse_up()

    def state(self):
        return [l.state() for l in self.layers()]

    def load(self, states):
        for l, s in zip(self.layers(), states):
            l.load(s)

    def save_npz(self, path):
        """FP32 master weights and biases, layer by layer (w0, b0, w1, b1, ...)."""
        arrs = {}
        for i, st in enumerate(self.state()):
            arrs[f"w{i}"] = st["w"]
            arrs[f"b{i}"] = st["b"]
        np.savez(path, **arrs)

    def load_npz(self, path):
        with np.load(path) as z:
            states = [{"w": z[f"w{i}"], "b": z[f"b{i}"]} for i in range(len(self.layers()))]
        for l, st in zip(self.layers(), states):
            if st["w"].shape != tuple(l.w32.shape) or st["b"].shape != tuple(l.b32.shape):
                raise ValueError(f"{path}: weight shapes do not match the network")
        self.load(states)


class Sample:
    """One case on the device: network input, its FP32 dose channel, and
    (for training) the target correction; dose_scale maps back to Gy."""

    def __init__(self, dose_low, density, dose_high=None, density_scale=0.5):
        import torch
        self.shape = tuple(dose_low.shape)  # (nz, ny, nx)
        n = dose_low.numel()
        dev = dose_low.device
        self.scale = float(dose_low.max())
        if self.scale <= 0:
            self.scale = 1.0
        self.x = torch.empty((1,) + self.shape + (16,), dtype=torch.bfloat16, device=dev)
        self.dose_in = torch.empty(self.shape, dtype=torch.float32, device=dev)
        self.target = torch.empty(self.shape, dtype=torch.float32, device=dev) if dose_high is not None else None
        _ok(fdc.lib().fdc_unet_prepare(_p(dose_low), _p(density), _p(dose_high), n, self.scale, density_scale,
                                       _p(self.x), _p(self.dose_in), _p(self.target), _s()), "prepare")


class _Transformed:
    """Scratch pair holding a sample after a lateral symmetry (input and target)."""

    def __init__(self, like):
        import torch
        self.shape = like.shape
        self.x = torch.empty_like(like.x)
        self.target = torch.empty_like(like.target)
        self.dose_in = like.dose_in

    def load(self, sample, code):
        d, h, w = sample.shape
        _ok(fdc.lib().fdc_unet_dihedral(_p(sample.x), _p(sample.target), d, h, w, code, _p(self.x),
                                        _p(self.target), _s()), "dihedral")
        return self


def train_step(net, sample, lr):
    """Forward, loss, backward and Adam step; returns the loss tensor (FP32,
    device) without synchronising."""
    import torch
    f1 = net.features(sample.x)
    loss = torch.zeros(1, dtype=torch.float32, device=f1.device)
    df1 = torch.empty_like(f1)
    net.zero_grad()
    net.head_loss(f1, sample.target, loss, df1)
    net.backward(df1)
    net.step(lr)
    return loss


def evaluate_loss(net, sample):
    import torch
    f1 = net.features(sample.x, keep=False)
    loss = torch.zeros(1, dtype=torch.float32, device=f1.device)
    net.head_loss(f1, sample.target, loss)
    return loss


def denoise(net, sample):
    """Denoised dose (Gy, FP64 on the device) of a prepared sample."""
    import torch
    f1 = net.features(sample.x, keep=False)
    out = torch.empty(sample.shape, dtype=torch.float64, device=f1.device)
    _ok(fdc.lib().fdc_unet_head(_p(f1), f1.shape[-1], _p(net.head.w16), _p(net.head.b32), out.numel(),
                                _p(sample.dose_in), sample.scale, None, _p(out), _s()), "head")
    return out


class InferenceGraph:
    """Repeated inference on fixed buffers as one CUDA graph: denoise() of
    `sample` is captured once (after a warm-up pass that sets every kernel's
    attributes) and replayed by run(); refill sample.x / sample.dose_in in
    place (e.g. fdc_unet_prepare into them) between runs.  The graph holds its
    own output buffer, returned by run()."""

    def __init__(self, net, sample):
        import torch
        self.net, self.sample = net, sample
        denoise(net, sample)  # warm-up outside the capture
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.out = denoise(net, sample)

    def run(self):
        self.graph.replay()
        return self.out


class DenoisedPath:
    """The denoised path on fixed device buffers: the engine's low-history
    run writes its dose into `dose`, then one CUDA graph computes the dose
    scale on the device (fdc_unet_dose_scale), the network input, the network
    and the head's denoised dose (no host read of the scale, no launch from
    the host between them).  Same result as denoise(net, Sample(dose,
    density)).  `density` is copied in by set_density (e.g. per phantom)."""

    def __init__(self, net, shape, density_scale=0.5, device="cuda:0"):
        import torch
        self.net, self.shape, self.density_scale = net, tuple(shape), density_scale
        n = int(np.prod(shape))
        self.n = n
        self.dose = torch.zeros(self.shape, dtype=torch.float64, device=device)
        self.density = torch.ones(self.shape, dtype=torch.float32, device=device)
        self.scale = torch.zeros(1, dtype=torch.float64, device=device)
        self.x = torch.empty((1,) + self.shape + (16,), dtype=torch.bfloat16, device=device)
        self.dose_in = torch.empty(self.shape, dtype=torch.float32, device=device)
        self._graph = None

    def set_density(self, density):
        self.density.copy_(density)

    def _pass(self):
        import torch
        L = fdc.lib()
        _ok(L.fdc_unet_dose_scale(_p(self.dose), self.n, _p(self.scale), _s()), "dose scale")
        _ok(L.fdc_unet_prepare_dev(_p(self.dose), _p(self.density), self.n, _p(self.scale), self.density_scale,
                                   _p(self.x), _p(self.dose_in), _s()), "prepare")
        f1 = self.net.features(self.x, keep=False)
        out = torch.empty(self.shape, dtype=torch.float64, device=f1.device)
        _ok(L.fdc_unet_head_dev(_p(f1), f1.shape[-1], _p(self.net.head.w16), _p(self.net.head.b32), self.n,
                                _p(self.dose_in), _p(self.scale), _p(out), _s()), "head")
        return out

    def denoise(self):
        """Denoised dose (Gy, FP64 on the device) of the dose now in `dose`;
        the graph is captured at the first call (after one pass outside it)."""
        import torch
        if self._graph is None:
            self._pass()
            torch.cuda.synchronize()
            self._graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self._graph):
                self.out = self._pass()
        self._graph.replay()
        return self.out

    def run(self, eng, beam, seed, stream=None):
        """Low-history run of `beam` (engine with the case's phantom loaded)
        into `dose`, then the denoising graph; returns the denoised dose."""
        eng.run_ex(beam, 0, seed, dose=self.dose, stream=stream)
        return self.denoise()


def gamma_pass_rate(ref, ev, spacing, dose_frac=0.02, dta=0.2, threshold=0.1, gamma_out=None):
    """Gamma pass rate (fraction of voxels above threshold * max(ref) with
    gamma <= 1) of an evaluated dose against a reference (FP64 device grids
    [nz][ny][nx], spacing (dx, dy, dz) cm)."""
    import torch
    nz, ny, nx = ref.shape
    scratch = torch.zeros(3, dtype=torch.int64, device=ref.device)
    r = C.c_double()
    _ok(fdc.lib().fdc_gamma(_p(ref), _p(ev), nz, ny, nx, float(spacing[2]), float(spacing[1]), float(spacing[0]),
                            dose_frac, dta, threshold, _p(gamma_out), _p(scratch), C.byref(r), _s()), "gamma")
    return r.value


# ----------------------------------------------------------------------------
# Training pairs from the engine, training and evaluation.

def case_beam(seed, n):
    """Random rectangular field of case `seed`: 100-180 MeV, 2-6 cm sides,
    centre within 3 cm of the axis, 1 % energy spread."""
    from . import synth
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    E = rng.uniform(100.0, 180.0)
    w, h = rng.uniform(2.0, 6.0, 2)
    cx, cy = rng.uniform(-3.0, 3.0, 2)
    return synth.make_spots([dict(x=cx, y=cy, energy=E, sigma_e=0.01 * E, a=w, b=h,
                                  profile=synth.PROFILE_RECT, layer=0, n_histories=int(n))])


def case_phantom(seed, n=128, voxel_cm=0.2):
    from . import synth
    return synth.thorax_phantom(seed=20_000 + seed, shape=(n, n, n), voxel_cm=voxel_cm)


class Case:
    def __init__(self, seed, phantom, density, low, high, beam_low):
        self.seed, self.phantom, self.density, self.low, self.high = seed, phantom, density, low, high
        self.beam_low = beam_low


def _mirrored(ph, variant):
    """The phantom mirrored in x (variant & 1) and/or y (variant & 2)."""
    import copy
    q = copy.copy(ph)
    m, d = ph.material, ph.density
    if variant & 1:
        m, d = m[:, :, ::-1], d[:, :, ::-1]
    if variant & 2:
        m, d = m[:, ::-1, :], d[:, ::-1, :]
    q.material, q.density = np.ascontiguousarray(m), np.ascontiguousarray(d)
    return q


def generate_cases(eng, seeds, n_low=100_000, n_high=100_000_000, grid=128, keep_phantom=False, variants=1):
    """Per seed: random phantom (and, with variants > 1, its mirror images in
    x, y and xy), each with its own random field; low- and high-history doses
    from the engine (device FP64), plus the density (device FP32).  The
    engine's dose is the total of its histories, so the high-history dose is
    rescaled to the low-history count (both are then the dose of n_low
    protons)."""
    import torch
    cases = []
    for sd0 in seeds:
        base = case_phantom(sd0, grid)
        for var in range(variants):
            sd = sd0 if variants == 1 else 1_000_000 + sd0 * variants + var
            ph = base if var == 0 else _mirrored(base, var)
            cases.extend(_one_case(eng, sd, ph, n_low, n_high, keep_phantom))
    return cases


def _one_case(eng, sd, ph, n_low, n_high, keep_phantom):
    import torch
    eng.load_phantom(ph)
    bl = case_beam(sd, n_low)
    bh = case_beam(sd, n_high)
    low = eng.run(bl, 0, 1_000_003 * sd + 1)
    high = eng.run(bh, 0, 1_000_003 * sd + 2)
    high.mul_(n_low / n_high)
    eng.sync()
    dens = torch.from_numpy(np.ascontiguousarray(ph.density)).cuda()
    return [Case(sd, ph if keep_phantom else None, dens, low, high, bl)]


def train(net, samples, epochs, lr=1e-3, lr_final=1e-4, log=None, seed=0, augment=False, held_out=None):
    """Adam over the samples in a seeded random order; cosine learning rate
    from lr to lr_final.  With augment, every visit of a sample sees it under
    a random lateral symmetry (mirror x / y, exchange x and y: exact symmetries
    of a field along +z).  Returns the per-epoch mean training losses and, with
    held_out samples, their mean loss after every epoch."""
    import torch
    rng = np.random.default_rng(seed)
    total = epochs * len(samples)
    it = 0
    hist, hist_out = [], []
    scratch = _Transformed(samples[0]) if augment and samples else None
    for ep in range(epochs):
        losses = []
        for i in rng.permutation(len(samples)):
            f = it / max(1, total - 1)
            cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * f))
            s = samples[i]
            if scratch is not None:
                d, h, w = s.shape
                code = int(rng.integers(0, 8 if h == w else 4))
                if code:
                    s = scratch.load(s, code)
            losses.append(train_step(net, s, cur))
            it += 1
        m = float(torch.cat(losses).mean())
        hist.append(m)
        if held_out:
            hist_out.append(float(torch.cat([evaluate_loss(net, s) for s in held_out]).mean()))
        if log:
            log(ep, m)
    return (hist, hist_out) if held_out else hist


def evaluate(net, eng, cases, n_low, spacing, dose_frac=0.02, dta=0.2, threshold=0.1, target_sigma=0.02,
             host_timing=False):
    """Per held-out case: gamma pass rate (dose_frac / dta) against the
    high-history plain dose of the denoised low-history dose and of the raw
    low-history dose; device time of the denoised path (low-history run +
    network, as DenoisedPath runs it: the run, then one CUDA graph from the
    dose scale to the denoised dose; timed after a warm pass) and of the
    plain method run to ``target_sigma`` mean batch uncertainty (eq. (1),
    voxels above half the maximum).  With host_timing, also the host wall
    time of both from the beam in host memory to the dose in (pinned) host
    memory, copies included: the denoised path as that run, graph and one
    dose download; the plain method as one fdc_run_host call of the history
    count it needs for target_sigma."""
    import time
    import torch
    from .measure import time_to_sigma
    rows = []
    path = None
    for c in cases:
        eng.load_phantom(c.phantom)
        shape = c.phantom.shape[::-1]
        if path is None or path.shape != tuple(shape):
            path = DenoisedPath(net, shape, device=c.density.device)
        path.set_density(c.density)
        # denoised path, timed from the start of the low-history run to the dose
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        path.run(eng, c.beam_low, 7 + c.seed)  # warm (the first case also captures the graph)
        e0.record()
        out = path.run(eng, c.beam_low, 7 + c.seed)
        e1.record()
        e1.synchronize()
        t_den = e0.elapsed_time(e1) * 1e-3
        low = path.dose.clone()
        out = out.clone()
        g_den = gamma_pass_rate(c.high, out, spacing, dose_frac, dta, threshold)
        g_raw = gamma_pass_rate(c.high, low, spacing, dose_frac, dta, threshold)
        plain = time_to_sigma(eng, case_beam(c.seed, 100_000_000), shape, 11 + c.seed, target_sigma)
        # the plain method's own dose at that history count, against the same reference
        n2 = plain["histories"]
        d2 = eng.run(case_beam(c.seed, n2), 0, 13 + c.seed)
        d2.mul_(n_low / n2)
        g_plain = gamma_pass_rate(c.high, d2, spacing, dose_frac, dta, threshold)
        row = {"seed": c.seed, "gamma_denoised": g_den, "gamma_low": g_raw, "gamma_plain_2pct": g_plain,
               "seconds_denoised": t_den, "seconds_plain_2pct": plain["seconds"],
               "histories_plain_2pct": n2, "plain_reached": plain["reached"]}
        if host_timing:
            host = torch.empty(shape, dtype=torch.float64).pin_memory()
            host_np = np.empty(shape, np.float64)
            walls = []
            for rep in range(3):
                torch.cuda.synchronize()
                t = time.perf_counter()
                host.copy_(path.run(eng, c.beam_low, 17 + c.seed + rep))
                torch.cuda.synchronize()
                walls.append(time.perf_counter() - t)
            row["wall_seconds_denoised"] = min(walls[1:])
            bp = case_beam(c.seed, n2)
            walls = []
            for rep in range(3):
                t = time.perf_counter()
                eng.run_host(bp, n2, 19 + c.seed + rep, host_np)
                walls.append(time.perf_counter() - t)
            row["wall_seconds_plain_2pct"] = min(walls[1:])
        rows.append(row)
    keys = ["gamma_denoised", "gamma_low", "gamma_plain_2pct", "seconds_denoised", "seconds_plain_2pct",
            "histories_plain_2pct"]
    if host_timing:
        keys += ["wall_seconds_denoised", "wall_seconds_plain_2pct"]
    summary = {k: float(np.mean([r[k] for r in rows])) for k in keys}
    summary["min_gamma_denoised"] = float(min(r["gamma_denoised"] for r in rows))
    summary["cases_gamma_ge_98"] = int(sum(r["gamma_denoised"] >= 0.98 for r in rows))
    return rows, summary
