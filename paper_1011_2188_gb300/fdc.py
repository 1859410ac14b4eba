"""Python binding of the C ABI in ``include/fdc.h`` (argument marshalling only).

Every step of the dose calculation runs in ``libfdc.so``; this module only
converts numpy inputs to the C structs, hands over device pointers of torch
tensors and the current torch stream, and turns status codes into
exceptions.  There is no CPU fallback: if the library is missing the import
of the engine fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdc.so")

FDC_OK = 0
ERRORS = {1: "FDC_ERR_INVALID", 2: "FDC_ERR_NOT_LOADED", 3: "FDC_ERR_CUDA", 4: "FDC_ERR_OOM",
          5: "FDC_ERR_STEP_LIMIT", 6: "FDC_ERR_OVERFLOW", 7: "FDC_ERR_TIMEOUT"}
TALLY_UNITS_PER_MEV = float(1 << 28)

# Every function the header declares, with its C signature.
_p = C.c_void_p
SIGNATURES = {
    "fdc_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "fdc_destroy": (None, [_p]),
    "fdc_last_error": (C.c_char_p, [_p]),
    "fdc_load_database": (C.c_int, [_p, _p]),
    "fdc_load_phantom": (C.c_int, [_p, _p]),
    "fdc_run": (C.c_int, [_p, _p, C.c_uint64, C.c_uint64, _p, _p]),
    "fdc_run_ex": (C.c_int, [_p, _p, C.c_uint64, C.c_uint64, _p, _p, _p]),
    "fdc_run_host": (C.c_int, [_p, _p, C.c_uint64, C.c_uint64, _p, _p]),
    "fdc_sync": (C.c_int, [_p, _p, _p]),
    "fdc_dose_from_tally": (C.c_int, [_p, _p, _p, _p]),
    "fdc_batch_stats": (C.c_int, [_p, _p, _p, C.c_int32, C.c_double, _p, _p, _p, _p]),
    "fdc_history_stats": (C.c_int, [_p, _p, _p, C.c_uint64, C.c_double, _p, _p, _p, _p]),
    "fdc_autotune": (C.c_int, [_p, _p, C.c_uint64, C.c_uint64, _p, _p]),
    "fdc_set_timing": (C.c_int, [_p, C.c_int32]),
    "fdc_last_kernel_ms": (C.c_int, [_p, _p, _p]),
    "fdc_probe_atomics": (C.c_int, [_p, C.c_uint64, C.c_uint64, _p, _p]),
    "fdc_run_noalloc": (C.c_int, [_p, _p, C.c_uint64, C.c_uint64, _p, _p, _p]),
    # denoiser kernels (include/fdc_unet.h)
    "fdc_conv3d_forward": (C.c_int, [_p, _p, _p, _p, _p, _p, _p]),
    "fdc_conv3d_forward_fused": (C.c_int, [_p, _p, C.c_int32, C.c_int32, _p, _p, _p, _p, _p, _p]),
    "fdc_conv3d_forward_up": (C.c_int, [_p, _p, _p, _p, _p, _p, _p]),
    "fdc_conv3d_collapse_up_weights": (C.c_int, [_p, _p, _p, _p]),
    "fdc_conv3d_backward_data_up": (C.c_int, [_p, _p, _p, _p, _p, _p]),
    "fdc_conv3d_collapse_up_weights_t": (C.c_int, [_p, _p, _p, _p]),
    "fdc_conv3d_backward_data": (C.c_int, [_p, _p, _p, _p, _p, _p]),
    "fdc_conv3d_backward_data_add": (C.c_int, [_p, _p, _p, _p, _p, _p, _p]),
    "fdc_conv3d_backward_weights": (C.c_int, [_p, _p, _p, _p, _p, _p]),
    "fdc_conv3d_backward_weights_fused": (C.c_int, [_p, _p, C.c_int32, C.c_int32, _p, _p, _p, _p, _p]),
    "fdc_conv3d_backward_data_fused": (C.c_int, [_p, _p, _p, _p, C.c_int32, C.c_int32, _p, _p, _p, _p]),
    "fdc_conv3d_transpose_weights": (C.c_int, [_p, _p, _p, _p]),
    "fdc_conv3d_transpose_weights_batch": (C.c_int, [C.c_int32, _p, _p, _p, _p]),
    "fdc_relu_backward": (C.c_int, [_p, _p, _p, C.c_int64, _p]),
    "fdc_upsample2": (C.c_int, [_p, _p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _p]),
    "fdc_concat_channels": (C.c_int, [_p, C.c_int32, _p, C.c_int32, _p, C.c_int64, C.c_int32, _p]),
    "fdc_mse": (C.c_int, [_p, C.c_int32, _p, C.c_int64, _p, _p, _p]),
    "fdc_adam": (C.c_int, [_p, _p, _p, _p, _p, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32,
                           _p]),
    "fdc_f32_to_bf16": (C.c_int, [_p, _p, C.c_int64, _p]),
    "fdc_add_bf16": (C.c_int, [_p, _p, _p, C.c_int64, _p]),
    "fdc_unet_prepare": (C.c_int, [_p, _p, _p, C.c_int64, C.c_double, C.c_float, _p, _p, _p, _p]),
    "fdc_unet_finish": (C.c_int, [_p, _p, C.c_int64, C.c_double, _p, _p]),
    "fdc_unet_dose_scale": (C.c_int, [_p, C.c_int64, _p, _p]),
    "fdc_unet_prepare_dev": (C.c_int, [_p, _p, C.c_int64, _p, C.c_float, _p, _p, _p]),
    "fdc_unet_head_dev": (C.c_int, [_p, C.c_int32, _p, _p, C.c_int64, _p, _p, _p, _p]),
    "fdc_unet_head": (C.c_int, [_p, C.c_int32, _p, _p, C.c_int64, _p, C.c_double, _p, _p, _p]),
    "fdc_unet_head_loss": (C.c_int, [_p, C.c_int32, _p, _p, _p, C.c_int64, _p, _p, _p, _p, _p]),
    "fdc_unet_status": (C.c_int, [C.c_int32]),
    "fdc_debug_wait_timeout": (C.c_int, [C.c_int64, _p]),
    "fdc_unet_dihedral": (C.c_int, [_p, _p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _p, _p, _p]),
    "fdc_gamma": (C.c_int, [_p, _p, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                            C.c_double, C.c_double, C.c_double, _p, _p, _p, _p]),
    "fdc_debug_philox": (C.c_int, [C.c_uint64, C.c_uint64, _p, C.c_uint64, _p, _p]),
    "fdc_debug_sample": (C.c_int, [_p, _p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int32, C.c_int32,
                                   _p, _p, _p]),
}


class Database(C.Structure):
    _fields_ = [("n_energies", C.c_int32), ("energy", _p), ("track_begin", _p), ("step_begin", _p),
                ("dE", _p), ("len", _p), ("theta", _p), ("phi", _p), ("esec", _p)]


class Phantom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_mat", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("material", _p), ("density", _p), ("s_rel", _p), ("k_theta", _p)]


class Spot(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("energy", C.c_double), ("sigma_e", C.c_double),
                ("a", C.c_double), ("b", C.c_double), ("profile", C.c_int32), ("layer", C.c_int32),
                ("n_histories", C.c_uint64)]


class Beam(C.Structure):
    _fields_ = [("n_spots", C.c_int32), ("spots", _p)]


class Schedule(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("warps_per_cta", C.c_int32), ("chunk", C.c_int32),
                ("aggregate", C.c_int32)]


class RunOpts(C.Structure):
    _fields_ = [("history_offset", C.c_uint64), ("track_group", C.c_int32), ("no_rotation", C.c_int32),
                ("scaling_mode", C.c_int32), ("fp64_geometry", C.c_int32), ("n_batches", C.c_int32),
                ("no_graph", C.c_int32), ("schedule", Schedule)]


class Outputs(C.Structure):
    _fields_ = [("dose", _p), ("layer_dose", _p), ("batch_sum", _p), ("batch_sumsq", _p), ("tally", _p),
                ("history_sumsq", _p)]


class Counters(C.Structure):
    _fields_ = [("histories", C.c_uint64), ("steps", C.c_uint64), ("segments", C.c_uint64),
                ("replayed", C.c_int64), ("escaped", C.c_int64), ("status", C.c_int32), ("pad", C.c_int32),
                ("bad_history", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


SPOT_DTYPE = np.dtype([("x", "<f8"), ("y", "<f8"), ("energy", "<f8"), ("sigma_e", "<f8"),
                       ("a", "<f8"), ("b", "<f8"), ("profile", "<i4"), ("layer", "<i4"),
                       ("n_histories", "<u8")])
assert SPOT_DTYPE.itemsize == C.sizeof(Spot) == 64

_lib = None


def lib():
    """Load libfdc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfdc.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class FdcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class _Keep(list):
    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.append(a)
        return a.ctypes.data


def beam_struct(spots, keep):
    s = np.zeros(len(spots), dtype=SPOT_DTYPE)
    for name in SPOT_DTYPE.names:
        s[name] = spots[name]
    keep.append(s)
    return Beam(len(s), s.ctypes.data)


def philox(counters, key, stream=None):
    """Device Philox4x64-10 on counters (torch uint64/int64 [n, 4] on the GPU)."""
    import torch
    out = torch.empty_like(counters)
    rc = lib().fdc_debug_philox(int(key[0]), int(key[1]), _ptr(counters), counters.shape[0], _ptr(out),
                                _stream_handle(stream))
    if rc:
        raise FdcError(rc, "debug_philox")
    return out


def probe_atomics(slots, n_ops, stream=None):
    """Time n_ops hashed 64-bit atomic adds into the int64 CUDA tensor
    ``slots``; returns milliseconds."""
    ms = C.c_double()
    rc = lib().fdc_probe_atomics(_ptr(slots), slots.numel(), int(n_ops), C.byref(ms), _stream_handle(stream))
    if rc:
        raise FdcError(rc, "probe_atomics")
    return ms.value


class Engine:
    """One dose-calculation context on a CUDA device."""

    def __init__(self, device=0):
        self._lib = lib()
        h = C.c_void_p()
        rc = self._lib.fdc_create(C.byref(h), int(device))
        if rc:
            raise FdcError(rc, f"fdc_create(device={device})")
        self.h = h
        self.device = int(device)
        self.shape = None
        self.n_layers = 1

    def close(self):
        if getattr(self, "h", None):
            self._lib.fdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc:
            raise FdcError(rc, f"{what}: {self._lib.fdc_last_error(self.h).decode()}")

    # ---- inputs
    def load_database(self, db):
        k = _Keep()
        s = Database(int(len(db.energy)), k.arr(db.energy, np.float32), k.arr(db.track_begin, np.int64),
                     k.arr(db.step_begin, np.int64), k.arr(db.dE, np.float32), k.arr(db.len, np.float32),
                     k.arr(db.theta, np.float32), k.arr(db.phi, np.float32), k.arr(db.esec, np.float32))
        self._check(self._lib.fdc_load_database(self.h, C.byref(s)), "load_database")

    def load_phantom(self, ph):
        k = _Keep()
        nx, ny, nz = ph.shape
        s = Phantom(nx, ny, nz, int(len(ph.s_rel)), *map(float, ph.spacing), *map(float, ph.origin),
                    k.arr(ph.material, np.uint8), k.arr(ph.density, np.float32),
                    k.arr(ph.s_rel, np.float32), k.arr(ph.k_theta, np.float32))
        self._check(self._lib.fdc_load_phantom(self.h, C.byref(s)), "load_phantom")
        self.shape = (nz, ny, nx)

    # ---- runs
    def run(self, spots, n_histories=0, seed=0, dose=None, stream=None):
        """Dose (Gy) of histories [0, n_histories) into a float64 CUDA tensor."""
        import torch
        if dose is None:
            # without a phantom the library reports FDC_ERR_NOT_LOADED
            shape = self.shape if self.shape is not None else (1,)
            dose = torch.empty(shape, dtype=torch.float64, device=f"cuda:{self.device}")
        k = _Keep()
        b = beam_struct(spots, k)
        self._check(self._lib.fdc_run(self.h, C.byref(b), int(n_histories), int(seed), _ptr(dose),
                                      _stream_handle(stream)), "run")
        return dose

    def run_ex(self, spots, n_histories=0, seed=0, history_offset=0, track_group=1, rotate=True,
               scaling_mode=0, fp64_geometry=False, n_batches=0, schedule=None, dose=None,
               layer_dose=None, batch_sum=None, batch_sumsq=None, tally=None, stream=None, graph=True,
               history_sumsq=None):
        k = _Keep()
        b = beam_struct(spots, k)
        sch = Schedule(*(schedule or (0, 0, 0, 0)))
        o = RunOpts(int(history_offset), int(track_group), 0 if rotate else 1, int(scaling_mode),
                    1 if fp64_geometry else 0, int(n_batches), 0 if graph else 1, sch)
        out = Outputs(_ptr(dose), _ptr(layer_dose), _ptr(batch_sum), _ptr(batch_sumsq), _ptr(tally),
                      _ptr(history_sumsq))
        self._check(self._lib.fdc_run_ex(self.h, C.byref(b), int(n_histories), int(seed), C.byref(o),
                                         C.byref(out), _stream_handle(stream)), "run_ex")

    def run_noalloc(self, spots, n_histories=0, seed=0, dose=None, counters=None, stream=None):
        """fdc_run_noalloc: the run's scratch lives in the library's static
        device array, so the call allocates no device memory (the caller must
        provide ``dose``; ``counters`` is an optional device buffer of at
        least sizeof(fdc_counters) = 56 bytes, e.g. a uint8 tensor, that
        receives the run's counters)."""
        if dose is None:
            raise ValueError("run_noalloc needs a caller-provided dose tensor")
        k = _Keep()
        b = beam_struct(spots, k)
        self._check(self._lib.fdc_run_noalloc(self.h, C.byref(b), int(n_histories), int(seed), _ptr(dose),
                                              _ptr(counters), _stream_handle(stream)), "run_noalloc")
        return dose

    def run_host(self, spots, n_histories=0, seed=0, dose_host=None, track_group=1):
        """End-to-end call with a host (numpy float64) dose buffer."""
        if dose_host is None:
            dose_host = np.empty(self.shape, np.float64)
        k = _Keep()
        b = beam_struct(spots, k)
        o = RunOpts(0, int(track_group), 0, 0, 0, 0, 0, Schedule(0, 0, 0, 0))
        self._check(self._lib.fdc_run_host(self.h, C.byref(b), int(n_histories), int(seed), C.byref(o),
                                           C.c_void_p(dose_host.ctypes.data)), "run_host")
        return dose_host

    def dose_from_tally(self, tally, dose=None, stream=None):
        """Dose (Gy) of an int64 energy tally (CUDA tensor, e.g. the sum of the
        tallies of several history ranges) into a float64 CUDA tensor."""
        import torch
        if dose is None:
            dose = torch.empty(tally.shape, dtype=torch.float64, device=tally.device)
        self._check(self._lib.fdc_dose_from_tally(self.h, _ptr(tally), _ptr(dose), _stream_handle(stream)),
                    "dose_from_tally")
        return dose

    def sync(self, stream=None):
        c = Counters()
        self._check(self._lib.fdc_sync(self.h, _stream_handle(stream), C.byref(c)), "sync")
        return c.as_dict()

    def sync_status(self, stream=None):
        """(status, counters) without raising on a device error."""
        c = Counters()
        rc = self._lib.fdc_sync(self.h, _stream_handle(stream), C.byref(c))
        return rc, c.as_dict()

    def set_timing(self, enable=True):
        self._check(self._lib.fdc_set_timing(self.h, 1 if enable else 0), "set_timing")

    def last_kernel_ms(self):
        a, b = C.c_double(), C.c_double()
        self._check(self._lib.fdc_last_kernel_ms(self.h, C.byref(a), C.byref(b)), "last_kernel_ms")
        return a.value, b.value

    def batch_stats(self, batch_sum, batch_sumsq, n_batches, frac=0.5, stream=None):
        import torch
        mean = torch.empty_like(batch_sum)
        sigma = torch.empty_like(batch_sum)
        r = C.c_double()
        self._check(self._lib.fdc_batch_stats(self.h, _ptr(batch_sum), _ptr(batch_sumsq), int(n_batches),
                                              float(frac), _ptr(mean), _ptr(sigma), C.byref(r),
                                              _stream_handle(stream)), "batch_stats")
        return mean, sigma, r.value

    def history_stats(self, dose_sum, history_sumsq, n_histories, frac=0.5, stream=None):
        """Eq. (2): per-history mean dose, its sigma, and the mean sigma/mean."""
        import torch
        mean = torch.empty_like(dose_sum)
        sigma = torch.empty_like(dose_sum)
        r = C.c_double()
        self._check(self._lib.fdc_history_stats(self.h, _ptr(dose_sum), _ptr(history_sumsq), int(n_histories),
                                                float(frac), _ptr(mean), _ptr(sigma), C.byref(r),
                                                _stream_handle(stream)), "history_stats")
        return mean, sigma, r.value

    def autotune(self, spots, n_histories, seed=0, history_offset=0, track_group=1, rotate=True,
                 scaling_mode=0, fp64_geometry=False):
        """fdc_autotune for runs with these options; returns the chosen
        (ctas_per_sm, warps_per_cta, chunk, aggregate)."""
        k = _Keep()
        b = beam_struct(spots, k)
        o = RunOpts(int(history_offset), int(track_group), 0 if rotate else 1, int(scaling_mode),
                    1 if fp64_geometry else 0, 0, 0, Schedule(0, 0, 0, 0))
        s = Schedule()
        self._check(self._lib.fdc_autotune(self.h, C.byref(b), int(n_histories), int(seed), C.byref(o),
                                           C.byref(s)), "autotune")
        return (s.ctas_per_sm, s.warps_per_cta, s.chunk, s.aggregate)

    def debug_sample(self, spots, seed, h_begin, n, track_group=1, rotate=True, stream=None):
        import torch
        dev = f"cuda:{self.device}"
        f = torch.empty((n, 4), dtype=torch.float32, device=dev)
        i = torch.empty((n, 3), dtype=torch.int64, device=dev)
        k = _Keep()
        b = beam_struct(spots, k)
        self._check(self._lib.fdc_debug_sample(self.h, C.byref(b), int(seed), int(h_begin), int(n),
                                               int(track_group), 0 if rotate else 1, _ptr(f), _ptr(i),
                                               _stream_handle(stream)), "debug_sample")
        return f, i
