"""CPU oracle for the track-repeating dose engine.

TEST INFRASTRUCTURE ONLY: the plain, sequential FP64 implementation in
``fdc_oracle.c`` plus the statistics of ``stats.py``.  Only the test suite,
the smoke check and the benchmark's CPU-baseline leg may import this package;
the GPU library never calls it and shares no code with it.

Inputs are plain objects with the attributes of the project's synthetic
inputs (database: energy, track_begin, step_begin, dE, len, theta, phi, esec;
phantom: shape, spacing, origin, material, density, s_rel, k_theta; beam: a
numpy structured array with fields x, y, energy, sigma_e, a, b, profile,
layer, n_histories).  Nothing here imports the GPU package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Db(C.Structure):
    _fields_ = [("n_energies", C.c_int32), ("energy", C.c_void_p), ("track_begin", C.c_void_p),
                ("step_begin", C.c_void_p), ("dE", C.c_void_p), ("len", C.c_void_p),
                ("theta", C.c_void_p), ("phi", C.c_void_p), ("esec", C.c_void_p)]


class _Ph(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_mat", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("material", C.c_void_p), ("density", C.c_void_p),
                ("s_rel", C.c_void_p), ("k_theta", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("h_begin", C.c_uint64), ("h_end", C.c_uint64),
                ("track_group", C.c_int32), ("scaling_mode", C.c_int32), ("per_layer", C.c_int32),
                ("rotate", C.c_int32)]


class _Out(C.Structure):
    _fields_ = [("edep", C.c_void_p), ("hh_sumsq", C.c_void_p), ("replayed", C.c_double),
                ("escaped", C.c_double), ("n_histories", C.c_uint64), ("n_steps", C.c_uint64),
                ("n_segments", C.c_uint64), ("hv_sumsq", C.c_void_p)]


SPOT_FIELDS = [("x", "<f8"), ("y", "<f8"), ("energy", "<f8"), ("sigma_e", "<f8"),
               ("a", "<f8"), ("b", "<f8"), ("profile", "<i4"), ("layer", "<i4"),
               ("n_histories", "<u8")]
_SPOT_DTYPE = np.dtype(SPOT_FIELDS)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.fdco_run.restype = C.c_int
            L.fdco_run.argtypes = [C.POINTER(_Db), C.POINTER(_Ph), C.c_void_p, C.c_int32,
                                   C.POINTER(_Opts), C.POINTER(_Out)]
            L.fdco_sample.restype = C.c_int
            L.fdco_sample.argtypes = [C.POINTER(_Db), C.c_void_p, C.c_int32, C.c_uint64,
                                      C.c_uint64, C.c_uint64, C.c_int32, C.c_int32, C.c_void_p,
                                      C.c_void_p]
            L.fdco_philox4x64_10.restype = None
            L.fdco_philox4x64_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
            L.fdco_dose.restype = None
            L.fdco_dose.argtypes = [C.POINTER(_Ph), C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class _Keep:
    """Holds the contiguous arrays behind a ctypes struct alive."""

    def __init__(self):
        self.refs = []

    def ptr(self, a, dtype):
        a = _c(a, dtype)
        self.refs.append(a)
        return a.ctypes.data


def _db_struct(db, keep):
    return _Db(int(len(db.energy)), keep.ptr(db.energy, np.float32), keep.ptr(db.track_begin, np.int64),
               keep.ptr(db.step_begin, np.int64), keep.ptr(db.dE, np.float32),
               keep.ptr(db.len, np.float32), keep.ptr(db.theta, np.float32),
               keep.ptr(db.phi, np.float32), keep.ptr(db.esec, np.float32))


def _ph_struct(ph, keep):
    nx, ny, nz = ph.shape
    return _Ph(nx, ny, nz, int(len(ph.s_rel)), *[float(v) for v in ph.spacing],
               *[float(v) for v in ph.origin], keep.ptr(ph.material, np.uint8),
               keep.ptr(ph.density, np.float32), keep.ptr(ph.s_rel, np.float32),
               keep.ptr(ph.k_theta, np.float32))


def _spots(beam, keep):
    b = np.zeros(len(beam), dtype=_SPOT_DTYPE)
    for name, _ in SPOT_FIELDS:
        b[name] = beam[name]
    keep.refs.append(b)
    return b.ctypes.data, len(b)


def philox4x64_10(counters, key):
    """counters: uint64 [n, 4]; key: 2 uint64 -> uint64 [n, 4]."""
    ctr = _c(counters, np.uint64).reshape(-1, 4)
    k = _c(key, np.uint64).reshape(2)
    out = np.empty_like(ctr)
    lib().fdco_philox4x64_10(ctr.ctypes.data, k.ctypes.data, out.ctypes.data, ctr.shape[0])
    return out


def sample(db, beam, seed, h_begin, n, track_group=1, rotate=True):
    """Task 1 of each history: returns (xyEpsi float32 [n,4], bin/track/k0 int64 [n,3])."""
    keep = _Keep()
    d = _db_struct(db, keep)
    sp, ns = _spots(beam, keep)
    f = np.zeros((n, 4), np.float32)
    i = np.zeros((n, 3), np.int64)
    rc = lib().fdco_sample(C.byref(d), sp, ns, seed, h_begin, n, track_group, 1 if rotate else 0,
                           f.ctypes.data, i.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle sample failed: {rc}")
    return f, i


class Result:
    def __init__(self, edep, hh_sumsq, out, hv_sumsq=None):
        self.edep = edep
        self.hh_sumsq = hh_sumsq
        self.hv_sumsq = hv_sumsq
        self.replayed = out.replayed
        self.escaped = out.escaped
        self.n_histories = int(out.n_histories)
        self.n_steps = int(out.n_steps)
        self.n_segments = int(out.n_segments)


def run(db, ph, beam, seed, h_begin=0, h_end=None, track_group=1, scaling_mode=0,
        per_layer=False, history_squares=False, rotate=True, visit_squares=False):
    """Replay histories [h_begin, h_end) in FP64.  Returns a ``Result`` whose
    ``edep`` is MeV per voxel, shape (nz, ny, nx) or (n_layers, nz, ny, nx);
    with history_squares, ``hh_sumsq`` sums each history's squared energy per
    voxel, with visit_squares ``hv_sumsq`` each voxel visit's (MeV^2)."""
    keep = _Keep()
    d = _db_struct(db, keep)
    p = _ph_struct(ph, keep)
    sp, ns = _spots(beam, keep)
    total = int(np.sum(np.asarray(beam["n_histories"], dtype=np.uint64)))
    if h_end is None:
        h_end = total
    nx, ny, nz = ph.shape
    n_layers = int(np.max(beam["layer"])) + 1 if per_layer else 1
    edep = np.zeros((n_layers, nz, ny, nx), np.float64)
    sq = np.zeros((nz, ny, nx), np.float64) if history_squares else None
    vq = np.zeros((nz, ny, nx), np.float64) if visit_squares else None
    out = _Out(edep.ctypes.data, sq.ctypes.data if sq is not None else None, 0.0, 0.0, 0, 0, 0,
               vq.ctypes.data if vq is not None else None)
    opts = _Opts(seed, h_begin, h_end, track_group, scaling_mode, 1 if per_layer else 0,
                 1 if rotate else 0)
    rc = lib().fdco_run(C.byref(d), C.byref(p), sp, ns, C.byref(opts), C.byref(out))
    if rc:
        raise RuntimeError(f"oracle run failed: {rc}")
    return Result(edep if per_layer else edep[0], sq, out, vq)


def run_parallel(db, ph, beam, seed, h_begin=0, h_end=None, threads=None, **kw):
    """``run`` over [h_begin, h_end) split into contiguous history ranges, one
    per thread (the C oracle keeps no global state and ctypes releases the GIL
    during the call); the per-thread FP64 grids and counters are summed.
    Histories are independent (Sec. 2.3), so this is the same replay as one
    sequential call up to the order of the FP64 additions."""
    from concurrent.futures import ThreadPoolExecutor
    lib()
    total = int(np.sum(np.asarray(beam["n_histories"], dtype=np.uint64)))
    if h_end is None:
        h_end = total
    if threads is None:
        try:
            threads = len(os.sched_getaffinity(0))
        except AttributeError:
            threads = os.cpu_count() or 1
    n = h_end - h_begin
    threads = max(1, min(int(threads), n))
    cuts = [h_begin + n * i // threads for i in range(threads + 1)]
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda i: run(db, ph, beam, seed, h_begin=cuts[i], h_end=cuts[i + 1], **kw),
                            range(threads)))
    res = parts[0]
    for r in parts[1:]:
        res.edep += r.edep
        if res.hh_sumsq is not None:
            res.hh_sumsq += r.hh_sumsq
        if res.hv_sumsq is not None:
            res.hv_sumsq += r.hv_sumsq
        res.replayed += r.replayed
        res.escaped += r.escaped
        res.n_histories += r.n_histories
        res.n_steps += r.n_steps
        res.n_segments += r.n_segments
    return res


def dose(ph, edep):
    """Energy (MeV per voxel) to dose (Gy), Sec. 2.3."""
    keep = _Keep()
    p = _ph_struct(ph, keep)
    e = _c(edep, np.float64)
    out = np.zeros_like(e)
    lib().fdco_dose(C.byref(p), e.ctypes.data, out.ctypes.data)
    return out
