"""Helpers of the GPU tests: run the engine through the C ABI and compare
with the oracle."""
from __future__ import annotations

import numpy as np

# Parity bar (GPU vs FP64 oracle on identical random streams): per voxel
# within 0.1 % of the maximum, total deposited energy within 1e-6 relative.
VOXEL_TOL = 1e-3
TOTAL_TOL = 1e-6


def engine(db, ph):
    from paper_1011_2188_gb300 import fdc
    e = fdc.Engine(0)
    e.load_database(db)
    e.load_phantom(ph)
    return e


def gpu_energy(eng, ph, beam, seed, n=0, layers=False, **kw):
    """Run through the C ABI; returns (energy MeV per voxel (float64 numpy),
    raw int64 tally, counters, dose)."""
    import torch
    from paper_1011_2188_gb300 import fdc
    shape = ph.shape[::-1]
    tally = torch.zeros(shape, dtype=torch.int64, device="cuda:0")
    dose = torch.zeros(shape, dtype=torch.float64, device="cuda:0")
    ld = None
    if layers:
        nl = int(np.max(beam["layer"])) + 1
        ld = torch.zeros((nl,) + tuple(shape), dtype=torch.float64, device="cuda:0")
    eng.run_ex(beam, n, seed, tally=tally, dose=dose, layer_dose=ld, **kw)
    cnt = eng.sync()
    t = tally.cpu().numpy()
    out = dict(energy=t.astype(np.float64) / fdc.TALLY_UNITS_PER_MEV, tally=t, counters=cnt,
               dose=dose.cpu().numpy())
    if layers:
        out["layer_dose"] = ld.cpu().numpy()
    return out


def assert_parity(gpu_e, ref_e, what=""):
    mx = float(ref_e.max())
    err = float(np.abs(gpu_e - ref_e).max())
    assert err <= VOXEL_TOL * mx, f"{what}: max voxel error {err / mx:.3g} of max"
    tot = abs(float(gpu_e.sum()) - float(ref_e.sum())) / float(ref_e.sum())
    assert tot <= TOTAL_TOL, f"{what}: total energy error {tot:.3g}"
    return err / mx, tot


def assert_conservation(res):
    c = res["counters"]
    assert int(res["tally"].sum()) + c["escaped"] == c["replayed"], "tally + escaped != replayed"
