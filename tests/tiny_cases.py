"""Tiny hand-checkable transport cases (inputs and closed-form expectations).

Grid: 2 x 2 x 3 voxels of 1 cm, origin (-1, -1, 0); voxel index
v = ix + 2 iy + 4 iz.  Material 0: s_rel = 1, k_theta = 1; material 1:
s_rel = 1, k_theta = 2.  Every proton enters at z = 0 along +z with the bin
energy unless stated, from a zero-width rectangle (exact entry point), and
tracks are replayed unrotated (psi = 0), so each case is a fixed path whose
voxel energies follow from elementary geometry:

* step lengths are water-equivalent; in a voxel of density rho and s_rel 1 a
  geometric length g consumes g * rho (Sec. 2.2: step length scaled by the
  material);
* a step's energy loss is shared among the voxels it crosses in proportion
  to the water-equivalent length consumed in each;
* the deflection at the end of a step is theta * sqrt(sum_i w_i k_i^2)
  (scattering angle scaled by the material), azimuth phi measured from +x
  when the direction is +z;
* esec goes to the voxel where the step ends; leaving the grid ends the
  history and the rest of its energy is "escaped".

Each case returns (database, phantom, beam, options, expected) where
expected = {"edep": {v: MeV}, "escaped": MeV, "replayed": MeV, "layers": bool}.
"""
from __future__ import annotations

import math

import numpy as np

from paper_1011_2188_gb300 import synth

THETA_90 = 1.5703125      # pi/2 rounded to half precision
THETA_180 = 3.140625      # pi rounded to half precision
PHI_45 = float(np.float32(8192 * 2.0 * math.pi / 65536))


def grid(rho_by_z=(1.0, 1.0, 1.0), mat_by_z=(0, 0, 0)):
    ph = synth.Phantom(shape=(2, 2, 3), spacing=(1.0, 1.0, 1.0), origin=(-1.0, -1.0, 0.0),
                       material=np.zeros((3, 2, 2), np.uint8), density=np.ones((3, 2, 2), np.float32),
                       s_rel=np.array([1.0, 1.0], np.float32), k_theta=np.array([1.0, 2.0], np.float32))
    for iz in range(3):
        ph.density[iz] = rho_by_z[iz]
        ph.material[iz] = mat_by_z[iz]
    return ph


def beam_at(x, y, energies=(100.0,)):
    rows = [dict(x=x, y=y, energy=e, sigma_e=0.0, a=0.0, b=0.0, profile=synth.PROFILE_RECT,
                 layer=i, n_histories=1) for i, e in enumerate(energies)]
    return synth.make_spots(rows)


def one_track(steps, energy=100.0):
    return synth.database_from_tracks([energy], [[steps]])


def f32(x):
    return float(np.float32(x))


def _straight_water():
    db = one_track([(10.0, 2.5, 0.0, 0.0, 0.0)])
    exp = {3: 4.0, 7: 4.0, 11: 2.0}
    return db, grid(), beam_at(0.5, 0.5), {}, dict(edep=exp, escaped=0.0, replayed=10.0)


def _density_scaling():
    db = one_track([(12.0, 2.25, 0.0, 0.0, 0.0), (6.0, 0.5, 0.0, 0.0, 0.0)])
    ph = grid(rho_by_z=(2.0, 0.5, 1.0))
    # step 1: 1 cm at rho 2 -> 2.0 of 2.25; the last 0.25 at rho 0.5 -> 0.5 cm (z = 1.5)
    # step 2: 0.5 cm to z = 2 at rho 0.5 -> 0.25 of 0.5; the other 0.25 in iz = 2
    exp = {3: 12.0 * 2.0 / 2.25, 7: 12.0 * 0.25 / 2.25 + 3.0, 11: 3.0}
    return db, ph, beam_at(0.5, 0.5), {}, dict(edep=exp, escaped=0.0, replayed=18.0)


def _start_voxel_scaling():
    db = one_track([(12.0, 2.25, 0.0, 0.0, 0.0), (6.0, 0.5, 0.0, 0.0, 0.0)])
    ph = grid(rho_by_z=(2.0, 0.5, 1.0))
    # mode 1: the whole step uses the scaling of its start voxel.
    # step 1 (S = 2): 1 cm in iz0 consumes 2.0, 0.125 cm in iz1 the last 0.25 (z = 1.125)
    # step 2 (S = 0.5): geometric length 1 cm: 0.875 in iz1, 0.125 in iz2
    exp = {3: 12.0 * 2.0 / 2.25, 7: 12.0 * 0.25 / 2.25 + 6.0 * 0.875, 11: 6.0 * 0.125}
    return db, ph, beam_at(0.5, 0.5), {"scaling_mode": 1}, dict(edep=exp, escaped=0.0, replayed=18.0)


def _deflect_90():
    db = one_track([(1.0, 0.5, THETA_90, 0.0, 0.0), (4.0, 1.0, 0.0, 0.0, 0.0)])
    # after step 1 the direction is (sin T, 0, cos T); step 2 leaves ix = 0 after 0.5 / sin T
    tx = 0.5 / math.sin(THETA_90)
    exp = {0: 1.0 + 4.0 * tx, 1: 4.0 * (1.0 - tx)}
    return db, grid(), beam_at(-0.5, -0.5), {}, dict(edep=exp, escaped=0.0, replayed=5.0)


def _corner():
    db = one_track([(1.0, 0.5, THETA_90, PHI_45, 0.0), (4.0, 1.0, 0.0, 0.0, 0.0)])
    s = math.sin(THETA_90)
    dx, dy = s * math.cos(PHI_45), s * math.sin(PHI_45)
    t1, t2 = 0.5 / max(dx, dy), 0.5 / min(dx, dy)
    # segments: (0,0,0) until t1, a (near) zero-length piece in (1,0,0) or
    # (0,1,0) until t2, then (1,1,0)
    exp = {0: 1.0 + 4.0 * t1, 3: 4.0 * (1.0 - t2), "mid": ((1, 2), 4.0 * (t2 - t1))}
    return db, grid(), beam_at(-0.5, -0.5), {}, dict(edep=exp, escaped=0.0, replayed=5.0)


def _k_theta_scaling():
    db = one_track([(1.0, 0.5, 0.5, 0.0, 0.0), (4.0, 1.0, 0.0, 0.0, 0.0)])
    ph = grid(mat_by_z=(1, 0, 0))
    tm = 0.5 * math.sqrt(0.5 * 4.0 / 0.5)        # = 1.0: all of step 1 in k_theta = 2
    tx, tz = 0.5 / math.sin(tm), 0.5 / math.cos(tm)
    exp = {0: 1.0 + 4.0 * tx, 1: 4.0 * (tz - tx), 5: 4.0 * (1.0 - tz)}
    return db, ph, beam_at(-0.5, -0.5), {}, dict(edep=exp, escaped=0.0, replayed=5.0)


def _mixed_k_theta():
    db = one_track([(1.0, 0.5, 0.0, 0.0, 0.0), (2.0, 1.0, 0.25, 0.0, 0.0), (4.0, 1.0, 0.0, 0.0, 0.0)])
    ph = grid(mat_by_z=(1, 0, 0))
    tm = 0.25 * math.sqrt((0.5 * 4.0 + 0.5 * 1.0) / 1.0)   # step 2 half in each material
    tz = 0.5 / math.cos(tm)
    assert 0.5 / math.sin(tm) > 1.0
    exp = {0: 1.0 + 1.0, 4: 1.0 + 4.0 * tz, 8: 4.0 * (1.0 - tz)}
    return db, ph, beam_at(-0.5, -0.5), {}, dict(edep=exp, escaped=0.0, replayed=7.0)


def _esec_end():
    db = one_track([(3.0, 1.5, 0.0, 0.0, 0.7)])
    exp = {3: 2.0, 7: 1.0 + f32(0.7)}
    return db, grid(), beam_at(0.5, 0.5), {}, dict(edep=exp, escaped=0.0, replayed=3.0 + f32(0.7))


def _escape():
    db = one_track([(8.0, 4.0, 0.0, 0.0, 1.0), (5.0, 1.0, 0.0, 0.0, 0.5)])
    exp = {3: 2.0, 7: 2.0, 11: 2.0}
    return db, grid(), beam_at(0.5, 0.5), {}, dict(edep=exp, escaped=2.0 + 1.0 + 5.5, replayed=14.5)


def _backscatter():
    db = one_track([(3.0, 1.5, THETA_180, 0.0, 0.0), (2.0, 1.0, 0.0, 0.0, 0.0), (2.0, 1.0, 0.0, 0.0, 0.0)])
    c = -math.cos(THETA_180)                 # |dz| after the reversal
    t_a = 0.5 / c                           # step 2: z 1.5 -> 1 in iz1
    z2 = 1.0 - (1.0 - t_a) * c              # end of step 2 in iz0
    t_b = z2 / c                            # step 3 reaches z = 0 and leaves
    exp = {0: 2.0 + 2.0 * (1.0 - t_a) + 2.0 * t_b, 4: 1.0 + 2.0 * t_a}
    return db, grid(), beam_at(-0.5, -0.5), {}, dict(edep=exp, escaped=2.0 * (1.0 - t_b), replayed=7.0)


def _start_step():
    db = synth.database_from_tracks(
        [60.0, 100.0],
        [[[(60.0, 0.5, 0.0, 0.0, 0.0)]],
         [[(10.0, 0.7, 0.0, 0.0, 0.0), (20.0, 0.7, 0.0, 0.0, 0.0), (30.0, 0.7, 0.0, 0.0, 0.0),
           (40.0, 0.7, 0.0, 0.0, 0.0)]]])
    # layer 0: E = 75 -> bin 100; residual energies 100, 90, 70, 40 -> start at step 2
    # layer 1: E = 120 above the top bin -> bin 100, start at step 0
    # layer 2: E = 55 -> bin 60; residual 60 > 55 -> nothing to replay
    # layer 3: E = 60 -> bin 60, start at step 0
    L = f32(0.7)  # stored step length; steps end at z = L, 2L, ...
    layers = {
        0: {3: 30.0 + 40.0 * (1.0 - L) / L, 7: 40.0 * (2 * L - 1.0) / L},
        1: {3: 10.0 + 20.0 * (1.0 - L) / L, 7: 20.0 * (2 * L - 1.0) / L + 30.0 * (2.0 - 2 * L) / L,
            11: 30.0 * (3 * L - 2.0) / L + 40.0},
        2: {},
        3: {3: 60.0},
    }
    return (db, grid(), beam_at(0.5, 0.5, energies=(75.0, 120.0, 55.0, 60.0)), {"per_layer": True},
            dict(edep=layers, escaped=0.0, replayed=70.0 + 100.0 + 0.0 + 60.0, layers=True))


def _miss():
    db = one_track([(10.0, 2.5, 0.0, 0.0, 0.0)])
    return db, grid(), beam_at(1.5, 0.5), {}, dict(edep={}, escaped=10.0, replayed=10.0)


CASES = {
    "straight_water": _straight_water,
    "density_scaling": _density_scaling,
    "start_voxel_scaling": _start_voxel_scaling,
    "deflect_90": _deflect_90,
    "corner": _corner,
    "k_theta_scaling": _k_theta_scaling,
    "mixed_k_theta": _mixed_k_theta,
    "esec_end": _esec_end,
    "escape": _escape,
    "backscatter": _backscatter,
    "start_step": _start_step,
    "miss": _miss,
}


def check(edep_flat_or_layers, escaped, replayed, expected, atol=2e-5):
    """Compare a run's voxel energies (flat [nvox] or [n_layers, nvox]) with
    a case's expectations; unnamed voxels must be ~0."""
    def check_one(e, exp):
        e = np.asarray(e, np.float64).reshape(-1).copy()
        mid = exp.get("mid")
        for v, val in exp.items():
            if v == "mid":
                continue
            assert abs(e[v] - val) <= atol, (v, e[v], val)
            e[v] = 0.0
        if mid is not None:
            cand, val = mid
            assert abs(sum(e[c] for c in cand) - val) <= atol
            for c in cand:
                e[c] = 0.0
        assert np.all(np.abs(e) <= atol), np.nonzero(np.abs(e) > atol)

    if expected.get("layers"):
        for layer, exp in expected["edep"].items():
            check_one(edep_flat_or_layers[layer], exp)
    else:
        check_one(edep_flat_or_layers, expected["edep"])
    assert abs(escaped - expected["escaped"]) <= atol, (escaped, expected["escaped"])
    assert abs(replayed - expected["replayed"]) <= atol * max(1.0, expected["replayed"]), (replayed, expected["replayed"])
