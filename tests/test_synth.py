"""Pins of the synthetic input generators (no GPU)."""
import math

import numpy as np
import pytest

from paper_1011_2188_gb300 import synth


def test_bragg_kleeman_track_closed_form():
    """Without straggling a track's lengths add up to R(E0) = alpha E0^p and
    its energy losses to E0 (continuous slowing down, 1 mm steps)."""
    for E0 in (70.0, 150.0, 250.0):
        db = synth.water_database([E0], 3, seed=1, scatter=False)
        s0, s1 = db.step_begin[0], db.step_begin[1]
        R = synth.BK_ALPHA * E0 ** synth.BK_P
        assert abs(db.len[s0:s1].astype(np.float64).sum() - R) < 2e-6 * R
        assert abs(db.dE[s0:s1].astype(np.float64).sum() - E0) < 2e-6 * E0
        assert s1 - s0 == math.ceil(R / 0.1 - 1e-9)
        assert np.all(db.len[s0:s1 - 1] == np.float32(0.1))
        # energy after k steps follows the range-energy relation
        E = E0 - np.cumsum(db.dE[s0:s1].astype(np.float64))
        Rk = R - np.cumsum(db.len[s0:s1].astype(np.float64))
        np.testing.assert_allclose(E[:-1], (np.maximum(Rk[:-1], 0) / synth.BK_ALPHA) ** (1 / synth.BK_P),
                                   rtol=0, atol=2e-6 * E0)


def test_highland_width():
    """First-step deflections: theta_x, theta_y ~ N(0, theta0) so E[theta^2]
    = 2 theta0^2 with theta0 the PDG Highland width at E0 for 1 mm of water."""
    E0 = 150.0
    db = synth.water_database([E0], 100000, seed=3)
    first = db.theta[db.step_begin[:-1]].astype(np.float64)
    pc2 = E0 * E0 + 2 * E0 * 938.272
    bcp = pc2 / (E0 + 938.272)
    x = 0.1 / 36.08
    th0 = 13.6 / bcp * math.sqrt(x) * (1 + 0.038 * math.log(x))
    assert abs(np.mean(first ** 2) / (2 * th0 ** 2) - 1) < 0.01
    phi = db.phi[db.step_begin[:-1]]
    assert phi.min() >= -math.pi and phi.max() <= math.pi
    assert abs(np.mean(np.cos(phi))) < 0.01


@pytest.mark.parametrize("kw", [{}, {"straggling": True, "nuclear": True}])
def test_angles_are_not_rounded_to_a_storage_grid(kw):
    """The generator emits FP32 angles as computed: almost none sits on the
    IEEE-half grid or on a multiple of 2 pi / 65536 (a record format that
    stored them on such grids would have to round them)."""
    db = synth.water_database([100.0, 150.0], 200, seed=2, **kw)
    th = db.theta[db.theta > 0]
    on_half = th.astype(np.float16).astype(np.float32) == th
    assert on_half.mean() < 0.01
    code = db.phi.astype(np.float64) / (2 * math.pi / 65536)
    assert np.mean(np.abs(code - np.rint(code)) < 1e-3) < 0.01
    assert db.theta.dtype == np.float32 and db.phi.dtype == np.float32


def test_phantoms_and_plan():
    ph = synth.slab_phantom()
    assert ph.shape == (64, 64, 64) and ph.density[25, 0, 0] == np.float32(1.85)
    assert ph.density[19, 0, 0] == 1.0 and ph.density[30, 0, 0] == 1.0
    th = synth.thorax_phantom(seed=7, shape=(64, 64, 32), voxel_cm=0.8)
    for m in range(4):
        assert np.any(th.material == m)
    lung = th.density[th.material == synth.MAT_LUNG]
    assert lung.min() >= 0.2 and lung.max() <= 0.3
    plan = synth.spot_plan(total=2_000_000, n_layers=40, spots_per_layer=50)
    assert len(plan) == 2000 and int(plan["n_histories"].sum()) == 2_000_000
    assert set(np.unique(plan["layer"])) == set(range(40))
    assert plan["energy"].min() == 70.0 and plan["energy"].max() == 230.0
