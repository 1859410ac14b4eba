"""Pins of the CPU oracle against things fixed outside it (runs without a GPU).

* Philox4x64-10 against numpy's independent implementation of the same
  published generator;
* the sampling of the phase space against the distributions it claims;
* hand-computed tiny transport cases (closed-form expectations);
* water replay of a single track against an independent geometric
  computation of its chords (Sec. 2.2: a water track replayed in water
  reproduces itself);
* exact energy bookkeeping;
* Bragg-Kleeman range in uniform slabs;
* dose conversion and the statistics of eqs. (1) and (2).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import stats
from paper_1011_2188_gb300 import synth
import tiny_cases


# --------------------------------------------------------------------------
# random numbers

def _numpy_philox_block(counter, key):
    """numpy's Philox increments its 256-bit counter before each block, so
    the block for counter c comes from a generator started at c - 1."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(counter))
    c = (c - 1) % (1 << 256)
    start = np.array([(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    return bg.random_raw(4)


@pytest.mark.parametrize("key", [(0, 0), (42, 0), (0xFFFFFFFFFFFFFFFF, 0x123456789ABCDEF0)])
def test_philox_matches_numpy(key):
    rng = np.random.default_rng(5)
    ctrs = [(0, 0, 0, 0), (1, 1, 0, 0), (7, 3, 0, 0), (2**64 - 1, 2, 0, 0)]
    ctrs += [tuple(int(v) for v in rng.integers(0, 2**63, 4, dtype=np.int64)) for _ in range(20)]
    ours = oracle.philox4x64_10(np.array(ctrs, dtype=np.uint64), np.array(key, dtype=np.uint64))
    for c, o in zip(ctrs, ours):
        ref = _numpy_philox_block(c, key)
        assert np.array_equal(o, ref), (c, o, ref)


def _db_multi():
    return synth.water_database([100.0, 150.0, 200.0], 64, seed=3)


def test_sampling_gaussian_profile_and_energy():
    db = _db_multi()
    beam = synth.make_spots([dict(x=1.0, y=-2.0, energy=150.0, sigma_e=1.5, a=0.3,
                                  profile=synth.PROFILE_GAUSS, layer=0, n_histories=100000)])
    f, i = oracle.sample(db, beam, seed=9, h_begin=0, n=100000)
    x, y, E, psi = f.T.astype(np.float64)
    assert abs(x.mean() - 1.0) < 0.005 and abs(x.std() / 0.3 - 1) < 0.01
    assert abs(y.mean() + 2.0) < 0.005 and abs(y.std() / 0.3 - 1) < 0.01
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.01
    assert abs(E.mean() - 150.0) < 0.02 and abs(E.std() / 1.5 - 1) < 0.01
    assert psi.min() >= 0 and psi.max() < 2 * math.pi
    h, _ = np.histogram(psi, bins=16, range=(0, 2 * math.pi))
    chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
    assert chi2 < 40  # 15 dof
    # energy bin: nearest database energy >= E (top bin above the table)
    bins = i[:, 0]
    expect = np.searchsorted(db.energy, f[:, 2], side="left")
    expect = np.minimum(expect, db.n_energies - 1)
    assert np.array_equal(bins, expect)


def test_sampling_rect_and_disk():
    db = _db_multi()
    rect = synth.make_spots([dict(x=0.0, y=0.0, energy=100.0, sigma_e=0.0, a=10.0, b=4.0,
                                  profile=synth.PROFILE_RECT, layer=0, n_histories=50000)])
    f, _ = oracle.sample(db, rect, 1, 0, 50000)
    assert f[:, 0].min() >= -5 and f[:, 0].max() <= 5 and f[:, 1].min() >= -2 and f[:, 1].max() <= 2
    assert abs(f[:, 0].var() / (100 / 12) - 1) < 0.03 and abs(f[:, 1].var() / (16 / 12) - 1) < 0.03
    assert np.all(f[:, 2] == np.float32(100.0))
    disk = synth.make_spots([dict(x=0.0, y=0.0, energy=100.0, sigma_e=0.0, a=4.0,
                                  profile=synth.PROFILE_DISK, layer=0, n_histories=50000)])
    f, _ = oracle.sample(db, disk, 1, 0, 50000)
    r2 = f[:, 0].astype(np.float64) ** 2 + f[:, 1].astype(np.float64) ** 2
    assert r2.max() <= 16.0 + 1e-4
    # r^2 is uniform on [0, R^2]
    assert abs(r2.mean() / 8.0 - 1) < 0.02 and abs(r2.var() / (256 / 12) - 1) < 0.03


def test_sampling_tracks_uniform_and_shared_by_group():
    db = synth.water_database([150.0], 40, seed=3)
    beam = synth.pencil_beam(64000, energy=150.0)
    _, i1 = oracle.sample(db, beam, 4, 0, 64000, track_group=1)
    counts = np.bincount(i1[:, 1], minlength=40)
    chi2 = ((counts - 1600.0) ** 2 / 1600.0).sum()
    assert chi2 < 80  # 39 dof
    _, i32 = oracle.sample(db, beam, 4, 0, 64000, track_group=32)
    t = i32[:, 1].reshape(-1, 32)
    assert np.all(t == t[:, :1])
    assert len(np.unique(t[:, 0])) == 40
    # with one bin and a mono-energetic beam every history starts at step 0
    assert np.all(i1[:, 2] == 0)


def test_sampling_start_step_rule():
    db = synth.water_database([100.0, 150.0], 16, seed=3)
    beam = synth.make_spots([dict(x=0.0, y=0.0, energy=125.0, sigma_e=20.0, a=0.3,
                                  profile=synth.PROFILE_GAUSS, layer=0, n_histories=4000)])
    f, i = oracle.sample(db, beam, 5, 0, 4000)
    E = f[:, 2]
    for n in range(4000):
        b, t, k0 = i[n]
        s0, s1 = db.step_begin[t], db.step_begin[t + 1]
        used = np.concatenate([[0.0], np.cumsum(db.dE[s0:s1].astype(np.float64) + db.esec[s0:s1])])
        eres = (np.float64(db.energy[b]) - used[:-1]).astype(np.float32)
        if E[n] <= 0:
            assert k0 == s1 - s0
            continue
        assert db.track_begin[b] <= t < db.track_begin[b + 1]
        if k0 < s1 - s0:
            assert eres[k0] <= E[n]
        if k0 > 0:
            assert eres[k0 - 1] > E[n]


def test_sampling_spot_order():
    db = _db_multi()
    beam = synth.make_spots([dict(x=0, y=0, energy=e, sigma_e=0, a=0.1, profile=0, layer=k,
                                  n_histories=n) for k, (e, n) in enumerate([(100., 3), (120., 5), (180., 2)])])
    f, _ = oracle.sample(db, beam, 1, 0, 10)
    assert list(f[:, 2]) == [100.0] * 3 + [120.0] * 5 + [180.0] * 2
    f2, _ = oracle.sample(db, beam, 1, 4, 3)
    assert np.array_equal(f2, f[4:7])


# --------------------------------------------------------------------------
# tiny transport cases

@pytest.mark.parametrize("name", sorted(tiny_cases.CASES))
def test_tiny_case(name):
    db, ph, beam, opts, exp = tiny_cases.CASES[name]()
    r = oracle.run(db, ph, beam, seed=1, rotate=False, **opts)
    edep = r.edep.reshape(r.edep.shape[0], -1) if exp.get("layers") else r.edep.reshape(-1)
    tiny_cases.check(edep, r.escaped, r.replayed, exp, atol=1e-9 * 100)
    assert abs(r.edep.sum() + r.escaped - r.replayed) < 1e-9


# --------------------------------------------------------------------------
# water identity: one track replayed in water, checked against its chords

def _chords(db, t, x0, y0, psi):
    """Independent geometry: step end points of track t entering at (x0, y0, 0)
    along +z, with each deflection applied in the frame e2 = z x d / |z x d|,
    e1 = e2 x d (x, y axes at d = +z), the whole track rotated by psi about
    the beam axis afterwards."""
    s0, s1 = db.step_begin[t], db.step_begin[t + 1]
    d = np.array([0.0, 0.0, 1.0])
    p = np.zeros(3)
    pts = [p.copy()]
    for k in range(s0, s1):
        p = p + float(db.len[k]) * d
        pts.append(p.copy())
        th, ph = float(db.theta[k]), float(db.phi[k])
        zc = np.cross([0.0, 0.0, 1.0], d)
        if np.linalg.norm(zc) == 0.0:
            e1, e2 = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
        else:
            e2 = zc / np.linalg.norm(zc)
            e1 = np.cross(e2, d)
        d = math.sin(th) * (math.cos(ph) * e1 + math.sin(ph) * e2) + math.cos(th) * d
    pts = np.array(pts)
    c, s = math.cos(psi), math.sin(psi)
    rot = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
    pts = pts @ rot.T
    pts[:, 0] += x0
    pts[:, 1] += y0
    return pts


def _fine_deposit(ph, db, t, pts, sub=4000):
    """Brute force: cut every chord into ``sub`` equal pieces and give each
    piece its share of the step's energy at its midpoint voxel."""
    nx, ny, nz = ph.shape
    out = np.zeros(ph.nvox)
    s0 = db.step_begin[t]
    o = np.array(ph.origin)
    h = np.array(ph.spacing)
    for k in range(len(pts) - 1):
        a, b = pts[k], pts[k + 1]
        u = (np.arange(sub) + 0.5) / sub
        mid = a[None, :] + u[:, None] * (b - a)[None, :]
        idx = np.floor((mid - o) / h).astype(np.int64)
        v = idx[:, 0] + nx * (idx[:, 1] + ny * idx[:, 2])
        np.add.at(out, v, float(db.dE[s0 + k]) / sub)
        last = np.floor((b - o) / h).astype(np.int64)
        out[last[0] + nx * (last[1] + ny * last[2])] += float(db.esec[s0 + k])
    return out


def test_water_identity_depth_dose_exact():
    """A single water track replayed in water: the z-binned deposits equal
    the energy each chord spends in each z-slab (energy uniform along a
    chord), for any entry point and rotation."""
    db = synth.water_database([100.0], 1, seed=12)
    n = 1 + 2 * 2  # a few histories with different entry points and rotations
    ph = synth.uniform_phantom((40, 40, 45), (0.2, 0.2, 0.2), (-4.0, -4.0, 0.0))
    beam = synth.pencil_beam(n, energy=100.0, sigma_cm=0.3)
    r = oracle.run(db, ph, beam, seed=21)
    assert r.escaped == 0.0
    f, i = oracle.sample(db, beam, 21, 0, n)
    expect = np.zeros(45)
    zb = np.arange(46) * 0.2
    for hh in range(n):
        pts = _chords(db, 0, float(f[hh, 0]), float(f[hh, 1]), float(f[hh, 3]))
        for k in range(len(pts) - 1):
            za, zz = pts[k, 2], pts[k + 1, 2]
            lo, hi = min(za, zz), max(za, zz)
            ov = np.clip(np.minimum(zb[1:], hi) - np.maximum(zb[:-1], lo), 0, None)
            expect += float(db.dE[k]) * ov / (hi - lo)
    got = r.edep.sum(axis=(1, 2))
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-9 * expect.max())


def test_single_history_3d_brute_force():
    """3-D voxel energies of single histories against brute-force chord
    subdivision (pins the x/y/z indexing, the deflection frame and the
    rigid rotation of reused tracks)."""
    db = synth.water_database([60.0], 3, seed=5)
    ph = synth.uniform_phantom((16, 16, 18), (0.2, 0.2, 0.2), (-1.6, -1.6, 0.0))
    beam = synth.pencil_beam(6, energy=60.0, sigma_cm=0.2)
    f, i = oracle.sample(db, beam, 77, 0, 6)
    for hh in range(6):
        r = oracle.run(db, ph, beam, seed=77, h_begin=hh, h_end=hh + 1)
        assert r.escaped == 0.0
        t = int(i[hh, 1])
        pts = _chords(db, t, float(f[hh, 0]), float(f[hh, 1]), float(f[hh, 3]))
        bf = _fine_deposit(ph, db, t, pts)
        # midpoint rule error: at most one sub-piece per voxel face crossing
        step_e = float(db.dE[db.step_begin[t]:db.step_begin[t + 1]].max())
        np.testing.assert_allclose(r.edep.reshape(-1), bf, rtol=0, atol=4 * step_e / 4000)


# --------------------------------------------------------------------------
# energy bookkeeping, Bragg-Kleeman range, sharding

def test_energy_conservation_heterogeneous():
    db = synth.water_database(synth.database_energies(6, 70, 250), 50, seed=8, nuclear=True)
    assert db.esec.max() > 0
    ph = synth.thorax_phantom(seed=3, shape=(48, 48, 40))
    beam = synth.field_beam(3000, energy=150.0, width=8.0, height=8.0)
    r = oracle.run(db, ph, beam, seed=2)
    assert r.escaped > 0 and r.edep.sum() > 0
    assert abs(r.edep.sum() + r.escaped - r.replayed) <= 1e-12 * r.replayed


def test_bragg_kleeman_slabs():
    """Unscattered protons in uniform slabs stop where the water-equivalent
    depth sum_i t_i S_i equals the Bragg-Kleeman range alpha E^p, and each
    voxel receives the energy the track loses over its water-equivalent
    interval."""
    E0 = 100.0
    db = synth.water_database([E0], 1, seed=1, scatter=False)
    layers = [(10, synth.MAT_WATER, 1.0), (10, synth.MAT_BONE, 1.85), (20, synth.MAT_LUNG, 0.25),
              (20, synth.MAT_WATER, 1.0)]
    ph = synth.slabs_phantom((1, 1, 60), (2.0, 2.0, 0.2), layers)
    beam = synth.pencil_beam(3, energy=E0, sigma_cm=0.0)
    r = oracle.run(db, ph, beam, seed=1)
    S = (ph.density[:, 0, 0].astype(np.float64) * ph.s_rel[ph.material[:, 0, 0]].astype(np.float64))
    w_edges = np.concatenate([[0.0], np.cumsum(S * 0.2)])
    R = synth.BK_ALPHA * E0 ** synth.BK_P
    # closed form: stopping depth
    iz_stop = np.searchsorted(w_edges, R) - 1
    z_stop = 0.2 * iz_stop + (R - w_edges[iz_stop]) / S[iz_stop]
    got = r.edep[:, 0, 0]
    assert got[iz_stop] > 0 and np.all(got[iz_stop + 1:] == 0)
    # deepest deposit matches the closed-form stopping point within a voxel fraction
    total_wet = float(np.sum(db.len.astype(np.float64)))
    assert abs(total_wet - R) < 1e-5 * R
    # per-voxel energies: energy lost along the track between the voxel's
    # water-equivalent edges (piecewise-linear in water-equivalent depth)
    cum_w = np.concatenate([[0.0], np.cumsum(db.len.astype(np.float64))])
    cum_e = np.concatenate([[0.0], np.cumsum(db.dE.astype(np.float64))])
    e_at = np.interp(np.minimum(w_edges, cum_w[-1]), cum_w, cum_e)
    expect = 3 * np.diff(e_at)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-9 * expect.max())
    assert 0.0 < z_stop < 12.0


def test_sharding_adds_up():
    db, ph, beam = synth.workload_slab(n_histories=3000, n_tracks=200)
    full = oracle.run(db, ph, beam, seed=3)
    a = oracle.run(db, ph, beam, seed=3, h_begin=0, h_end=1234)
    b = oracle.run(db, ph, beam, seed=3, h_begin=1234, h_end=3000)
    np.testing.assert_allclose(a.edep + b.edep, full.edep, rtol=1e-12, atol=1e-9)
    assert a.n_steps + b.n_steps == full.n_steps


# --------------------------------------------------------------------------
# dose conversion and statistics

def test_dose_conversion_hand_arithmetic():
    ph = tiny_cases.grid(rho_by_z=(1.0, 2.0, 0.0))
    e = np.zeros(12)
    e[0] = 1.0      # 1 MeV in 1 g of water
    e[4] = 1.0      # 1 MeV in 2 g
    e[8] = 5.0      # no mass
    d = oracle.dose(ph, e)
    assert d[0] == pytest.approx(1.602176634e-13 / 1e-3, rel=1e-15)
    assert d[4] == pytest.approx(0.5 * 1.602176634e-10, rel=1e-15)
    assert d[8] == 0.0


def test_batch_sigma_matches_numpy():
    rng = np.random.default_rng(0)
    b = rng.normal(5.0, 0.3, size=(7, 100))
    mean, sig = stats.batch_sigma(b)
    np.testing.assert_allclose(sig, np.std(b, axis=0, ddof=1) / np.sqrt(7), rtol=1e-12)
    m2, s2 = stats.batch_sigma_from_sums(b.sum(0), (b * b).sum(0), 7)
    np.testing.assert_allclose(m2, mean, rtol=1e-12)
    np.testing.assert_allclose(s2, sig, rtol=1e-9)


def test_history_sigma_matches_numpy():
    rng = np.random.default_rng(1)
    d = rng.exponential(2.0, size=(5000, 30))
    s = stats.history_sigma(d.sum(0), (d * d).sum(0), 5000)
    np.testing.assert_allclose(s, np.std(d, axis=0, ddof=1) / np.sqrt(5000), rtol=1e-9)


def test_mean_relative_uncertainty():
    dose = np.array([1.0, 10.0, 6.0, 4.0])
    sig = np.array([1.0, 1.0, 0.6, 10.0])
    assert stats.mean_relative_uncertainty(dose, sig) == pytest.approx(0.1)


def test_batch_uncertainty_scales_as_inverse_sqrt_n():
    """Sec. 2.4 / Fig. 5: the batch uncertainty follows C / sqrt(N)."""
    db = synth.water_database([121.0], 200, seed=4)
    ph = synth.slab_phantom(n=32, voxel_cm=0.4)
    res = {}
    for n_per in (500, 2000):
        beam = synth.disk_beam(n_per * 8, energy=121.0, radius=1.5)
        d = []
        for b in range(8):
            r = oracle.run(db, ph, beam, seed=100, h_begin=b * n_per, h_end=(b + 1) * n_per)
            d.append(r.edep.reshape(-1) / n_per)
        mean, sig = stats.batch_sigma(np.array(d))
        res[n_per] = stats.mean_relative_uncertainty(mean, sig)
    ratio = res[500] / res[2000]
    assert 1.6 < ratio < 2.5, ratio


def test_history_squares_exact():
    """The oracle's per-history sums of squares equal the squares of single
    history runs added up."""
    db = synth.water_database([80.0], 5, seed=2)
    ph = synth.slab_phantom(n=16, voxel_cm=0.3)
    beam = synth.pencil_beam(6, energy=80.0, sigma_cm=0.3)
    r = oracle.run(db, ph, beam, seed=8, history_squares=True)
    sq = np.zeros_like(r.edep)
    for hh in range(6):
        one = oracle.run(db, ph, beam, seed=8, h_begin=hh, h_end=hh + 1)
        sq += one.edep ** 2
    np.testing.assert_allclose(r.hh_sumsq, sq, rtol=1e-12, atol=1e-12)


def test_visit_squares_of_a_back_scattered_track():
    """Per-visit squares by hand on the back-scattering tiny case: the track
    deposits 2 MeV in voxel 0, 1 MeV in voxel 4, turns round, deposits
    2 t_a more in voxel 4 (the same visit: no other voxel in between), then
    2 (1 - t_a) and 2 t_b in voxel 0 -- a second visit of voxel 0.  The
    per-history squares see one (summed) visit per voxel."""
    import math
    db, ph, beam, opts, exp = tiny_cases.CASES["backscatter"]()
    r = oracle.run(db, ph, beam, seed=1, rotate=False, history_squares=True, visit_squares=True, **opts)
    c = -math.cos(tiny_cases.THETA_180)
    t_a = 0.5 / c
    z2 = 1.0 - (1.0 - t_a) * c
    t_b = z2 / c
    back = 2.0 * (1.0 - t_a) + 2.0 * t_b
    hv, hh = r.hv_sumsq.reshape(-1), r.hh_sumsq.reshape(-1)
    assert hv[0] == pytest.approx(2.0 ** 2 + back ** 2, rel=1e-12)
    assert hv[4] == pytest.approx((1.0 + 2.0 * t_a) ** 2, rel=1e-12)
    assert hh[0] == pytest.approx((2.0 + back) ** 2, rel=1e-12)
    assert hh[4] == pytest.approx(hv[4], rel=1e-12)
    assert np.count_nonzero(hv) == 2


def test_visit_squares_equal_history_squares_without_reentry():
    """Straight tracks along the axis enter every voxel once: the per-visit
    and per-history squares coincide; with scattering (voxels re-entered)
    the visit squares are never larger, voxel by voxel (a sum of squares of
    non-negative parts is at most the square of their sum)."""
    db = synth.water_database([100.0], 20, seed=4, scatter=False)
    ph = synth.slab_phantom(n=24, voxel_cm=0.4)
    beam = synth.pencil_beam(300, energy=100.0, sigma_cm=0.5)
    r = oracle.run(db, ph, beam, seed=3, history_squares=True, visit_squares=True)
    np.testing.assert_allclose(r.hv_sumsq, r.hh_sumsq, rtol=1e-12, atol=0)
    db = synth.water_database([100.0], 20, seed=4)
    r = oracle.run(db, ph, beam, seed=3, history_squares=True, visit_squares=True)
    assert np.all(r.hv_sumsq <= r.hh_sumsq * (1 + 1e-12))
    assert r.hv_sumsq.sum() < r.hh_sumsq.sum()


def test_per_layer_tallies_partition_the_run():
    """Per-layer tallies (a history scores into its spot's layer): the layers
    add up to the plain run, and each layer equals a run over exactly the
    histories of its spots (histories are numbered over the spots in order)."""
    db = synth.water_database([120.0, 150.0], 60, seed=3)
    ph = synth.slab_phantom()
    beam = synth.make_spots([
        dict(x=-0.5, y=0.0, energy=120.0, sigma_e=0.0, a=0.3, profile=synth.PROFILE_GAUSS, layer=0, n_histories=300),
        dict(x=0.5, y=0.2, energy=118.0, sigma_e=0.0, a=0.3, profile=synth.PROFILE_GAUSS, layer=0, n_histories=200),
        dict(x=0.0, y=-0.4, energy=150.0, sigma_e=0.0, a=0.2, profile=synth.PROFILE_GAUSS, layer=1, n_histories=400),
    ])
    per = oracle.run(db, ph, beam, seed=21, per_layer=True)
    whole = oracle.run(db, ph, beam, seed=21)
    assert per.edep.shape[0] == 2
    np.testing.assert_allclose(per.edep.sum(axis=0), whole.edep, rtol=1e-12, atol=1e-9)
    first = oracle.run(db, ph, beam, seed=21, h_begin=0, h_end=500)
    second = oracle.run(db, ph, beam, seed=21, h_begin=500, h_end=900)
    np.testing.assert_allclose(per.edep[0], first.edep, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(per.edep[1], second.edep, rtol=1e-12, atol=1e-9)
    assert per.edep[1][:, :, :].sum() > 0 and per.edep[0].sum() > 0
