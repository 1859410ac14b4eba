"""Seeded synthetic inputs for the track-repeating dose engine.

This module generates the *inputs* of the method -- the water track database,
the voxel phantoms and the beam (spot) lists -- and nothing else.  It holds
none of the track-repeating arithmetic (no step scaling, no voxel traversal,
no tallying, no random draws of the replay itself) and imports nothing from
the rest of the package, so the CUDA path and the CPU oracle can both be fed
from it without sharing any of the method.

Stand-ins for the paper's inputs (the paper's GEANT4 water database and its
thorax CT are not available, Sec. 2.1, 2.2, 2.5):

* ``water_database``: a seeded condensed-history simulation of protons in
  water with 1 mm steps.  Energy loss per step follows the Bragg-Kleeman
  range-energy relation R(E) = alpha * E**p exactly (CSDA, optional Gaussian
  straggling); the polar deflection at the end of each step is drawn from the
  Highland width (PDG form) using the energy at the step start.  Each step
  record holds what Sec. 2.2 says the database stores per step (direction
  change, length, energy loss) plus the energy deposited locally by
  secondaries (zero unless the optional local-deposit model is enabled).
* ``slab_phantom``: water cube with a bone slab (64^3 voxels of 2 mm).
* ``thorax_phantom``: thorax-like heterogeneous phantom built from random
  ellipsoids (body outline, lungs, spine, ribs), 256x256x128 voxels of 2 mm.
* ``pencil_beam`` / ``field_beam`` / ``spot_plan``: beam descriptions.

The deflection angles are emitted as the generator computes them (FP32
theta in [0, pi], phi = atan2 in [-pi, pi]), on no storage grid: whatever
packing a consumer uses is its own business, and the oracle reads the values
as given.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Bragg-Kleeman constants for water (alpha in cm/MeV^p).
BK_ALPHA = 0.0022
BK_P = 1.77
# Proton rest energy (MeV) and radiation length of water (cm).
M_P = 938.272
X_WATER = 36.08
STEP_CM = 0.1

# Synthetic material table: (name, mass stopping-power ratio to water,
# radiation-length ratio X_water/X_material (mass units)).  These are this
# project's constants, not the paper's.  The scattering-power ratio is
# k_theta = sqrt(xratio / s_rel): the Highland variance scales as the
# geometric length over the radiation length, and density cancels between the
# two.
MATERIALS = (
    ("air", 0.88, 0.99),
    ("water", 1.00, 1.00),
    ("lung", 0.99, 1.00),
    ("bone", 0.90, 1.30),
)
MAT_AIR, MAT_WATER, MAT_LUNG, MAT_BONE = 0, 1, 2, 3


def material_tables():
    """Return (s_rel, k_theta) float32 arrays for ``MATERIALS``."""
    s_rel = np.array([m[1] for m in MATERIALS], dtype=np.float32)
    xr = np.array([m[2] for m in MATERIALS], dtype=np.float64)
    k_theta = np.sqrt(xr / s_rel.astype(np.float64)).astype(np.float32)
    return s_rel, k_theta


def bk_range(E):
    return BK_ALPHA * np.power(E, BK_P)


def bk_energy(R):
    return np.power(np.maximum(R, 0.0) / BK_ALPHA, 1.0 / BK_P)


def highland_theta0(E, step):
    """PDG Highland width (rad) for a proton of kinetic energy E (MeV) after
    ``step`` cm of water."""
    pc2 = E * E + 2.0 * E * M_P
    beta_cp = pc2 / (E + M_P)
    x = step / X_WATER
    corr = np.maximum(1.0 + 0.038 * np.log(np.maximum(x, 1e-300)), 0.0)
    return 13.6 / np.maximum(beta_cp, 1e-12) * np.sqrt(x) * corr


@dataclass
class Database:
    energy: np.ndarray       # float32 [n_energies], strictly increasing (MeV)
    track_begin: np.ndarray  # int64 [n_energies + 1] CSR into tracks
    step_begin: np.ndarray   # int64 [n_tracks + 1] CSR into steps
    dE: np.ndarray           # float32 [n_steps] MeV (ionisation along the step)
    len: np.ndarray          # float32 [n_steps] cm of water
    theta: np.ndarray        # float32 [n_steps] polar deflection at step end (rad)
    phi: np.ndarray          # float32 [n_steps] azimuth of that deflection (rad)
    esec: np.ndarray         # float32 [n_steps] MeV deposited locally at step end

    @property
    def n_energies(self):
        return int(self.energy.shape[0])

    @property
    def n_tracks(self):
        return int(self.step_begin.shape[0] - 1)

    @property
    def n_steps(self):
        return int(self.dE.shape[0])

    def nbytes(self):
        return sum(a.nbytes for a in (self.energy, self.track_begin, self.step_begin,
                                      self.dE, self.len, self.theta, self.phi, self.esec))


def _simulate_bin(E0, n_tracks, rng, step_cm, scatter, straggling, nuclear):
    """Condensed-history protons of energy E0 in water; returns per-track
    ragged columns as a list of per-step arrays plus per-track step counts."""
    E = np.full(n_tracks, float(E0))
    alive = np.ones(n_tracks, dtype=bool)
    cols = []  # (alive_idx, dE, len, theta, phi, esec)
    guard = 0
    while alive.any():
        guard += 1
        if guard > 100000:
            raise RuntimeError("water_database: runaway track")
        idx = np.nonzero(alive)[0]
        e = E[idx]
        R = bk_range(e)
        ln = np.minimum(step_cm, R)
        last = ln >= R
        e_new = np.where(last, 0.0, bk_energy(R - ln))
        de = e - e_new
        if straggling:
            # Gaussian energy-loss straggling with Bohr's variance in water
            # (0.157 * Z/A MeV^2 per g/cm^2), kept inside [0, e].
            sig = np.sqrt(0.157 * 0.5551 * ln)
            de = np.clip(de + sig * rng.standard_normal(idx.size), 0.0, e)
            e_new = np.where(last, 0.0, e - de)
            de = np.where(last, e, de)
        esec = np.zeros_like(de)
        if nuclear:
            # Optional local-deposit model: non-elastic interaction with
            # probability 0.012 per cm of water above 10 MeV; the primary
            # stops and a fraction U(0.1, 0.4) of its remaining energy is
            # deposited locally, the rest is carried away.
            p_int = np.where(e > 10.0, 1.0 - np.exp(-0.012 * ln), 0.0)
            hit = (rng.random(idx.size) < p_int) & ~last
            frac = rng.uniform(0.1, 0.4, idx.size)
            esec = np.where(hit, frac * e_new, 0.0)
            last = last | hit
            e_new = np.where(hit, 0.0, e_new)
        if scatter:
            th0 = highland_theta0(e, ln)
            tx = rng.standard_normal(idx.size) * th0
            ty = rng.standard_normal(idx.size) * th0
            theta = np.hypot(tx, ty)
            phi = np.arctan2(ty, tx)
        else:
            theta = np.zeros_like(e)
            phi = np.zeros_like(e)
        cols.append((idx, de, ln, theta, phi, esec))
        E[idx] = e_new
        alive[idx[last]] = False
    n_steps = np.zeros(n_tracks, dtype=np.int64)
    for c in cols:
        n_steps[c[0]] += 1
    return cols, n_steps


def water_database(energies, n_tracks, seed, step_cm=STEP_CM, scatter=True,
                   straggling=False, nuclear=False) -> Database:
    """Seeded water track database: ``n_tracks`` tracks per energy (MeV)."""
    energies = np.asarray(energies, dtype=np.float64).reshape(-1)
    if np.any(np.diff(energies) <= 0):
        raise ValueError("energies must be strictly increasing")
    rng = np.random.Generator(np.random.PCG64(seed))
    if not straggling and not nuclear:
        return _water_database_csda(energies, n_tracks, rng, step_cm, scatter)
    per_bin = []
    total_steps = 0
    for E0 in energies:
        cols, n_steps = _simulate_bin(float(np.float32(E0)), n_tracks, rng, step_cm,
                                      scatter, straggling, nuclear)
        per_bin.append((cols, n_steps))
        total_steps += int(n_steps.sum())
    n_all = len(energies) * n_tracks
    step_begin = np.zeros(n_all + 1, dtype=np.int64)
    arrays = {k: np.empty(total_steps, dtype=np.float32) for k in ("dE", "len", "theta", "phi", "esec")}
    t0 = 0
    for cols, n_steps in per_bin:
        starts = np.concatenate([[0], np.cumsum(n_steps)]) + step_begin[t0]
        step_begin[t0:t0 + n_tracks + 1] = starts
        fill = np.zeros(n_tracks, dtype=np.int64)
        for (idx, de, ln, theta, phi, esec) in cols:
            pos = starts[idx] + fill[idx]
            arrays["dE"][pos] = de
            arrays["len"][pos] = ln
            arrays["theta"][pos] = np.minimum(theta, math.pi)
            arrays["phi"][pos] = phi
            arrays["esec"][pos] = esec
            fill[idx] += 1
        t0 += n_tracks
    track_begin = np.arange(len(energies) + 1, dtype=np.int64) * n_tracks
    return Database(energy=energies.astype(np.float32), track_begin=track_begin,
                    step_begin=step_begin, **arrays)


def _csda_steps(E0, step_cm):
    """Deterministic continuous-slowing-down steps of a proton of energy E0:
    (energy at step start, length, energy loss) per step."""
    e_start, lens, des = [], [], []
    e = float(E0)
    while True:
        R = BK_ALPHA * e ** BK_P
        ln = min(step_cm, R)
        last = ln >= R
        e_new = 0.0 if last else ((R - ln) / BK_ALPHA) ** (1.0 / BK_P)
        e_start.append(e)
        lens.append(ln)
        des.append(e - e_new)
        if last:
            break
        e = e_new
    return np.array(e_start), np.array(lens), np.array(des)


def _water_database_csda(energies, n_tracks, rng, step_cm, scatter, chunk=20000):
    """Fast path without straggling or local deposits: every track of a bin
    has the same lengths and energy losses; only the deflections differ."""
    per_bin = [_csda_steps(float(np.float32(E0)), step_cm) for E0 in energies]
    n_steps = [len(b[0]) for b in per_bin]
    total = sum(n * n_tracks for n in n_steps)
    arrays = {k: np.empty(total, dtype=np.float32) for k in ("dE", "len", "theta", "phi", "esec")}
    arrays["esec"][:] = 0.0
    step_begin = np.empty(len(energies) * n_tracks + 1, dtype=np.int64)
    pos = 0
    t0 = 0
    for (e_start, lens, des), n in zip(per_bin, n_steps):
        step_begin[t0:t0 + n_tracks] = pos + n * np.arange(n_tracks, dtype=np.int64)
        blk = slice(pos, pos + n * n_tracks)
        arrays["dE"][blk] = np.tile(des.astype(np.float32), n_tracks)
        arrays["len"][blk] = np.tile(lens.astype(np.float32), n_tracks)
        th0 = highland_theta0(e_start, lens)
        for c0 in range(0, n_tracks, chunk):
            c1 = min(n_tracks, c0 + chunk)
            sub = slice(pos + c0 * n, pos + c1 * n)
            if scatter:
                th0f = th0.astype(np.float32)[None, :]
                tx = rng.standard_normal((c1 - c0, n), dtype=np.float32) * th0f
                ty = rng.standard_normal((c1 - c0, n), dtype=np.float32) * th0f
                arrays["theta"][sub] = np.minimum(np.hypot(tx, ty), np.float32(math.pi)).reshape(-1)
                arrays["phi"][sub] = np.arctan2(ty, tx).reshape(-1)
            else:
                arrays["theta"][sub] = 0.0
                arrays["phi"][sub] = 0.0
        pos += n * n_tracks
        t0 += n_tracks
    step_begin[-1] = pos
    track_begin = np.arange(len(energies) + 1, dtype=np.int64) * n_tracks
    return Database(energy=np.asarray(energies, np.float64).astype(np.float32), track_begin=track_begin,
                    step_begin=step_begin, **arrays)


def database_from_tracks(energy, tracks) -> Database:
    """Build a database from explicit per-track step lists.

    ``energy``: list of bin energies; ``tracks``: list (per bin) of lists of
    tracks, each a sequence of (dE, len, theta, phi, esec) tuples.  Used for
    small hand-made test cases.
    """
    energy = np.asarray(energy, dtype=np.float32)
    track_begin = [0]
    step_begin = [0]
    rows = []
    for bin_tracks in tracks:
        for tr in bin_tracks:
            rows.extend(tr)
            step_begin.append(step_begin[-1] + len(tr))
        track_begin.append(track_begin[-1] + len(bin_tracks))
    a = np.asarray(rows, dtype=np.float64).reshape(-1, 5)
    return Database(energy=energy, track_begin=np.asarray(track_begin, np.int64),
                    step_begin=np.asarray(step_begin, np.int64),
                    dE=a[:, 0].astype(np.float32), len=a[:, 1].astype(np.float32),
                    theta=a[:, 2].astype(np.float32), phi=a[:, 3].astype(np.float32),
                    esec=a[:, 4].astype(np.float32))


@dataclass
class Phantom:
    shape: tuple            # (nx, ny, nz); voxel index v = ix + nx*(iy + ny*iz)
    spacing: tuple          # (dx, dy, dz) cm
    origin: tuple           # (x0, y0, z0) cm: corner of voxel (0,0,0)
    material: np.ndarray    # uint8 [nz, ny, nx] (x fastest in memory)
    density: np.ndarray     # float32 [nz, ny, nx] g/cm^3
    s_rel: np.ndarray       # float32 [n_mat] mass stopping-power ratio to water
    k_theta: np.ndarray     # float32 [n_mat] scattering-power ratio to water

    @property
    def nvox(self):
        nx, ny, nz = self.shape
        return nx * ny * nz


def _grid_centres(shape, spacing, origin):
    nx, ny, nz = shape
    x = origin[0] + (np.arange(nx) + 0.5) * spacing[0]
    y = origin[1] + (np.arange(ny) + 0.5) * spacing[1]
    z = origin[2] + (np.arange(nz) + 0.5) * spacing[2]
    return x, y, z


def uniform_phantom(shape, spacing, origin, material=MAT_WATER, density=1.0):
    nx, ny, nz = shape
    s_rel, k_theta = material_tables()
    return Phantom(shape=tuple(shape), spacing=tuple(float(s) for s in spacing),
                   origin=tuple(float(o) for o in origin),
                   material=np.full((nz, ny, nx), material, np.uint8),
                   density=np.full((nz, ny, nx), density, np.float32),
                   s_rel=s_rel, k_theta=k_theta)


def slab_phantom(n=64, voxel_cm=0.2, slab_z=(4.0, 6.0), slab_density=1.85):
    """Water cube (rho = 1.0) with a bone slab across z in ``slab_z`` (cm).

    The beam axis is z; x and y are centred on it and z = 0 is the entrance
    face.
    """
    half = 0.5 * n * voxel_cm
    ph = uniform_phantom((n, n, n), (voxel_cm,) * 3, (-half, -half, 0.0))
    zc = (np.arange(n) + 0.5) * voxel_cm
    sl = (zc >= slab_z[0]) & (zc < slab_z[1])
    ph.material[sl] = MAT_BONE
    ph.density[sl] = np.float32(slab_density)
    return ph


def slabs_phantom(shape, spacing, layers):
    """Phantom of uniform slabs along z.  ``layers``: list of
    (thickness_in_voxels, material, density)."""
    nx, ny, nz = shape
    if sum(t for t, _, _ in layers) != nz:
        raise ValueError("slab thicknesses must add up to nz")
    half_x, half_y = 0.5 * nx * spacing[0], 0.5 * ny * spacing[1]
    ph = uniform_phantom(shape, spacing, (-half_x, -half_y, 0.0))
    z = 0
    for t, m, rho in layers:
        ph.material[z:z + t] = m
        ph.density[z:z + t] = np.float32(rho)
        z += t
    return ph


def thorax_phantom(seed=7, shape=(256, 256, 128), voxel_cm=0.2):
    """Thorax-like phantom: the beam enters along +z (anterior to posterior),
    y runs cranio-caudally.  Body outline: elliptic cylinder along y in the
    (x, z) plane; air outside (rho 0.0012).  Inside: soft tissue rho ~
    N(1.0, 0.02), two lung ellipsoids rho ~ U(0.2, 0.3), a spine cylinder and
    rib ellipsoids rho ~ U(1.6, 1.9).  Geometry jitter from ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = shape
    sp = (voxel_cm,) * 3
    origin = (-0.5 * nx * voxel_cm, -0.5 * ny * voxel_cm, 0.0)
    xs, ys, zs = _grid_centres(shape, sp, origin)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    depth = nz * voxel_cm
    zc = 0.5 * depth + rng.uniform(-0.5, 0.5)
    ax = min(0.45 * nx * voxel_cm, 17.0) * rng.uniform(0.95, 1.05)
    az = 0.42 * depth * rng.uniform(0.95, 1.05)
    body = (X / ax) ** 2 + ((Z - zc) / az) ** 2 <= 1.0
    mat = np.full(shape[::-1], MAT_AIR, np.uint8)
    rho = np.full(shape[::-1], 0.0012, np.float32)
    mat[body] = MAT_WATER
    rho[body] = (1.0 + 0.02 * rng.standard_normal(int(body.sum()))).astype(np.float32)
    for side in (-1.0, 1.0):
        cx = side * ax * rng.uniform(0.38, 0.46)
        cy = rng.uniform(-2.0, 2.0)
        cz = zc + rng.uniform(-1.0, 1.0)
        rx, ry, rz = ax * rng.uniform(0.26, 0.32), 0.4 * ny * voxel_cm, az * rng.uniform(0.55, 0.65)
        lung = ((X - cx) / rx) ** 2 + ((Y - cy) / ry) ** 2 + ((Z - cz) / rz) ** 2 <= 1.0
        lung &= body
        mat[lung] = MAT_LUNG
        rho[lung] = rng.uniform(0.2, 0.3, int(lung.sum())).astype(np.float32)
    bone = np.zeros(shape[::-1], bool)
    # spine: cylinder along y near the posterior wall
    sz = zc + az * rng.uniform(0.62, 0.70)
    sr = rng.uniform(1.6, 2.2)
    bone |= (X / sr) ** 2 + ((Z - sz) / sr) ** 2 <= 1.0
    # sternum: flat ellipsoidal bar near the anterior wall
    bone |= (X / 1.2) ** 2 + ((Z - (zc - az * 0.85)) / 0.5) ** 2 <= 1.0
    # ribs: thin ellipsoids hugging the body outline at several y positions
    n_ribs = 10
    for k in range(n_ribs):
        cy = (k - (n_ribs - 1) / 2.0) * 2.4 + rng.uniform(-0.3, 0.3)
        for side in (-1.0, 1.0):
            ang = rng.uniform(0.2, 1.2)
            cx = side * ax * 0.9 * math.sin(ang)
            cz = zc + az * 0.9 * math.cos(ang) * rng.choice([-1.0, 1.0])
            r = ((X - cx) / 2.5) ** 2 + ((Y - cy) / 0.5) ** 2 + ((Z - cz) / 0.6) ** 2 <= 1.0
            bone |= r
    bone &= body
    mat[bone] = MAT_BONE
    rho[bone] = rng.uniform(1.6, 1.9, int(bone.sum())).astype(np.float32)
    s_rel, k_theta = material_tables()
    return Phantom(shape=tuple(shape), spacing=sp, origin=origin, material=np.ascontiguousarray(mat),
                   density=np.ascontiguousarray(rho), s_rel=s_rel, k_theta=k_theta)


# ----------------------------------------------------------------------------
# Beams.  A beam is a list of spots; each spot is a record with the fields of
# SPOT_DTYPE (one row per spot).  Profiles: 0 = Gaussian (a = sigma),
# 1 = rectangle (a = width, b = height), 2 = disk (a = radius); cm.

PROFILE_GAUSS, PROFILE_RECT, PROFILE_DISK = 0, 1, 2

SPOT_DTYPE = np.dtype([
    ("x", "<f8"), ("y", "<f8"), ("energy", "<f8"), ("sigma_e", "<f8"),
    ("a", "<f8"), ("b", "<f8"), ("profile", "<i4"), ("layer", "<i4"),
    ("n_histories", "<u8"),
])


def make_spots(rows):
    arr = np.zeros(len(rows), dtype=SPOT_DTYPE)
    for i, r in enumerate(rows):
        for k, v in r.items():
            arr[i][k] = v
    return arr


def pencil_beam(n_histories, energy=150.0, sigma_cm=0.3, sigma_e=0.0, x=0.0, y=0.0):
    return make_spots([dict(x=x, y=y, energy=energy, sigma_e=sigma_e, a=sigma_cm,
                            profile=PROFILE_GAUSS, layer=0, n_histories=n_histories)])


def field_beam(n_histories, energy=150.0, width=10.0, height=10.0, sigma_e_rel=0.01):
    return make_spots([dict(x=0.0, y=0.0, energy=energy, sigma_e=sigma_e_rel * energy,
                            a=width, b=height, profile=PROFILE_RECT, layer=0,
                            n_histories=n_histories)])


def disk_beam(n_histories, energy=121.0, radius=4.0, sigma_e=0.0):
    return make_spots([dict(x=0.0, y=0.0, energy=energy, sigma_e=sigma_e, a=radius,
                            profile=PROFILE_DISK, layer=0, n_histories=n_histories)])


def spot_plan(seed=11, n_layers=40, spots_per_layer=50, grid_cm=0.5, e_min=70.0,
              e_max=230.0, total=20_000_000, count_range=(1_000, 100_000),
              sigma_cm=0.3, sigma_e_rel=0.01):
    """Scanning-spot plan: ``n_layers`` energy layers linearly spaced over
    [e_min, e_max]; in each layer ``spots_per_layer`` positions of a
    ``grid_cm`` grid inside a centred disk, picked by a seeded shuffle;
    log-normal per-spot history counts clipped to ``count_range`` and
    rescaled to ``total``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    # disk radius holding comfortably more grid points than needed
    r = grid_cm * math.sqrt(spots_per_layer / math.pi) * 1.25
    k = int(math.ceil(r / grid_cm)) + 1
    pts = [(i * grid_cm, j * grid_cm) for i in range(-k, k + 1) for j in range(-k, k + 1)
           if (i * grid_cm) ** 2 + (j * grid_cm) ** 2 <= r * r]
    if len(pts) < spots_per_layer:
        raise ValueError("disk too small")
    energies = np.linspace(e_min, e_max, n_layers)
    lo, hi = count_range
    mu = 0.5 * (math.log(lo) + math.log(hi))
    sig = (math.log(hi) - math.log(lo)) / 4.0
    n_spots = n_layers * spots_per_layer
    counts = np.clip(np.exp(mu + sig * rng.standard_normal(n_spots)), lo, hi)
    for _ in range(8):
        counts = np.clip(counts * (total / counts.sum()), lo, hi)
    counts = np.floor(counts).astype(np.int64)
    counts = np.maximum(counts, 1)
    # distribute the remainder so that the total is exact
    rem = total - int(counts.sum())
    order = rng.permutation(n_spots)
    i = 0
    while rem != 0:
        j = order[i % n_spots]
        step = 1 if rem > 0 else -1
        if counts[j] + step >= 1:
            counts[j] += step
            rem -= step
        i += 1
    rows = []
    s = 0
    for layer, E in enumerate(energies):
        sel = rng.permutation(len(pts))[:spots_per_layer]
        for q in sel:
            x, y = pts[q]
            rows.append(dict(x=x, y=y, energy=float(E), sigma_e=sigma_e_rel * float(E),
                             a=sigma_cm, profile=PROFILE_GAUSS, layer=layer,
                             n_histories=int(counts[s])))
            s += 1
    return make_spots(rows)


def database_energies(n=24, e_min=70.0, e_max=250.0):
    return np.linspace(e_min, e_max, n)


# Named workloads (phantom, database, beam) shaped like the paper's: see the
# project's design notes for the recipe of each.

def workload_slab(n_histories=100_000, n_tracks=10_000, energy=150.0, seed_db=1):
    db = water_database([energy], n_tracks, seed_db)
    ph = slab_phantom()
    beam = pencil_beam(n_histories, energy=energy, sigma_cm=0.3)
    return db, ph, beam


def workload_thorax(n_histories=10_000_000, n_tracks=100_000, seed_db=2, seed_ph=7,
                    shape=(256, 256, 128)):
    db = water_database(database_energies(), n_tracks, seed_db)
    ph = thorax_phantom(seed_ph, shape=shape)
    beam = field_beam(n_histories, energy=150.0, width=10.0, height=10.0, sigma_e_rel=0.01)
    return db, ph, beam


def workload_spots(total=20_000_000, n_tracks=100_000, seed_db=2, seed_plan=11, db=None):
    if db is None:
        db = water_database(database_energies(), n_tracks, seed_db)
    ph = slab_phantom()
    beam = spot_plan(seed_plan, total=total)
    return db, ph, beam
