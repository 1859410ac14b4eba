/*
 * fdc.h -- C ABI of the GB300 track-repeating proton dose engine.
 *
 * The engine implements the track-repeating algorithm of Yepes, Mirkovic &
 * Taddei, "A GPU implementation of a track-repeating algorithm for proton
 * radiotherapy dose calculations":
 *   Sec. 2.2  a database of proton tracks pre-generated in water, stored step
 *             by step, is re-traced through a voxel phantom by scaling each
 *             step length and each scattering angle with the local material;
 *   Sec. 2.3  the problem statement the calls below follow: load the material
 *             scaling tables and the voxel geometry, load the track database,
 *             simulate N incident protons drawn from a phase space, tally the
 *             deposited energy in a grid shaped like the phantom and convert
 *             it to dose by dividing by the voxel mass;
 *   Sec. 2.4  batch statistics, eq. (1).
 *
 * Conventions shared by every call:
 *   - Units: cm, MeV, g/cm^3, Gy.  The beam travels along +z and enters the
 *     phantom at its upstream face z = z0.
 *   - Voxel (ix, iy, iz) has linear index v = ix + nx * (iy + ny * iz)
 *     (x fastest); every per-voxel array uses that order.
 *   - "host" pointers are ordinary CPU memory, read during the call and not
 *     retained; "device" pointers are CUDA global memory on the context's
 *     device, owned by the caller unless stated otherwise.
 *   - Streams are cudaStream_t values passed as void * (NULL = legacy default
 *     stream).  Device work is asynchronous on that stream; argument errors
 *     are returned synchronously; errors found on the device are latched in
 *     a status word returned by fdc_sync.  Nothing traps.
 *   - Return value: FDC_OK (0) or one of the FDC_ERR_* codes below;
 *     fdc_last_error gives a one-line message.
 *   - Determinism: for the same database, phantom, beam, seed and history
 *     range the integer energy tally, and hence the dose, is bitwise
 *     identical whatever the launch schedule or the split of the history
 *     range into calls.
 */
#ifndef FDC_H
#define FDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FDC_OK = 0,
    FDC_ERR_INVALID = 1,     /* bad argument or input data */
    FDC_ERR_NOT_LOADED = 2,  /* database or phantom missing */
    FDC_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    FDC_ERR_OOM = 4,         /* device allocation failed */
    FDC_ERR_STEP_LIMIT = 5,  /* device: a step crossed more voxels than the grid allows */
    FDC_ERR_OVERFLOW = 6,    /* fixed-point headroom would be exceeded */
    FDC_ERR_TIMEOUT = 7      /* a bounded device wait gave up */
};

enum { FDC_PROFILE_GAUSS = 0, FDC_PROFILE_RECT = 1, FDC_PROFILE_DISK = 2 };

/* Energy tally unit: the dose grid accumulates int64 multiples of
 * 2^-FDC_TALLY_SHIFT MeV. */
#define FDC_TALLY_SHIFT 28

typedef struct fdc_ctx fdc_ctx;

/* Water track database (Sec. 2.2), host arrays in CSR form.
 *   energy[n_energies]        bin energies (MeV), strictly increasing;
 *   track_begin[n_energies+1] tracks of bin b are [track_begin[b], track_begin[b+1]),
 *                             every bin holds at least one track;
 *   step_begin[n_tracks+1]    steps of track t are [step_begin[t], step_begin[t+1]);
 *   per step k, in track order:
 *     dE[k]    energy lost along the step (MeV, >= 0);
 *     len[k]   step length in water (cm, > 0);
 *     theta[k] polar deflection applied at the end of the step (rad, [0, pi]);
 *     phi[k]   its azimuth (rad);
 *     esec[k]  energy deposited locally at the end of the step (MeV, >= 0).
 * Storage: one 16-byte record per step holds len, dE and the deflection as
 * the vector theta * (cos phi, sin phi), formed in FP64 and rounded once to
 * FP32 (so theta and phi keep FP32 precision; phi needs no range reduction
 * by the caller); esec goes to a side array that is read only for tracks
 * with a nonzero entry. */
typedef struct fdc_database {
    int32_t n_energies;
    const float *energy;
    const int64_t *track_begin;
    const int64_t *step_begin;
    const float *dE, *len, *theta, *phi, *esec;
} fdc_database;

/* Voxel phantom (Sec. 2.3: material index per voxel plus per-material
 * scaling parameters).  host arrays:
 *   material[nvox] in [0, n_mat); density[nvox] (g/cm^3, >= 0);
 *   s_rel[n_mat]   mass stopping-power ratio to water: a geometric length g in
 *                  voxel v consumes g * density[v] * s_rel[material[v]] of the
 *                  water step length;
 *   k_theta[n_mat] scattering-power ratio to water: a step's deflection is
 *                  theta * sqrt(sum_i w_i k_theta_i^2) over the voxels it
 *                  crossed, w_i the water-equivalent fraction in each.
 * Geometry: nx, ny, nz voxels of dx, dy, dz cm; (x0, y0, z0) is the corner of
 * voxel (0, 0, 0).  n_mat <= 256. */
typedef struct fdc_phantom {
    int32_t nx, ny, nz, n_mat;
    double dx, dy, dz, x0, y0, z0;
    const uint8_t *material;
    const float *density;
    const float *s_rel;
    const float *k_theta;
} fdc_phantom;

/* One beam spot (phase-space source, Sec. 2.3).  The spot's histories have
 * consecutive global indices, spots in array order.  Per history:
 *   entry (x, y): GAUSS: centre + a * N(0,1) per axis; RECT: uniform over
 *   a x b around the centre; DISK: uniform over a disk of radius a;
 *   energy: energy + sigma_e * N(0,1) (sigma_e = 0: mono-energetic);
 *   layer: index of the per-layer tally the history scores into. */
typedef struct fdc_spot {
    double x, y, energy, sigma_e, a, b;
    int32_t profile, layer;
    uint64_t n_histories;
} fdc_spot;

typedef struct fdc_beam {
    int32_t n_spots;
    const fdc_spot *spots;   /* host [n_spots] */
} fdc_beam;

/* Launch schedule of the replay kernel.  Zero fields take the context's
 * tuned (or built-in) value. */
typedef struct fdc_schedule {
    int32_t ctas_per_sm;     /* persistent CTAs per SM */
    int32_t warps_per_cta;   /* 1..8 */
    int32_t chunk;           /* 32-history groups a warp claims per atomic */
    int32_t aggregate;       /* 1: combine the tally atomics of warp lanes that hit the same
                                voxel; 2: one atomic per lane (default) */
} fdc_schedule;

/* Options of fdc_run_ex.  Zero-initialise for the defaults. */
typedef struct fdc_run_opts {
    uint64_t history_offset; /* first global history index of this call */
    int32_t track_group;     /* histories h with equal h / track_group draw the same
                                track (0 or 1: independent draws) */
    int32_t no_rotation;     /* 1: replay every track unrotated (psi = 0) */
    int32_t scaling_mode;    /* 0: per-voxel water-equivalent scaling; 1: the
                                voxel where a step starts scales the whole step */
    int32_t fp64_geometry;   /* 1: step geometry in FP64 instead of FP32 */
    int32_t n_batches;       /* >= 2: split the histories into equal batches and
                                accumulate the per-voxel batch dose sum and sum of
                                squares (eq. (1)); 0 or 1: one batch */
    int32_t no_graph;        /* 1: issue the launches directly; 0: run them as a CUDA
                                graph, captured once and relaunched while the launch
                                configuration repeats */
    fdc_schedule schedule;
} fdc_run_opts;

/* Outputs of fdc_run_ex; any pointer may be NULL.  device arrays, written
 * (not accumulated) by the call:
 *   dose[nvox]                  total dose (Gy);
 *   layer_dose[n_layers * nvox] dose per layer, n_layers = 1 + max spot layer;
 *   batch_sum[nvox], batch_sumsq[nvox]
 *                               sum over batches of the batch dose and of its
 *                               square (needs n_batches >= 2);
 *   tally[nvox]                 raw int64 energy tally of the whole call
 *                               (units of 2^-FDC_TALLY_SHIFT MeV). */
typedef struct fdc_outputs {
    double *dose;
    double *layer_dose;
    double *batch_sum;
    double *batch_sumsq;
    int64_t *tally;
    double *history_sumsq;   /* [nvox]: sum over histories of the square of the history's
                                dose in the voxel (Gy^2), the second tally of Sec. 2.3 for
                                eq. (2); squared per voxel visit, so a history that leaves a
                                voxel and re-enters it later adds two squares */
} fdc_outputs;

/* Counters of the last run, valid after fdc_sync.  Energies are in tally
 * units: replayed = energy of the replayed steps, escaped = the part that left
 * the grid; the tally holds replayed - escaped exactly. */
typedef struct fdc_counters {
    uint64_t histories, steps, segments;
    int64_t replayed, escaped;
    int32_t status;
    int32_t pad;
    uint64_t bad_history;    /* first history that raised a device error */
} fdc_counters;

/* Create a context on CUDA device `device`.  *out receives the handle. */
int fdc_create(fdc_ctx **out, int device);
/* Free every device buffer of the context (waits for its work first). */
void fdc_destroy(fdc_ctx *ctx);
/* Message of the last error on this context (static storage of the context). */
const char *fdc_last_error(const fdc_ctx *ctx);

/* Sec. 2.2: validate and copy the database to the device (replaces any
 * previous one).  Synchronous. */
int fdc_load_database(fdc_ctx *ctx, const fdc_database *db);
/* Sec. 2.3: validate and copy the phantom and material tables to the device
 * (replaces any previous one).  Synchronous. */
int fdc_load_phantom(fdc_ctx *ctx, const fdc_phantom *ph);

/* Sec. 2.3: simulate histories [0, n_histories) of `beam` with random stream
 * `seed` and write the dose (Gy) to device array dose_out[nvox].
 * n_histories = 0 means all histories of the beam; more than the beam holds
 * is FDC_ERR_INVALID.  Asynchronous on `stream`. */
int fdc_run(fdc_ctx *ctx, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
            double *dose_out, void *stream);

/* As fdc_run, for histories [opts->history_offset, opts->history_offset +
 * n_histories) with the options and outputs above. */
int fdc_run_ex(fdc_ctx *ctx, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
               const fdc_run_opts *opts, const fdc_outputs *out, void *stream);

/* As fdc_run_ex with a HOST dose buffer: copies the beam in, runs with
 * `opts` (may be NULL), copies the dose out and waits.  Returns the device
 * status as fdc_sync does. */
int fdc_run_host(fdc_ctx *ctx, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
                 const fdc_run_opts *opts, double *dose_host);

/* Sec. 2.3 (end of run: energy divided by the voxel mass) for a tally the
 * caller holds: converts tally[nvox] (device, int64 energy in units of
 * 2^-FDC_TALLY_SHIFT MeV, read only) to dose_out[nvox] (device, Gy) with the
 * loaded phantom's densities and voxel volume.  This is the last step after
 * runs over disjoint history ranges -- on one device or on several (the
 * paper's two GPUs each replayed part of the histories and the doses were
 * summed at the end, Sec. 2.3) -- whose `tally` outputs were added: integer
 * sums are exact, so the dose equals that of one run over all the
 * histories, bit for bit.  Asynchronous on `stream`. */
int fdc_dose_from_tally(fdc_ctx *ctx, const int64_t *tally, double *dose_out, void *stream);

/* Wait for `stream`, read the device status word of the last run and its
 * counters.  Returns FDC_OK or the first device error (FDC_ERR_STEP_LIMIT,
 * ...); `counters` (host, may be NULL) receives the counters. */
int fdc_sync(fdc_ctx *ctx, void *stream, fdc_counters *counters);

/* Eq. (1) on the device: from batch_sum/batch_sumsq over n_batches (>= 2)
 * write mean[nvox] and sigma[nvox] (device, Gy), and to *mean_rel (host) the
 * average of sigma/mean over voxels whose mean exceeds frac * max(mean)
 * (Sec. 2.4 uses frac = 0.5).  Synchronous. */
int fdc_batch_stats(fdc_ctx *ctx, const double *batch_sum, const double *batch_sumsq,
                    int32_t n_batches, double frac, double *mean, double *sigma,
                    double *mean_rel, void *stream);

/* Eq. (2) on the device: from dose_sum[nvox] (the run's dose, i.e. the sum of
 * the N per-history doses) and history_sumsq[nvox] write the mean dose per
 * history mean[nvox] and its uncertainty sigma[nvox] (device, Gy), and to
 * *mean_rel (host) the average sigma/mean over voxels above frac * max(mean).
 * Synchronous. */
int fdc_history_stats(fdc_ctx *ctx, const double *dose_sum, const double *history_sumsq,
                      uint64_t n_histories, double frac, double *mean, double *sigma,
                      double *mean_rel, void *stream);

/* Pick the replay schedule for this beam and these run options by timing
 * candidates on the device (Sec. 3 tuned the paper's N_B and N_T by hand):
 * the built-in default and warps per CTA x CTAs per SM x chunk x tally
 * aggregation, each CTA count bounded by the occupancy of the kernel
 * instantiation the options select (track group, FP64 geometry, and whether
 * the database has local deposits).  Runs histories [h, h + n_histories) of
 * the beam, h = opts->history_offset, several times and keeps the candidate
 * with the shortest replay-kernel time (CUDA events); results are discarded.
 * opts (host, may be NULL) is read for history_offset, track_group,
 * no_rotation, scaling_mode and fp64_geometry; its schedule and n_batches
 * are ignored.  The choice becomes the context's default schedule for runs
 * that select the same kernel instantiation; *best (host, may be NULL)
 * receives it.  Synchronous. */
int fdc_autotune(fdc_ctx *ctx, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
                 const fdc_run_opts *opts, fdc_schedule *best);

/* Measurement.  fdc_set_timing(ctx, 1) makes later runs record CUDA events
 * on their stream around the replay kernel(s) and the finalize kernel (timed
 * runs launch their kernels directly instead of through a CUDA graph);
 * fdc_last_kernel_ms waits for them and returns the last run's replay time
 * (first to last replay launch) and finalize time in milliseconds. */
int fdc_set_timing(fdc_ctx *ctx, int32_t enable);
int fdc_last_kernel_ms(fdc_ctx *ctx, double *replay_ms, double *finalize_ms);

/* L2 atomic throughput probe (roofline denominator of the tally updates; no
 * counterpart in the paper): n_ops 64-bit atomic adds of 1 spread by a hash
 * over the first P counters of device array slots[n_slots] (zeroed by the
 * call), P the largest power of two <= n_slots, issued by a full-occupancy
 * grid with four independent updates in flight per thread; *ms (host)
 * receives the kernel time.  Synchronous on `stream`. */
int fdc_probe_atomics(uint64_t *slots, uint64_t n_slots, uint64_t n_ops, double *ms, void *stream);

/* Run without allocating device memory.
 *
 * For callers that must not allocate during a run: for example a planning
 * system that reserves all of its device memory at start-up and keeps other
 * work in flight on the GPU, where a cudaMalloc or cudaFree (which may wait
 * for the whole device) or an out-of-memory failure in the middle of a plan
 * is not acceptable.  The paper has no counterpart to this call.
 *
 * Same computation and result as fdc_run with default options -- histories
 * [0, n_histories), one track per history (track group 1), rotated reuse,
 * per-voxel step scaling, FP32 geometry, the context's default schedule --
 * and bit for bit the same dose; there are no run options, so runs with a
 * track group, batches or per-layer dose need fdc_run_ex.  The database and phantom must
 * already be loaded into ctx (those loads allocate, once, beforehand); the
 * caller passes the beam (host) and dose_out[nvox] (device).  All scratch --
 * the int64 tally, the counters, the work counter and the device copy of the
 * spot table -- lives in one static device array of FDC_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads the library holds until the process exits; the
 * call makes no cudaMalloc, cudaFree or other allocating call.
 * Limits: nvox <= FDC_NOALLOC_MAX_VOXELS, n_spots <= FDC_NOALLOC_MAX_SPOTS;
 * larger inputs return FDC_ERR_INVALID.
 * The first call on a device looks up the static array's device address
 * (once per device); make that first call before any stream capture.
 * Every call on a device shares the one array and reuses it as the last call
 * left it (the call clears what must start at zero): calls whose GPU work
 * overlaps -- on different streams or host threads without ordering -- race
 * and corrupt each other's results.
 * counters_dev (device, may be NULL) receives the run's counters and device
 * status (as fdc_sync reports them for other runs) once the work on `stream`
 * completes.  Asynchronous on `stream`, except for the copy of the spot
 * table from the caller's host memory: from pageable memory that copy is
 * synchronous (the host waits for it) and cannot be recorded in a stream
 * capture; from pinned memory it is asynchronous.  The call allocates no
 * staging buffer for it. */
#define FDC_NOALLOC_MAX_VOXELS (1 << 21)
#define FDC_NOALLOC_MAX_SPOTS 4096
#define FDC_NOALLOC_SCRATCH_BYTES                                                  \
    (8u * FDC_NOALLOC_MAX_VOXELS + 256u + 64u * FDC_NOALLOC_MAX_SPOTS + \
     8u * (FDC_NOALLOC_MAX_SPOTS + 1) + 256u)
int fdc_run_noalloc(fdc_ctx *ctx, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
                    double *dose_out, fdc_counters *counters_dev, void *stream);

/* Test hooks.  fdc_debug_philox: Philox4x64-10 (Salmon et al., SC'11) with
 * key (key0, key1) on n device counters ctr[n][4], writing out[n][4] (device).
 * fdc_debug_sample: task 1 of histories [h_begin, h_begin + n) -- entry x, y,
 * energy and rotation psi (device xyEpsi[n][4]) and energy bin, track and
 * start step (device btk[n][3]). */
int fdc_debug_philox(uint64_t key0, uint64_t key1, const uint64_t *ctr, uint64_t n,
                     uint64_t *out, void *stream);
int fdc_debug_sample(fdc_ctx *ctx, const fdc_beam *beam, uint64_t seed, uint64_t h_begin,
                     uint64_t n, int32_t track_group, int32_t no_rotation, float *xyEpsi,
                     int64_t *btk, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FDC_H */
