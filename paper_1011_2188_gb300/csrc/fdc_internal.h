// Internal declarations shared by the host library (fdc_api.cu) and the
// kernels (fdc_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fdc.h"

namespace fdc {

// One step of a track, 16 bytes, loaded with a single 128-bit load:
//   x: len (float bits, cm of water)   y: dE (float bits, MeV)
//   z, w: the deflection at the end of the step as the vector
//         theta * (cos phi, sin phi) (float bits; computed in FP64 from the
//         database's theta and phi and rounded once to FP32)
// Per-step side arrays: eres (float residual energy at step start, used by
// the start-step search), tail (int64: tally units of all later steps of the
// track, used to book escaped energy exactly) and, only when the database
// has local deposits, esec (float MeV) with a per-track flag that says
// whether the track has any.
static_assert(sizeof(uint4) == 16, "step record must be 16 bytes");

constexpr double kTallyUnitsPerMeV = 268435456.0;  // 2^FDC_TALLY_SHIFT
constexpr double kMeVToJ = 1.602176634e-13;

struct DeviceCounters {  // same layout as fdc_counters
    unsigned long long histories, steps, segments;
    long long replayed, escaped;
    int status;
    int pad;
    unsigned long long bad_history;
};
static_assert(sizeof(DeviceCounters) == sizeof(fdc_counters), "counter layout");

struct ReplayArgs {
    // database (device)
    const uint4 *rec;
    const float *esec;             // null when no step has a local deposit
    const unsigned char *trk_esec; // per track: 1 if any of its steps has esec > 0
    const float *eres;
    const long long *tail;
    const long long *step_begin;
    const float *bin_energy;
    const long long *bin_track_begin;
    int n_bins;
    // phantom (device): per voxel (S_rel = density * s_rel[m], k_theta[m]^2)
    const float2 *vox;
    int nx, ny, nz;
    double dx, dy, dz, x0, y0, z0;
    double x1, y1;            // x0 + nx * dx, y0 + ny * dy (entry test)
    double idx_, idy_;        // 1 / dx, 1 / dy (entry voxel, FP64)
    float ihx, ihy, ihz;      // 1 / spacing in FP32 (grid units per cm)
    // beam (device)
    const fdc_spot *spots;
    const unsigned long long *spot_cum;  // [n_spots + 1]
    int n_spots;
    // run
    unsigned long long *tally;  // [n_tallies][nvox], int64 two's complement
    unsigned long long *sumsq;  // null, or [n_tallies][nvox]: sum of squared voxel visits (2^-28 MeV^2)
    long long nvox;
    int per_layer;
    unsigned long long h_begin, n;  // histories [h_begin, h_begin + n)
    unsigned long long seed;
    int track_group, rotate, scaling_mode;
    int u32;                      // 1: every step of the database is below 2^32 tally units
    int chunk;
    unsigned long long *work;     // work counter (zeroed before launch)
    DeviceCounters *counters;
};

struct FinalizeArgs {
    long long *tally;        // [n_tallies][nvox], read (and zeroed if zero_after)
    int n_tallies;
    long long nvox;
    const float *density;
    double scale;            // Gy per tally unit per (g/cm^3)
    const double *factor;    // [nvox] or null: scale / density (0 where density is 0), precomputed
    double *dose;            // [nvox] or null: dose of the summed tally
    double *layer_dose;      // [n_tallies][nvox] or null
    long long *tally_out;    // [nvox] or null: summed tally
    double *batch_sum;       // [nvox] or null: += dose
    double *batch_sumsq;     // [nvox] or null: += dose^2
    long long *accum;        // [n_tallies][nvox] or null: += tally
    int zero_after;          // 1: tally := 0 after reading
    const long long *sumsq;  // [n_tallies][nvox] or null: squared-visit tally ...
    double *hist_sumsq;      // ... summed over tallies and converted to Gy^2 here
};

cudaError_t launch_replay(const ReplayArgs &a, const fdc_schedule &s, int fp64, int sm_count,
                          cudaStream_t st);
cudaError_t launch_finalize(const FinalizeArgs &a, int sm_count, cudaStream_t st);
// factor[v] = scale / density[v] (0 where the density is 0), the finalize step's per-voxel factor
cudaError_t launch_dose_factor(const float *density, double scale, long long nvox, double *factor, cudaStream_t st);
// mode 0: eq. (1) from n batch sums; mode 1: eq. (2) from sums over n histories
cudaError_t launch_batch_stats(const double *sum, const double *sumsq, long long n, int mode, long long nvox,
                               double frac, double *mean, double *sigma, double *partials,
                               int n_partials, double *result, cudaStream_t st);
cudaError_t launch_debug_philox(unsigned long long k0, unsigned long long k1,
                                const unsigned long long *ctr, unsigned long long n,
                                unsigned long long *out, cudaStream_t st);
cudaError_t launch_debug_sample(const ReplayArgs &a, float *xyEpsi, long long *btk,
                                cudaStream_t st);
// What selects the replay kernel's instantiation (and so its register budget
// and occupancy).
struct ReplayVariant {
    int fp64, aggregate, squares, track_group, esec, u32;
};
ReplayVariant replay_variant(const ReplayArgs &a, const fdc_schedule &s, int fp64);
int replay_max_ctas_per_sm(int warps_per_cta, const ReplayVariant &v);
// Record packing at load: (len, dE, theta, phi) -> (len, dE, theta cos phi,
// theta sin phi), in place, FP64 arithmetic rounded to FP32.
cudaError_t launch_pack_deflections(uint4 *rec, long long n, cudaStream_t st);
// Static scratch of fdc_run_noalloc (defined in fdc_kernels.cu with the
// array): device addresses of its parts on the current device, looked up once
// per device.
struct NoallocScratch {
    unsigned long long *tally;  // [FDC_NOALLOC_MAX_VOXELS]
    DeviceCounters *counters;
    unsigned long long *work;
    fdc_spot *spots;            // [FDC_NOALLOC_MAX_SPOTS]
    unsigned long long *spot_cum;  // [FDC_NOALLOC_MAX_SPOTS + 1]
};
cudaError_t noalloc_scratch(int device, NoallocScratch *out);
cudaError_t launch_spot_prefix(const fdc_spot *spots, int n_spots, unsigned long long *cum,
                               cudaStream_t st);
cudaError_t launch_probe_atomics(unsigned long long *slots, unsigned long long n_slots,
                                 unsigned long long n_ops, int sm_count, cudaStream_t st);

}  // namespace fdc
