// Device code of the track-repeating dose engine (sm_103a).
//
// replay_kernel: persistent grid; every warp claims groups of 32 histories
// from a global counter and each lane re-traces one history at a time
// (Sec. 2.3, tasks 1 and 2):
//   task 1  Philox4x64-10 draws the entry point, energy and track rotation;
//           the energy picks the database bin and the start step (first step
//           whose residual energy is <= the proton energy);
//   task 2  for every step: one 128-bit load of the step record, an
//           Amanatides-Woo march over the voxels the step crosses in which
//           the water step length is consumed as water-equivalent length
//           (Sec. 2.2 step scaling), energy shared over the segments in
//           proportion, the deflection at the end scaled by the crossed
//           materials' scattering-power ratios (Sec. 2.2 angle scaling).
// Energy goes to an int64 fixed-point tally (2^-28 MeV units) with integer
// atomics, so the sum is independent of the order of the updates: the paper's
// blocking tally update (Sec. 2.3) becomes a single L2 reduction, optionally
// combined across the lanes of a warp that hit the same voxel.

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "fdc_internal.h"

namespace fdc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// 1: a lane sums consecutive deposits into one voxel before its atomic
// (fewer atomics, more registers; measured slower on GB300 under the
// 64-register cap, so off by default).
#ifndef FDC_LANE_COALESCE
#define FDC_LANE_COALESCE 0
#endif
constexpr float kUnitsF = 268435456.0f;  // 2^28
constexpr double kTwoPi = 6.283185307179586476925286766559;

// ---------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 64x64->128 multiplications and a key-dependent mix, the key bumped by the
// Weyl constants between rounds.
struct U64x4 {
    unsigned long long v0, v1, v2, v3;
};

__device__ __forceinline__ U64x4 philox(unsigned long long c0, unsigned long long c1,
                                        unsigned long long c2, unsigned long long c3,
                                        unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const unsigned long long n0 = hi1 ^ c1 ^ k0;
        const unsigned long long n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

// (0,1) uniform from the top 53 bits, centred in its cell.
__device__ __forceinline__ double u01(unsigned long long r) {
    return __dmul_rn(__dadd_rn((double)(r >> 11), 0.5), 0x1p-53);
}

// ---------------------------------------------------------------- task 1
struct Start {
    float x, y, E, psi;
    int bin, layer;
    long long track, s0, k0, n;  // steps [s0 + k0, s0 + n) are replayed
};

// Per-history draws in FP64 with explicit rounding (no contraction), then
// rounded to the single-precision per-proton state.
__device__ Start sample_start(const ReplayArgs &P, unsigned long long h) {
    Start st;
    const U64x4 A = philox(h, 1, 0, 0, P.seed, 0);
    const U64x4 B = philox(h, 2, 0, 0, P.seed, 0);
    const unsigned long long g = P.track_group > 1 ? h / (unsigned long long)P.track_group : h;
    const U64x4 C = philox(g, 3, 0, 0, P.seed, 0);

    // spot: largest s with cum[s] <= h
    int lo = 0, hi = P.n_spots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.spot_cum[mid] <= h) lo = mid; else hi = mid - 1;
    }
    const fdc_spot sp = P.spots[lo];
    st.layer = sp.layer;

    double x, y;
    if (sp.profile == FDC_PROFILE_GAUSS) {
        const double r = __dsqrt_rn(__dmul_rn(-2.0, log(u01(A.v0))));
        double s, c;
        sincos(__dmul_rn(kTwoPi, u01(A.v1)), &s, &c);
        x = __dadd_rn(sp.x, __dmul_rn(sp.a, __dmul_rn(r, c)));
        y = __dadd_rn(sp.y, __dmul_rn(sp.a, __dmul_rn(r, s)));
    } else if (sp.profile == FDC_PROFILE_RECT) {
        x = __dadd_rn(sp.x, __dmul_rn(sp.a, __dsub_rn(u01(A.v0), 0.5)));
        y = __dadd_rn(sp.y, __dmul_rn(sp.b, __dsub_rn(u01(A.v1), 0.5)));
    } else {
        const double r = __dmul_rn(sp.a, __dsqrt_rn(u01(A.v0)));
        double s, c;
        sincos(__dmul_rn(kTwoPi, u01(A.v1)), &s, &c);
        x = __dadd_rn(sp.x, __dmul_rn(r, c));
        y = __dadd_rn(sp.y, __dmul_rn(r, s));
    }
    double E = sp.energy;
    if (sp.sigma_e > 0.0) {
        const double r = __dsqrt_rn(__dmul_rn(-2.0, log(u01(A.v2))));
        const double n0 = __dmul_rn(r, cos(__dmul_rn(kTwoPi, u01(A.v3))));
        E = __dadd_rn(sp.energy, __dmul_rn(sp.sigma_e, n0));
    }
    st.x = (float)x;
    st.y = (float)y;
    st.E = (float)E;
    st.psi = P.rotate ? (float)__dmul_rn(kTwoPi, u01(B.v0)) : 0.0f;

    // energy bin: first bin energy >= E, else the top bin
    int b0 = 0, b1 = P.n_bins - 1;
    while (b0 < b1) {
        const int mid = (b0 + b1) >> 1;
        if (P.bin_energy[mid] >= st.E) b1 = mid; else b0 = mid + 1;
    }
    st.bin = b0;
    const long long tb = P.bin_track_begin[b0];
    const unsigned long long nb = (unsigned long long)(P.bin_track_begin[b0 + 1] - tb);
    st.track = tb + (long long)__umul64hi(C.v0, nb);
    st.s0 = P.step_begin[st.track];
    st.n = P.step_begin[st.track + 1] - st.s0;
    // start step: first k with eres[k] <= E (eres is non-increasing)
    long long k0 = st.n;
    if (st.E > 0.0f) {
        long long l = 0, r = st.n;
        while (l < r) {
            const long long mid = (l + r) >> 1;
            if (__ldg(P.eres + st.s0 + mid) <= st.E) r = mid; else l = mid + 1;
        }
        k0 = l;
    }
    st.k0 = k0;
    return st;
}

// ---------------------------------------------------------------- helpers
// Step records stream through L2 once per use; loading them with an
// evict-first L2 policy keeps the L2-resident tally and phantom words from
// being displaced by the stream.
#ifndef FDC_RECORD_EVICT_FIRST
#define FDC_RECORD_EVICT_FIRST 0
#endif
// A lane reads its track's records in order, eight to a 128-byte line; with
// FDC_RECORD_PREFETCH, entering a line prefetches the next one into L2 (some
// eight steps of lead).  Measured slower on GB300 (1.4 % with shared tracks,
// 4.9 % with independent ones), so off.
#ifndef FDC_RECORD_PREFETCH
#define FDC_RECORD_PREFETCH 0
#endif

#if FDC_RECORD_PREFETCH
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
#endif

__device__ __forceinline__ unsigned long long evict_first_policy() {
    unsigned long long pol = 0;
#if FDC_RECORD_EVICT_FIRST
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#endif
    return pol;
}

__device__ __forceinline__ uint4 load_record(const uint4 *p, unsigned long long pol) {
#if FDC_RECORD_EVICT_FIRST
    uint4 r;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
#else
    (void)pol;
    return __ldg(p);
#endif
}

__device__ __forceinline__ void sincos_(float a, float *s, float *c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_(double a, double *s, double *c) { sincos(a, s, c); }
// FP32 square roots of the deflection arithmetic: the hardware approximation
// (relative error ~2^-22, the order of FP32 rounding itself).
__device__ __forceinline__ float sqrt_(float a) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
__device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }
// Reciprocal: hardware approximation in FP32 (relative error ~1e-7, used for
// segment geometry only), IEEE in FP64.
__device__ __forceinline__ float rcp_(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double rcp_(double a) { return 1.0 / a; }
__device__ __forceinline__ double rsqrt_(double a) { return rsqrt(a); }
template <typename R> __device__ __forceinline__ R inf_();
template <> __device__ __forceinline__ float inf_<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double inf_<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

// Tally update.  AGG: lanes of the warp that add to the same tally word are
// combined first (match on the word's address -- not on the voxel index, since
// lanes may score into different layer tallies -- then add the four 16-bit
// limbs of the two's-complement value with redux.sync inside each group, one
// atomic per group); otherwise one atomic per lane.
template <bool AGG>
__device__ __forceinline__ void tally_add(unsigned long long *tally, int idx, long long units) {
    unsigned long long *const addr = tally + idx;
    if (!AGG) {
        atomicAdd(addr, (unsigned long long)units);
        return;
    }
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mask = __activemask();
    const unsigned peers = __match_any_sync(mask, (unsigned long long)addr);
    if (peers == (1u << lane)) {
        atomicAdd(addr, (unsigned long long)units);
        return;
    }
    const unsigned long long u = (unsigned long long)units;
    const unsigned l0 = __reduce_add_sync(peers, (unsigned)(u & 0xffffu));
    const unsigned l1 = __reduce_add_sync(peers, (unsigned)((u >> 16) & 0xffffu));
    const unsigned l2 = __reduce_add_sync(peers, (unsigned)((u >> 32) & 0xffffu));
    const unsigned l3 = __reduce_add_sync(peers, (unsigned)(u >> 48));
    if (lane == (unsigned)(__ffs(peers) - 1)) {
        const unsigned long long s = (unsigned long long)l0 + ((unsigned long long)l1 << 16) +
                                     ((unsigned long long)l2 << 32) + ((unsigned long long)l3 << 48);
        atomicAdd(addr, s);
    }
}

// Lane-local coalescing of tally updates: consecutive deposits of one lane
// into the same tally word are summed in registers and written with one
// atomic when the lane moves to another word (or finishes the history).
// Integer sums, so the tally is the same bit for bit.
// Energy (MeV) to tally units: round to nearest (even) integer.  Below 2^31
// units (8 MeV) the 32-bit conversion; above, the value is an integer-valued
// float and is rebuilt exactly from its bits (m * 2^e, e >= 8), so no 64-bit
// conversion instruction is issued (those run on the narrow FP64 pipe).
__device__ __forceinline__ long long units_of(float scaled) {
    const int r = __float2int_rn(scaled);
    if (fabsf(scaled) < 2147483520.0f) return r;
    const unsigned b = __float_as_uint(scaled);
    const int e = (int)((b >> 23) & 0xffu) - 150;
    const long long v = (long long)((b & 0x7fffffu) | 0x800000u) << e;
    return (b >> 31) ? -v : v;
}
__device__ __forceinline__ long long units_of(double scaled) { return __double2ll_rn(scaled); }
__device__ __forceinline__ float unit_scale(float) { return kUnitsF; }
__device__ __forceinline__ double unit_scale(double) { return 268435456.0; }

template <bool AGG, bool SQ>
struct PendingTally {
    unsigned long long *tally;  // this history's tally (layer offset included)
    unsigned long long *sumsq;  // SQ: the squares tally, same offset
    int idx = -1;               // voxel of the pending deposit
    long long units = 0;
    __device__ __forceinline__ PendingTally(const ReplayArgs &P, long long tbase)
        : tally(P.tally + tbase), sumsq(SQ ? P.sumsq + tbase : nullptr) {}
    __device__ __forceinline__ void add(int v, long long u) {
        if (!SQ && !FDC_LANE_COALESCE) {
            if (u) tally_add<AGG>(tally, v, u);
            return;
        }
        if (v == idx) {
            units += u;
            return;
        }
        flush();
        idx = v;
        units = u;
    }
    // With SQ the pending sum is one whole visit of the history to the voxel;
    // its square goes to the second tally (2^-28 MeV^2 units):
    // (u * 2^-14)^2 = u^2 * 2^-28.
    __device__ __forceinline__ void flush() {
        if (idx >= 0 && units) {
            tally_add<AGG>(tally, idx, units);
            if (SQ) {
                const float e = (float)units * 6.103515625e-05f;
                const long long q = units_of(e * e);
                if (q) atomicAdd(sumsq + idx, (unsigned long long)q);
            }
        }
        idx = -1;
        units = 0;
    }
};

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ void raise_status(DeviceCounters *c, int code, unsigned long long h) {
    if (atomicCAS(&c->status, 0, code) == 0) c->bad_history = h;
}

// ---------------------------------------------------------------- task 2
// Deflection factors of a step: with the record's vector q = theta_w (cos
// phi, sin phi) and the angle-scaling factor f^2 = sum_i w_i k_theta_i^2, the
// scaled polar angle is theta_m = f |q| and the new direction is
//   sin(theta_m) (cos phi e1 + sin phi e2) + cos(theta_m) d
//     = sfac * (q_x e1 + q_y e2) + cos(theta_m) d,  sfac = sin(theta_m) / |q|.
// Below theta_m = 0.25 rad (almost every step) sfac = f sinc(theta_m) and
// cos(theta_m) come from their Taylor series in theta_m^2 (to theta^8 /
// theta^10, truncation < 1e-11), so neither |q| nor a trig call is needed;
// above, sincos of theta_m.
template <typename R>
__device__ __forceinline__ void deflection_factors(R qx, R qy, R f2, R *sfac, R *c) {
    const R q2 = qx * qx + qy * qy;
    const R t2 = q2 * f2;  // theta_m^2
    if (t2 < (R)0.0625) {
        const R sinc = (R)1 - t2 * ((R)(1.0 / 6) - t2 * ((R)(1.0 / 120) - t2 * ((R)(1.0 / 5040) - t2 * (R)(1.0 / 362880))));
        *sfac = sqrt_(f2) * sinc;
        *c = (R)1 - t2 * ((R)0.5 - t2 * ((R)(1.0 / 24) - t2 * ((R)(1.0 / 720) - t2 * (R)(1.0 / 40320))));
    } else {
        const R q = sqrt_(q2);
        R s;
        sincos_(q * sqrt_(f2), &s, c);
        *sfac = s / q;
    }
}

// Integer type of a step's running deposit: 32-bit when every step of the
// database is below 2^32 tally units, else 64-bit; seg() converts a segment's
// share (non-negative, rounded to nearest).
template <bool U32> struct Dep;
template <> struct Dep<true> {
    using type = unsigned;
    __device__ static __forceinline__ unsigned seg(float x) { return __float2uint_rn(x); }
    __device__ static __forceinline__ unsigned seg(double x) { return __double2uint_rn(x); }
};
template <> struct Dep<false> {
    using type = long long;
    __device__ static __forceinline__ long long seg(float x) { return units_of(x); }
    __device__ static __forceinline__ long long seg(double x) { return units_of(x); }
};

struct Counts32 {  // per-history counters added to the lane's totals on exit
    unsigned long long &steps, &segs;
    unsigned st = 0, sg = 0;
    __device__ __forceinline__ Counts32(unsigned long long &a, unsigned long long &b) : steps(a), segs(b) {}
    __device__ __forceinline__ ~Counts32() {
        steps += st;
        segs += sg;
    }
};

// Re-trace one history.  Positions are kept as the voxel index plus the
// fractional position inside the voxel, f in [0, 1] per axis (grid units:
// faces at integers), which keeps FP32 rounding relative to the voxel rather
// than to the whole grid; distances along the ray are in cm.  Per-lane
// counters are updated in place.
// FIXED: the voxel where a step starts scales the whole step (ablation of
// Sec. 2.2's step scaling); a template parameter, so the default path carries
// no per-segment test.
// ESEC: the database has local deposits (read per step from the esec side
// array); a template parameter so that runs without any carry no extra state.
// U32: every step of the database loses less than 2^32 tally units (16 MeV),
// so a step's running deposit and the units of its segments are 32-bit
// integers (the per-voxel tally and the escape bookkeeping stay 64-bit); the
// host picks it per database.
template <typename R, bool AGG, bool SQ, bool FIXED, bool ESEC, bool U32>
__device__ __forceinline__ void replay_history(const ReplayArgs &P, const Start &st,
                                               unsigned long long h, unsigned long long &steps_tot,
                                               unsigned long long &segs_tot, long long &replayed,
                                               long long &escaped) {
    if (st.k0 >= st.n) return;
    // per-history 32-bit step and segment counts, added to the lane's 64-bit
    // totals when the history ends (a history has fewer than 2^32 of either)
    Counts32 cnt(steps_tot, segs_tot);
    unsigned &steps = cnt.st, &segs = cnt.sg;
    const long long s_first = st.s0 + st.k0, s_end = st.s0 + st.n;
    const unsigned long long pol = evict_first_policy();
    uint4 rec = load_record(P.rec + s_first, pol);
#if FDC_RECORD_PREFETCH
    if (s_first + 8 < s_end) prefetch_l2(P.rec + ((s_first + 8) & ~7ll));
#endif
    // local deposit of the current step (side array, tracks that have any)
    float esec = ESEC ? __ldg(P.esec + s_first) : 0.0f;
    // energy of the replayed steps, in tally units
    const long long rep = units_of(__uint_as_float(rec.y) * kUnitsF) + units_of(esec * kUnitsF) +
                          __ldg(P.tail + s_first);
    replayed += rep;
    // entry on the upstream face; inside test and voxel in FP64 (the
    // per-proton state is FP32, the comparison is exact in FP64)
    const double xe = (double)st.x, ye = (double)st.y;
    if (!(xe >= P.x0 && xe < P.x1 && ye >= P.y0 && ye < P.y1)) {
        escaped += rep;  // misses the phantom: the whole history escapes
        return;
    }
    const double gx = (xe - P.x0) * P.idx_, gy = (ye - P.y0) * P.idy_;
    int ix = min((int)floor(gx), P.nx - 1), iy = min((int)floor(gy), P.ny - 1), iz = 0;
    R fx = (R)(gx - ix), fy = (R)(gy - iy), fz = (R)0;
    R dx = (R)0, dy = (R)0, dz = (R)1;
    const R ihx = sizeof(R) == 4 ? (R)P.ihx : (R)(1.0 / P.dx);
    const R ihy = sizeof(R) == 4 ? (R)P.ihy : (R)(1.0 / P.dy);
    const R ihz = sizeof(R) == 4 ? (R)P.ihz : (R)(1.0 / P.dz);
    const int sy = P.nx, sz = P.nx * P.ny;  // fewer than 2^31 voxels
    int v = ix + sy * iy;
    const long long tbase = P.per_layer ? (long long)st.layer * P.nvox : 0ll;
    const R psi = (R)st.psi;
    const int seg_cap = P.nx + P.ny + P.nz + 8;
    const R INF = inf_<R>();
    const R US = unit_scale((R)0);
    // material of the current voxel, carried from one step to the next
    float2 sk = __ldg(P.vox + v);
    PendingTally<AGG, SQ> pend(P, tbase);

    // the step loop walks the track's records with a pointer and a 32-bit
    // count of the steps left (a track has at most 2^22 steps)
    const uint4 *rp = P.rec + s_first;
    int left = (int)(s_end - s_first);
    for (;;) {
        const float dE_f = __uint_as_float(rec.y);
        const R len = (R)__uint_as_float(rec.x), dE = (R)dE_f;
        const long long Qk = units_of(dE_f * kUnitsF);
        const long long Qs = ESEC ? units_of(esec * kUnitsF) : 0ll;
        const R inv_len = rcp_(len);
        const R dEu = dE * inv_len * US;  // tally units per cm of water-equivalent length
        ++steps;

        // ray in grid units per cm; distances to the next faces (cm)
        const R rx = dx * ihx, ry = dy * ihy, rz = dz * ihz;
        // components below 1e-30 grid units per cm never reach a face
        const R tiny = (R)1e-30;
        const int stx = rx > tiny ? 1 : (rx < -tiny ? -1 : 0);
        const int sty = ry > tiny ? 1 : (ry < -tiny ? -1 : 0);
        const int stz = rz > tiny ? 1 : (rz < -tiny ? -1 : 0);
        const R irx = stx ? rcp_(rx) : INF;
        const R iry = sty ? rcp_(ry) : INF;
        const R irz = stz ? rcp_(rz) : INF;
        R tmx = stx ? ((R)(stx > 0) - fx) * irx : INF;
        R tmy = sty ? ((R)(sty > 0) - fy) * iry : INF;
        R tmz = stz ? ((R)(stz > 0) - fz) * irz : INF;
        const int ix0 = ix, iy0 = iy, iz0 = iz;
        const R tdx = fabs(irx), tdy = fabs(iry), tdz = fabs(irz);
        tmx = tmx > (R)0 ? tmx : (R)0;
        tmy = tmy > (R)0 ? tmy : (R)0;
        tmz = tmz > (R)0 ? tmz : (R)0;

        R rem = len, t = (R)0, acc = (R)0;
        // the step's units and the units deposited so far in it (32 bits when
        // every step fits; only these stay live across the segment loop)
        const typename Dep<U32>::type Qkd = (typename Dep<U32>::type)Qk;
        typename Dep<U32>::type dep = 0;
        constexpr bool fixed = FIXED;
        const R S_fix = (R)sk.x, k2_fix = (R)sk.y;
        int nseg = 0;
        bool gone = false;
        for (;;) {
            const R S = fixed ? S_fix : (R)sk.x, k2 = fixed ? k2_fix : (R)sk.y;
            // nearest face; ties go to x, then y, then z
            int a = 0;
            R tm = tmx;
            if (tmy < tm) { a = 1; tm = tmy; }
            if (tmz < tm) { a = 2; tm = tmz; }
            R seg = tm - t;
            seg = seg > (R)0 ? seg : (R)0;
            const R wexit = seg * S;
            ++segs;
            if (wexit >= rem) {  // the step ends in this voxel
                // the remainder may be a few units negative (rounded shares of the
                // earlier segments): formed in 64 bits; dep itself stays below 2^32
                const long long units = (long long)Qkd - (long long)dep;
                pend.add(v, units);
                acc += rem * k2;
                t += rem * rcp_(S);
                break;
            }
            const typename Dep<U32>::type units = Dep<U32>::seg(wexit * dEu);
            dep += units;
            pend.add(v, (long long)units);
            acc += wexit * k2;
            rem -= wexit;
            t = tm;
            bool out;
            if (a == 0) { ix += stx; v += stx; out = (unsigned)ix >= (unsigned)P.nx; tmx += tdx; }
            else if (a == 1) { iy += sty; v += sty * sy; out = (unsigned)iy >= (unsigned)P.ny; tmy += tdy; }
            else { iz += stz; v += stz * sz; out = (unsigned)iz >= (unsigned)P.nz; tmz += tdz; }
            if (out) {  // left the grid: the rest of the history escapes
                escaped += ((long long)Qkd - (long long)dep) + Qs + __ldg(P.tail + (rp - P.rec));
                gone = true;
                break;
            }
            if (++nseg > seg_cap) {
                raise_status(P.counters, FDC_ERR_STEP_LIMIT, h);
                gone = true;
                break;
            }
            sk = __ldg(P.vox + v);
        }
        if (gone) {
            pend.flush();
            return;
        }
        // fractional position in the end voxel
        fx = ((R)(ix0 - ix) + fx) + t * rx;
        fy = ((R)(iy0 - iy) + fy) + t * ry;
        fz = ((R)(iz0 - iz) + fz) + t * rz;
        if (ESEC && Qs) pend.add(v, Qs);
        if (--left == 0) {
            pend.flush();
            return;
        }
        ++rp;
        const R qx = (R)__uint_as_float(rec.z), qy = (R)__uint_as_float(rec.w);
        rec = load_record(rp, pol);  // next record: issued before the deflection arithmetic
        if (ESEC) esec = __ldg(P.esec + (rp - P.rec));
#if FDC_RECORD_PREFETCH
        if (((rp - P.rec) & 7) == 0 && left > 8) prefetch_l2(rp + 8);
#endif

        // deflection at the end of the step, scaled by the crossed materials
        R sfac, ct_;
        deflection_factors(qx, qy, acc * inv_len, &sfac, &ct_);
        const R a = sfac * qx, b = sfac * qy;  // sin(theta_m) cos(phi), sin(theta_m) sin(phi)
        const R p2 = dx * dx + dy * dy;
        R nx_, ny_, nz_;
        if (p2 > (R)0) {
            const R ip = rsqrt_(p2), p = p2 * ip;
            // e1 = (dx dz, dy dz, -p^2)/p, e2 = (-dy, dx, 0)/p
            const R az = a * dz * ip;
            nx_ = az * dx - b * (dy * ip) + ct_ * dx;
            ny_ = az * dy + b * (dx * ip) + ct_ * dy;
            nz_ = -a * p + ct_ * dz;
        } else {
            // along the beam axis: the frame is (x, sgn y) turned by sgn psi,
            // which makes the replay a rigid rotation of the track:
            // azimuth phi + sgn psi, expanded with the record's cos/sin phi
            const R sgn = dz > (R)0 ? (R)1 : (R)-1;
            R sps, cps;
            sincos_(psi, &sps, &cps);
            nx_ = a * cps - sgn * b * sps;
            ny_ = sgn * b * cps + a * sps;
            nz_ = sgn * ct_;
        }
        // the rotation keeps |d| = 1 up to rounding: in FP32 the norm random-walks
        // by a few 1e-7 per step (below 3e-6 after 400 steps), so the direction
        // is not renormalised (doing so every eighth step cost 2.8 %, the lanes
        // of a warp reaching that step at different iterations)
        dx = nx_;
        dy = ny_;
        dz = nz_;
    }
}

// Minimum resident CTAs of 256 threads per SM requested from the register
// allocator: 4 caps the kernel at 64 registers (no spills).  With 32 or more
// histories per track (a warp shares one track) the kernel is bound by
// instruction issue and 5 CTAs (48 registers, a few spills, 40 warps per SM)
// was measured 3 % faster; with independent tracks it is bound by the latency
// of scattered record loads and 5 was 12 % slower.
#ifndef FDC_REPLAY_MIN_CTAS
#define FDC_REPLAY_MIN_CTAS 4
#endif
#ifndef FDC_REPLAY_MIN_CTAS_SHARED
#define FDC_REPLAY_MIN_CTAS_SHARED 5
#endif

template <typename R, bool AGG, bool SQ, bool ESEC, bool U32, int MINB = FDC_REPLAY_MIN_CTAS>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? MINB : 2)
    replay_kernel(const ReplayArgs P) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long steps = 0, segs = 0, hist = 0;
    long long replayed = 0, escaped = 0;
    const unsigned long long claim = 32ull * (unsigned long long)P.chunk;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(P.work, claim);
        base = __shfl_sync(kFull, base, 0);
        if (base >= P.n) break;
        for (int c = 0; c < P.chunk; ++c) {
            const unsigned long long li = base + 32ull * c + lane;
            if (li < P.n) {
                const unsigned long long h = P.h_begin + li;
                const Start st = sample_start(P, h);
                if (P.scaling_mode == 1)
                    replay_history<R, AGG, SQ, true, ESEC, U32>(P, st, h, steps, segs, replayed, escaped);
                else
                    replay_history<R, AGG, SQ, false, ESEC, U32>(P, st, h, steps, segs, replayed, escaped);
                ++hist;
            }
        }
    }
    hist = warp_sum_u64(hist);
    steps = warp_sum_u64(steps);
    segs = warp_sum_u64(segs);
    replayed = (long long)warp_sum_u64((unsigned long long)replayed);
    escaped = (long long)warp_sum_u64((unsigned long long)escaped);
    if (lane == 0) {
        atomicAdd(&P.counters->histories, hist);
        atomicAdd(&P.counters->steps, steps);
        atomicAdd(&P.counters->segments, segs);
        atomicAdd((unsigned long long *)&P.counters->replayed, (unsigned long long)replayed);
        atomicAdd((unsigned long long *)&P.counters->escaped, (unsigned long long)escaped);
    }
}

// ---------------------------------------------------------------- finalize
// Sec. 2.3: energy per voxel divided by the voxel mass; FP64.
__global__ void finalize_kernel(const FinalizeArgs A) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < A.nvox; v += stride) {
        // the per-voxel factor, precomputed at phantom load when available (an
        // FP64 division per voxel costs more than the rest of this kernel on GB300)
        double f;
        if (A.factor) {
            f = A.factor[v];
        } else {
            const double rho = (double)A.density[v];
            f = rho > 0.0 ? A.scale / rho : 0.0;
        }
        long long tot = 0;
        for (int l = 0; l < A.n_tallies; ++l) {
            const long long t = A.tally[l * A.nvox + v];
            tot += t;
            if (A.layer_dose) A.layer_dose[l * A.nvox + v] = (double)t * f;
            if (A.accum) A.accum[l * A.nvox + v] += t;
            if (A.zero_after) A.tally[l * A.nvox + v] = 0;
        }
        const double d = (double)tot * f;
        if (A.hist_sumsq) {
            long long q = 0;
            for (int l = 0; l < A.n_tallies; ++l) q += A.sumsq[l * A.nvox + v];
            // squared tally units are 2^-28 MeV^2; f converts 2^-28 MeV to Gy
            A.hist_sumsq[v] = (double)q * f * (f * 268435456.0);
        }
        if (A.dose) A.dose[v] = d;
        if (A.tally_out) A.tally_out[v] = tot;
        if (A.batch_sum) A.batch_sum[v] += d;
        if (A.batch_sumsq) A.batch_sumsq[v] += d * d;
    }
}

// ---------------------------------------------------------------- statistics
// Eq. (1) per voxel from batch sums, then a deterministic two-level
// reduction: per-block partials (max of the mean; then masked sum and count
// of sigma/mean), combined by one block in a fixed order.
// mode 0, eq. (1): n batch doses, sigma = sqrt(sum (D_b - mean)^2 / (n (n-1)));
// mode 1, eq. (2): n histories, sigma = sqrt((s2/n - mean^2) / (n - 1)).
__global__ void stats_pass1(const double *sum, const double *sumsq, long long n, int mode, long long nvox,
                            double *mean, double *sigma, double *part_max) {
    __shared__ double sm[256];
    double mx = 0.0;
    const double dn = (double)n;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        const double s = sum[v], m = s / dn;
        double sg;
        if (mode == 0) {
            const double ss = sumsq[v] - s * s / dn;
            sg = sqrt((ss > 0.0 ? ss : 0.0) / (dn * (dn - 1.0)));
        } else {
            const double var = sumsq[v] / dn - m * m;
            sg = sqrt((var > 0.0 ? var : 0.0) / (dn - 1.0));
        }
        mean[v] = m;
        sigma[v] = sg;
        mx = m > mx ? m : mx;
    }
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part_max[blockIdx.x] = sm[0];
}

__global__ void stats_pass2(const double *mean, const double *sigma, long long nvox, double frac,
                            const double *part_max, int n_parts, double *part_sum, double *part_cnt) {
    __shared__ double s1[256], s2[256];
    double mx = 0.0;
    for (int i = 0; i < n_parts; ++i) mx = fmax(mx, part_max[i]);
    const double thr = frac * mx;
    double acc = 0.0, cnt = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        if (mean[v] > thr) {
            acc += sigma[v] / mean[v];
            cnt += 1.0;
        }
    }
    s1[threadIdx.x] = acc;
    s2[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_sum[blockIdx.x] = s1[0];
        part_cnt[blockIdx.x] = s2[0];
    }
}

__global__ void stats_pass3(const double *part_sum, const double *part_cnt, int n_parts, double *result) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int i = 0; i < n_parts; ++i) {
            a += part_sum[i];
            c += part_cnt[i];
        }
        result[0] = c > 0.0 ? a / c : __longlong_as_double(0x7ff8000000000000ll);
    }
}

// ---------------------------------------------------------------- test hooks
__global__ void debug_philox_kernel(unsigned long long k0, unsigned long long k1,
                                    const unsigned long long *ctr, unsigned long long n,
                                    unsigned long long *out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const U64x4 r = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
        out[4 * i] = r.v0;
        out[4 * i + 1] = r.v1;
        out[4 * i + 2] = r.v2;
        out[4 * i + 3] = r.v3;
    }
}

__global__ void debug_sample_kernel(const ReplayArgs P, float *xyEpsi, long long *btk) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < P.n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const Start st = sample_start(P, P.h_begin + i);
        xyEpsi[4 * i] = st.x;
        xyEpsi[4 * i + 1] = st.y;
        xyEpsi[4 * i + 2] = st.E;
        xyEpsi[4 * i + 3] = st.psi;
        btk[3 * i] = st.bin;
        btk[3 * i + 1] = st.track;
        btk[3 * i + 2] = st.k0;
    }
}

// Database load: each record's (theta, phi) becomes the deflection vector
// theta (cos phi, sin phi), computed in FP64 and rounded once to FP32.
__global__ void pack_deflections_kernel(uint4 *rec, long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        uint4 r = rec[i];
        const double th = (double)__uint_as_float(r.z), ph = (double)__uint_as_float(r.w);
        double sp, cp;
        sincos(ph, &sp, &cp);
        r.z = __float_as_uint((float)(th * cp));
        r.w = __float_as_uint((float)(th * sp));
        rec[i] = r;
    }
}

// One thread: prefix sum of the spots' history counts (cum[0] = 0).
__global__ void spot_prefix_kernel(const fdc_spot *spots, int n_spots, unsigned long long *cum) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long a = 0;
        cum[0] = 0;
        for (int i = 0; i < n_spots; ++i) {
            a += spots[i].n_histories;
            cum[i + 1] = a;
        }
    }
}

// 64-bit atomic adds of 1 to pseudo-random 8-byte slots (the access pattern
// of the dose tally without the transport): update i goes to slot
// mix(i) & mask, mask = n_slots - 1 with n_slots a power of two, so the
// address costs a multiply, a shift and two logic operations; each thread
// issues four independent updates per iteration (fire-and-forget reductions,
// several in flight).
__global__ void probe_atomics_kernel(unsigned long long *slots, unsigned long long mask,
                                     unsigned long long n_ops) {
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = 4 * tid; i < n_ops; i += 4 * nth) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i + u < n_ops) {
                unsigned long long x = (i + u) * 0x9E3779B97F4A7C15ull;
                x ^= x >> 29;
                atomicAdd(slots + (x & mask), 1ull);
            }
        }
    }
}

using ReplayFn = void (*)(ReplayArgs);

template <typename R, bool AGG, bool SQ, int MINB = FDC_REPLAY_MIN_CTAS>
ReplayFn replay_fn_t(bool esec, bool u32) {
    if (u32) return esec ? replay_kernel<R, AGG, SQ, true, true, MINB> : replay_kernel<R, AGG, SQ, false, true, MINB>;
    return esec ? replay_kernel<R, AGG, SQ, true, false, MINB> : replay_kernel<R, AGG, SQ, false, false, MINB>;
}

// The one place that maps a run to its kernel instantiation; the launch and
// the occupancy query (schedule limits, autotuner) both go through it.
//   squares: per-visit sums and plain atomics;  aggregate == 1: warp-combined
//   atomics;  FP32 with plain atomics and 32 or more histories per track: the
//   48-register variant;  esec: the database has local deposits.
ReplayFn replay_fn(const ReplayVariant &v) {
    const bool u = v.u32 != 0;
    if (v.squares) return v.fp64 ? replay_fn_t<double, false, true>(v.esec, u) : replay_fn_t<float, false, true>(v.esec, u);
    const bool agg = v.aggregate == 1;
    if (v.fp64) return agg ? replay_fn_t<double, true, false>(v.esec, u) : replay_fn_t<double, false, false>(v.esec, u);
    if (!agg && v.track_group >= 32) return replay_fn_t<float, false, false, FDC_REPLAY_MIN_CTAS_SHARED>(v.esec, u);
    return agg ? replay_fn_t<float, true, false>(v.esec, u) : replay_fn_t<float, false, false>(v.esec, u);
}

}  // namespace

// ---------------------------------------------------------------- static scratch
// The scratch of fdc_run_noalloc: one file-scope device array, resident on
// every GPU that loads the library.  Host code must not use the symbol itself
// as a pointer (on the host it is only a stand-in); noalloc_scratch() looks up
// its device address with cudaGetSymbolAddress, once per device, with that
// device current.
constexpr size_t kNoallocTallyBytes = 8ull * FDC_NOALLOC_MAX_VOXELS;
constexpr size_t kNoallocCountersOff = kNoallocTallyBytes;
constexpr size_t kNoallocWorkOff = kNoallocCountersOff + 128;
constexpr size_t kNoallocSpotsOff = kNoallocCountersOff + 256;
constexpr size_t kNoallocCumOff = kNoallocSpotsOff + sizeof(fdc_spot) * FDC_NOALLOC_MAX_SPOTS;
constexpr size_t kNoallocBytes = kNoallocCumOff + 8ull * (FDC_NOALLOC_MAX_SPOTS + 1) + 256;
static_assert(kNoallocBytes == FDC_NOALLOC_SCRATCH_BYTES, "scratch size in fdc.h");
static_assert(sizeof(DeviceCounters) <= 128, "counters slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_base[kMaxDevices] = {};
}  // namespace

cudaError_t noalloc_scratch(int device, NoallocScratch *out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_base[device]) {
            int cur = -1;
            cudaError_t e = cudaGetDevice(&cur);
            if (e != cudaSuccess) return e;
            if (cur != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (cur != device) cudaSetDevice(cur);
            if (e != cudaSuccess) return e;
            g_noalloc_base[device] = (unsigned char *)p;
        }
        base = g_noalloc_base[device];
    }
    out->tally = (unsigned long long *)base;
    out->counters = (DeviceCounters *)(base + kNoallocCountersOff);
    out->work = (unsigned long long *)(base + kNoallocWorkOff);
    out->spots = (fdc_spot *)(base + kNoallocSpotsOff);
    out->spot_cum = (unsigned long long *)(base + kNoallocCumOff);
    return cudaSuccess;
}

__global__ void dose_factor_kernel(const float *density, double scale, long long nvox, double *factor) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += stride) {
        const double rho = (double)density[v];
        factor[v] = rho > 0.0 ? scale / rho : 0.0;
    }
}

cudaError_t launch_dose_factor(const float *density, double scale, long long nvox, double *factor, cudaStream_t st) {
    long long blocks = (nvox + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    dose_factor_kernel<<<(int)blocks, 256, 0, st>>>(density, scale, nvox, factor);
    return cudaGetLastError();
}

cudaError_t launch_pack_deflections(uint4 *rec, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    pack_deflections_kernel<<<(int)blocks, 256, 0, st>>>(rec, n);
    return cudaGetLastError();
}

cudaError_t launch_spot_prefix(const fdc_spot *spots, int n_spots, unsigned long long *cum,
                               cudaStream_t st) {
    spot_prefix_kernel<<<1, 32, 0, st>>>(spots, n_spots, cum);
    return cudaGetLastError();
}

ReplayVariant replay_variant(const ReplayArgs &a, const fdc_schedule &s, int fp64) {
    ReplayVariant v;
    v.fp64 = fp64 ? 1 : 0;
    v.aggregate = s.aggregate;
    v.squares = a.sumsq ? 1 : 0;
    v.track_group = a.track_group;
    v.esec = a.esec ? 1 : 0;
    v.u32 = a.u32;
    return v;
}

cudaError_t launch_replay(const ReplayArgs &a, const fdc_schedule &s, int fp64, int sm_count,
                          cudaStream_t st) {
    const ReplayFn fn = replay_fn(replay_variant(a, s, fp64));
    ReplayArgs args = a;
    void *params[] = {&args};
    return cudaLaunchKernel((const void *)fn, dim3((unsigned)(sm_count * s.ctas_per_sm)),
                            dim3((unsigned)(32 * s.warps_per_cta)), params, 0, st);
}

int replay_max_ctas_per_sm(int warps_per_cta, const ReplayVariant &v) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void *)replay_fn(v), 32 * warps_per_cta, 0) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_probe_atomics(unsigned long long *slots, unsigned long long n_slots,
                                 unsigned long long n_ops, int sm_count, cudaStream_t st) {
    unsigned long long p2 = 1;  // largest power of two <= n_slots
    while (p2 <= n_slots / 2) p2 <<= 1;
    probe_atomics_kernel<<<sm_count * 8, 256, 0, st>>>(slots, p2 - 1, n_ops);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs &a, int sm_count, cudaStream_t st) {
    long long blocks = (a.nvox + 255) / 256;
    const long long cap = (long long)sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    finalize_kernel<<<(int)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_stats(const double *sum, const double *sumsq, long long n, int mode, long long nvox,
                               double frac, double *mean, double *sigma, double *partials,
                               int n_partials, double *result, cudaStream_t st) {
    // partials: [3][n_partials]
    stats_pass1<<<n_partials, 256, 0, st>>>(sum, sumsq, n, mode, nvox, mean, sigma, partials);
    stats_pass2<<<n_partials, 256, 0, st>>>(mean, sigma, nvox, frac, partials, n_partials,
                                            partials + n_partials, partials + 2 * n_partials);
    stats_pass3<<<1, 32, 0, st>>>(partials + n_partials, partials + 2 * n_partials, n_partials, result);
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(unsigned long long k0, unsigned long long k1,
                                const unsigned long long *ctr, unsigned long long n,
                                unsigned long long *out, cudaStream_t st) {
    unsigned long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    debug_philox_kernel<<<(unsigned)blocks, 256, 0, st>>>(k0, k1, ctr, n, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_sample(const ReplayArgs &a, float *xyEpsi, long long *btk, cudaStream_t st) {
    unsigned long long blocks = (a.n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    debug_sample_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, xyEpsi, btk);
    return cudaGetLastError();
}

}  // namespace fdc
