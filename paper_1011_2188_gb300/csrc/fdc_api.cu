// Host side of the C ABI declared in include/fdc.h: validation, packing of
// the track database into 16-byte step records, device buffers, and the run
// sequence (zero tally -> replay -> finalize) on the caller's stream.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "fdc.h"
#include "fdc_internal.h"

using fdc::DeviceCounters;

namespace {

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;  // capacity in elements
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t ensure(size_t count) {
        if (count <= n && p) return cudaSuccess;
        release();
        size_t c = count ? count : 1;
        cudaError_t e = cudaMalloc((void **)&p, c * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = c;
        return cudaSuccess;
    }
};

}  // namespace

namespace {
// Everything a captured run depends on; compared bytewise (zero-filled first).
struct GraphKey {
    fdc::ReplayArgs a;
    fdc_schedule sched;
    fdc_outputs out;
    int n_batches, n_tallies, fp64, timing;
};
}  // namespace

struct fdc_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err;
    // database
    bool db_loaded = false;
    int n_bins = 0;
    long long n_tracks = 0, n_steps = 0;
    long long max_track_units = 0;
    long long max_step_units = 0;  // largest energy loss of one step, tally units
    DevBuf<uint4> rec;
    bool has_esec = false;
    DevBuf<float> esec;
    DevBuf<unsigned char> trk_esec;
    DevBuf<float> eres;
    DevBuf<long long> tail;
    DevBuf<long long> step_begin;
    DevBuf<float> bin_energy;
    DevBuf<long long> bin_track_begin;
    // phantom
    bool ph_loaded = false;
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dy = 0, dz = 0, x0 = 0, y0 = 0, z0 = 0;
    long long nvox = 0;
    DevBuf<float2> vox;
    DevBuf<float> density;
    DevBuf<double> dfac;  // per-voxel dose factor of the finalize step (set at phantom load)
    // run scratch
    DevBuf<long long> tally, accum, sumsq;
    DevBuf<fdc_spot> spots;
    DevBuf<unsigned long long> spot_cum;
    DevBuf<DeviceCounters> counters;
    DevBuf<unsigned long long> work;
    DevBuf<double> stats_part;
    DevBuf<double> scratch_dose;
    // pinned staging of the beam; the event marks the last copy out of it
    void *beam_stage = nullptr;
    size_t beam_stage_bytes = 0;
    cudaEvent_t beam_copied = nullptr;
    std::vector<fdc_spot> beam_cache;  // spots currently on the device
    // optional kernel timing of the last run
    bool timing = false;
    bool timed = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // captured run sequence
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    GraphKey graph_key;
    // schedule picked by fdc_autotune and the instantiation it was tuned on
    fdc_schedule tuned = {0, 0, 0, 0};
    bool tuned_valid = false;
    fdc::ReplayVariant tuned_variant = {0, 0, 0, 1, 0, 0};
    int last_fp64 = 0;
};

namespace {

int fail(fdc_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(fdc_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? FDC_ERR_OOM : FDC_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define FDC_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

inline long long to_units_host(float e) { return llrint((double)e * fdc::kTallyUnitsPerMeV); }

bool finite_f(float v) { return std::isfinite(v); }

// Pinned staging buffer for chunked uploads.
struct Pinned {
    void *p = nullptr;
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
};

// Every step of the loaded database loses fewer than 2^32 tally units: the
// replay may keep a step's running deposit in 32 bits.  The rounded shares of
// a step's segments can add up to slightly more than the step (FP32 products,
// relative error ~2^-24 each), so the bound keeps a margin of 2^12 units.
bool step_units_fit_32(const fdc_ctx *c) { return c->max_step_units < (1ll << 32) - (1ll << 12); }

// The tuned schedule applies to runs of the kernel instantiation it was
// tuned on (aggregate aside, which the schedule itself picks).
bool same_tuning_class(const fdc::ReplayVariant &a, const fdc::ReplayVariant &b) {
    return a.fp64 == b.fp64 && a.squares == b.squares && a.esec == b.esec &&
           (a.track_group >= 32) == (b.track_group >= 32);
}

// Fill the zero fields of a requested schedule from the tuned schedule (when
// it was tuned on this run's kernel instantiation) or the built-in defaults;
// ctas_per_sm is bounded by the occupancy of the instantiation that will run.
int resolve_schedule(fdc_ctx *c, const fdc_schedule *req, fdc::ReplayVariant v, fdc_schedule *out) {
    fdc_schedule s = {0, 0, 0, 0};
    if (req) s = *req;
    const fdc_schedule t = (c->tuned_valid && same_tuning_class(c->tuned_variant, v)) ? c->tuned
                                                                                     : fdc_schedule{0, 0, 0, 0};
    if (!s.warps_per_cta) s.warps_per_cta = t.warps_per_cta ? t.warps_per_cta : 8;
    if (!s.chunk) s.chunk = t.chunk ? t.chunk : 1;
    // plain atomics by default: on GB300 the L2 absorbs the tally updates
    // faster than a match/redux combine across the warp
    if (!s.aggregate) s.aggregate = t.aggregate ? t.aggregate : 2;
    // the replay kernel is compiled for at most 256 threads per CTA
    if (s.warps_per_cta < 1 || s.warps_per_cta > 8 || s.chunk < 1 || s.chunk > 1024 || s.aggregate < 1 ||
        s.aggregate > 2 || s.ctas_per_sm < 0)
        return fail(c, FDC_ERR_INVALID, "invalid schedule");
    v.aggregate = s.aggregate;
    const int maxc = fdc::replay_max_ctas_per_sm(s.warps_per_cta, v);
    if (!s.ctas_per_sm) s.ctas_per_sm = t.ctas_per_sm ? std::min(t.ctas_per_sm, maxc) : maxc;
    if (s.ctas_per_sm > maxc) s.ctas_per_sm = maxc;
    *out = s;
    return FDC_OK;
}

// The kernel instantiation a run with these options selects (aggregate is
// filled in by resolve_schedule).
fdc::ReplayVariant run_variant(const fdc_ctx *c, const fdc_run_opts &o, bool squares) {
    fdc::ReplayVariant v;
    v.fp64 = o.fp64_geometry ? 1 : 0;
    v.aggregate = 0;
    v.squares = squares ? 1 : 0;
    v.track_group = o.track_group > 1 ? o.track_group : 1;
    v.esec = c->has_esec ? 1 : 0;
    v.u32 = step_units_fit_32(c) ? 1 : 0;
    return v;
}

struct BeamInfo {
    unsigned long long total = 0;
    int n_layers = 0;
};

int check_beam(fdc_ctx *c, const fdc_beam *b, BeamInfo *info) {
    if (!b || b->n_spots <= 0 || !b->spots) return fail(c, FDC_ERR_INVALID, "empty beam");
    unsigned long long tot = 0;
    int max_layer = 0;
    for (int i = 0; i < b->n_spots; ++i) {
        const fdc_spot &s = b->spots[i];
        if (s.profile < 0 || s.profile > 2) return fail(c, FDC_ERR_INVALID, "spot %d: bad profile", i);
        if (s.layer < 0 || s.layer > 65535) return fail(c, FDC_ERR_INVALID, "spot %d: bad layer", i);
        if (!std::isfinite(s.x) || !std::isfinite(s.y) || !std::isfinite(s.energy) ||
            !std::isfinite(s.sigma_e) || !std::isfinite(s.a) || !std::isfinite(s.b) || s.sigma_e < 0 ||
            s.a < 0 || s.b < 0)
            return fail(c, FDC_ERR_INVALID, "spot %d: bad parameters", i);
        if (tot + s.n_histories < tot) return fail(c, FDC_ERR_INVALID, "history count overflow");
        tot += s.n_histories;
        max_layer = std::max(max_layer, s.layer);
    }
    info->total = tot;
    info->n_layers = max_layer + 1;
    return FDC_OK;
}

// Copy the spots and their prefix sum to the device through pinned staging
// (asynchronous on st).  Skipped when the device already holds this beam,
// unless `force`.
int upload_beam(fdc_ctx *c, const fdc_beam *b, cudaStream_t st, bool force) {
    const size_t ns = (size_t)b->n_spots;
    if (!force && c->beam_cache.size() == ns &&
        std::memcmp(c->beam_cache.data(), b->spots, sizeof(fdc_spot) * ns) == 0)
        return FDC_OK;
    const size_t bytes = sizeof(fdc_spot) * ns + sizeof(unsigned long long) * (ns + 1);
    if (c->beam_copied) FDC_CUDA(c, cudaEventSynchronize(c->beam_copied));
    if (bytes > c->beam_stage_bytes) {
        if (c->beam_stage) cudaFreeHost(c->beam_stage);
        c->beam_stage = nullptr;
        c->beam_stage_bytes = 0;
        FDC_CUDA(c, cudaMallocHost(&c->beam_stage, bytes));
        c->beam_stage_bytes = bytes;
    }
    if (!c->beam_copied) FDC_CUDA(c, cudaEventCreateWithFlags(&c->beam_copied, cudaEventDisableTiming));
    fdc_spot *hs = (fdc_spot *)c->beam_stage;
    unsigned long long *hc = (unsigned long long *)(hs + ns);
    std::memcpy(hs, b->spots, sizeof(fdc_spot) * ns);
    hc[0] = 0;
    for (size_t i = 0; i < ns; ++i) hc[i + 1] = hc[i] + b->spots[i].n_histories;
    FDC_CUDA(c, c->spots.ensure(ns));
    FDC_CUDA(c, c->spot_cum.ensure(ns + 1));
    FDC_CUDA(c, cudaMemcpyAsync(c->spots.p, hs, sizeof(fdc_spot) * ns, cudaMemcpyHostToDevice, st));
    FDC_CUDA(c, cudaMemcpyAsync(c->spot_cum.p, hc, sizeof(unsigned long long) * (ns + 1), cudaMemcpyHostToDevice, st));
    FDC_CUDA(c, cudaEventRecord(c->beam_copied, st));
    c->beam_cache.assign(b->spots, b->spots + ns);
    return FDC_OK;
}

fdc::ReplayArgs base_args(fdc_ctx *c) {
    fdc::ReplayArgs a;
    std::memset(&a, 0, sizeof a);
    a.rec = c->rec.p;
    a.esec = c->has_esec ? c->esec.p : nullptr;
    a.trk_esec = c->trk_esec.p;
    a.eres = c->eres.p;
    a.tail = c->tail.p;
    a.step_begin = c->step_begin.p;
    a.bin_energy = c->bin_energy.p;
    a.bin_track_begin = c->bin_track_begin.p;
    a.n_bins = c->n_bins;
    a.vox = c->vox.p;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.dx = c->dx;
    a.dy = c->dy;
    a.dz = c->dz;
    a.x0 = c->x0;
    a.y0 = c->y0;
    a.z0 = c->z0;
    a.x1 = c->x0 + c->nx * c->dx;
    a.y1 = c->y0 + c->ny * c->dy;
    a.idx_ = 1.0 / c->dx;
    a.idy_ = 1.0 / c->dy;
    a.ihx = (float)(1.0 / c->dx);
    a.ihy = (float)(1.0 / c->dy);
    a.ihz = (float)(1.0 / c->dz);
    a.spots = c->spots.p;
    a.spot_cum = c->spot_cum.p;
    a.nvox = c->nvox;
    a.u32 = step_units_fit_32(c) ? 1 : 0;
    a.work = c->work.p;
    a.counters = c->counters.p;
    return a;
}

}  // namespace

extern "C" {

const char *fdc_last_error(const fdc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int fdc_create(fdc_ctx **out, int device) {
    if (!out) return FDC_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return FDC_ERR_CUDA;
    fdc_ctx *c = new fdc_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        c->counters.ensure(1) != cudaSuccess || c->work.ensure(1) != cudaSuccess ||
        cudaMemset(c->counters.p, 0, sizeof(DeviceCounters)) != cudaSuccess) {
        delete c;
        return FDC_ERR_CUDA;
    }
    *out = c;
    return FDC_OK;
}

void fdc_destroy(fdc_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    c->rec.release();
    c->esec.release();
    c->trk_esec.release();
    c->eres.release();
    c->tail.release();
    c->step_begin.release();
    c->bin_energy.release();
    c->bin_track_begin.release();
    c->vox.release();
    c->density.release();
    c->dfac.release();
    c->tally.release();
    c->accum.release();
    c->sumsq.release();
    c->spots.release();
    c->spot_cum.release();
    c->counters.release();
    c->work.release();
    c->stats_part.release();
    c->scratch_dose.release();
    if (c->beam_stage) cudaFreeHost(c->beam_stage);
    if (c->beam_copied) cudaEventDestroy(c->beam_copied);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

int fdc_load_database(fdc_ctx *c, const fdc_database *db) {
    if (!c) return FDC_ERR_INVALID;
    if (!db || db->n_energies <= 0 || !db->energy || !db->track_begin || !db->step_begin || !db->dE ||
        !db->len || !db->theta || !db->phi || !db->esec)
        return fail(c, FDC_ERR_INVALID, "database: missing arrays");
    FDC_CUDA(c, cudaSetDevice(c->device));
    const int nb = db->n_energies;
    for (int b = 0; b < nb; ++b) {
        if (!finite_f(db->energy[b]) || db->energy[b] <= 0.0f) return fail(c, FDC_ERR_INVALID, "database: bad bin energy");
        if (b && !(db->energy[b] > db->energy[b - 1])) return fail(c, FDC_ERR_INVALID, "database: bin energies not increasing");
    }
    if (db->track_begin[0] != 0) return fail(c, FDC_ERR_INVALID, "database: track_begin[0] != 0");
    for (int b = 0; b < nb; ++b)
        if (db->track_begin[b + 1] <= db->track_begin[b]) return fail(c, FDC_ERR_INVALID, "database: empty energy bin %d", b);
    const long long nt = db->track_begin[nb];
    if (db->step_begin[0] != 0) return fail(c, FDC_ERR_INVALID, "database: step_begin[0] != 0");
    const long long kMaxTrack = 1 << 22;
    for (long long t = 0; t < nt; ++t) {
        const long long n = db->step_begin[t + 1] - db->step_begin[t];
        if (n < 0 || n > kMaxTrack) return fail(c, FDC_ERR_INVALID, "database: bad step range for track %lld", t);
    }
    const long long ns = db->step_begin[nt];
    for (long long k = 0; k < ns; ++k) {
        const float l = db->len[k], e = db->dE[k], s = db->esec[k], th = db->theta[k], ph = db->phi[k];
        if (!finite_f(l) || !(l > 0.0f) || !finite_f(e) || e < 0.0f || !finite_f(s) || s < 0.0f ||
            !finite_f(th) || th < 0.0f || th > 3.1416f || !finite_f(ph))
            return fail(c, FDC_ERR_INVALID, "database: bad step record %lld", k);
        if (e > 1.0e6f || s > 1.0e6f) return fail(c, FDC_ERR_OVERFLOW, "database: step energy %lld beyond the fixed-point range", k);
    }
    // tracks with local deposits (the kernel reads the esec side array only for those)
    std::vector<unsigned char> trk_esec((size_t)std::max<long long>(nt, 1), 0);
    bool any_esec = false;
    for (long long t = 0; t < nt; ++t)
        for (long long k = db->step_begin[t]; k < db->step_begin[t + 1]; ++k)
            if (db->esec[k] != 0.0f) {
                trk_esec[t] = 1;
                any_esec = true;
                break;
            }
    // ---- device buffers
    c->db_loaded = false;
    FDC_CUDA(c, c->rec.ensure(ns));
    FDC_CUDA(c, c->eres.ensure(ns));
    FDC_CUDA(c, c->tail.ensure(ns));
    FDC_CUDA(c, c->step_begin.ensure(nt + 1));
    FDC_CUDA(c, c->trk_esec.ensure(nt));
    FDC_CUDA(c, c->bin_energy.ensure(nb));
    FDC_CUDA(c, c->bin_track_begin.ensure(nb + 1));
    FDC_CUDA(c, cudaMemcpy(c->step_begin.p, db->step_begin, sizeof(long long) * (nt + 1), cudaMemcpyHostToDevice));
    FDC_CUDA(c, cudaMemcpy(c->trk_esec.p, trk_esec.data(), (size_t)nt, cudaMemcpyHostToDevice));
    FDC_CUDA(c, cudaMemcpy(c->bin_energy.p, db->energy, sizeof(float) * nb, cudaMemcpyHostToDevice));
    FDC_CUDA(c, cudaMemcpy(c->bin_track_begin.p, db->track_begin, sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice));
    if (any_esec) {
        FDC_CUDA(c, c->esec.ensure(ns));
        FDC_CUDA(c, cudaMemcpy(c->esec.p, db->esec, sizeof(float) * ns, cudaMemcpyHostToDevice));
    } else {
        c->esec.release();
    }
    c->has_esec = any_esec;
    // ---- pack in chunks of whole tracks through pinned staging; the
    // deflection vector of each record is formed on the device after the copy
    const long long CH = std::max<long long>(1 << 22, kMaxTrack);
    Pinned prec, peres, ptail;
    FDC_CUDA(c, cudaMallocHost(&prec.p, sizeof(uint4) * CH));
    FDC_CUDA(c, cudaMallocHost(&peres.p, sizeof(float) * CH));
    FDC_CUDA(c, cudaMallocHost(&ptail.p, sizeof(long long) * CH));
    uint4 *hr = (uint4 *)prec.p;
    float *he = (float *)peres.p;
    long long *ht = (long long *)ptail.p;
    long long chunk_first = 0, fill = 0, max_units = 0, max_step = 0;
    auto flush = [&]() -> int {
        if (!fill) return FDC_OK;
        FDC_CUDA(c, cudaMemcpy(c->rec.p + chunk_first, hr, sizeof(uint4) * fill, cudaMemcpyHostToDevice));
        FDC_CUDA(c, fdc::launch_pack_deflections(c->rec.p + chunk_first, fill, nullptr));
        FDC_CUDA(c, cudaMemcpy(c->eres.p + chunk_first, he, sizeof(float) * fill, cudaMemcpyHostToDevice));
        FDC_CUDA(c, cudaMemcpy(c->tail.p + chunk_first, ht, sizeof(long long) * fill, cudaMemcpyHostToDevice));
        // the pinned record staging is refilled next: wait for the packing kernel
        FDC_CUDA(c, cudaDeviceSynchronize());
        chunk_first += fill;
        fill = 0;
        return FDC_OK;
    };
    for (int b = 0; b < nb; ++b) {
        const double Eb = (double)db->energy[b];
        for (long long t = db->track_begin[b]; t < db->track_begin[b + 1]; ++t) {
            const long long s0 = db->step_begin[t], n = db->step_begin[t + 1] - s0;
            if (fill + n > CH) {
                int rc = flush();
                if (rc) return rc;
            }
            double used = 0.0;
            for (long long k = 0; k < n; ++k) {
                const long long g = s0 + k;
                // residual energy at step start, summed in FP64 in step order
                he[fill + k] = (float)(Eb - used);
                used += (double)db->dE[g] + (double)db->esec[g];
                uint4 r;
                const float l = db->len[g], e = db->dE[g], th = db->theta[g], ph = db->phi[g];
                std::memcpy(&r.x, &l, 4);
                std::memcpy(&r.y, &e, 4);
                std::memcpy(&r.z, &th, 4);  // (theta, phi) until packed on the device
                std::memcpy(&r.w, &ph, 4);
                hr[fill + k] = r;
            }
            long long acc = 0;
            for (long long k = n - 1; k >= 0; --k) {
                ht[fill + k] = acc;
                const long long ue = to_units_host(db->dE[s0 + k]);
                max_step = std::max(max_step, ue);
                acc += ue + to_units_host(db->esec[s0 + k]);
            }
            max_units = std::max(max_units, acc);
            fill += n;
        }
    }
    int rc = flush();
    if (rc) return rc;
    c->n_bins = nb;
    c->n_tracks = nt;
    c->n_steps = ns;
    c->max_track_units = max_units;
    c->max_step_units = max_step;
    c->db_loaded = true;
    return FDC_OK;
}

int fdc_load_phantom(fdc_ctx *c, const fdc_phantom *ph) {
    if (!c) return FDC_ERR_INVALID;
    if (!ph || !ph->material || !ph->density || !ph->s_rel || !ph->k_theta)
        return fail(c, FDC_ERR_INVALID, "phantom: missing arrays");
    if (ph->nx <= 0 || ph->ny <= 0 || ph->nz <= 0 || ph->n_mat <= 0 || ph->n_mat > 256)
        return fail(c, FDC_ERR_INVALID, "phantom: bad dimensions");
    if (!(ph->dx > 0 && ph->dy > 0 && ph->dz > 0) || !std::isfinite(ph->dx) || !std::isfinite(ph->dy) ||
        !std::isfinite(ph->dz) || !std::isfinite(ph->x0) || !std::isfinite(ph->y0) || !std::isfinite(ph->z0))
        return fail(c, FDC_ERR_INVALID, "phantom: bad spacing or origin");
    const long long nvox = (long long)ph->nx * ph->ny * ph->nz;
    if (nvox >= (1ll << 31)) return fail(c, FDC_ERR_INVALID, "phantom: more than 2^31 - 1 voxels");
    for (int m = 0; m < ph->n_mat; ++m)
        if (!finite_f(ph->s_rel[m]) || ph->s_rel[m] < 0 || !finite_f(ph->k_theta[m]) || ph->k_theta[m] < 0)
            return fail(c, FDC_ERR_INVALID, "phantom: bad material %d", m);
    FDC_CUDA(c, cudaSetDevice(c->device));
    std::vector<float2> vox(nvox);
    for (long long v = 0; v < nvox; ++v) {
        const int m = ph->material[v];
        const float rho = ph->density[v];
        if (m >= ph->n_mat) return fail(c, FDC_ERR_INVALID, "phantom: material index out of range at %lld", v);
        if (!finite_f(rho) || rho < 0) return fail(c, FDC_ERR_INVALID, "phantom: bad density at %lld", v);
        vox[v] = make_float2(rho * ph->s_rel[m], ph->k_theta[m] * ph->k_theta[m]);
    }
    c->ph_loaded = false;
    FDC_CUDA(c, c->vox.ensure(nvox));
    FDC_CUDA(c, c->density.ensure(nvox));
    FDC_CUDA(c, cudaMemcpy(c->vox.p, vox.data(), sizeof(float2) * nvox, cudaMemcpyHostToDevice));
    FDC_CUDA(c, cudaMemcpy(c->density.p, ph->density, sizeof(float) * nvox, cudaMemcpyHostToDevice));
    c->nx = ph->nx;
    c->ny = ph->ny;
    c->nz = ph->nz;
    c->dx = ph->dx;
    c->dy = ph->dy;
    c->dz = ph->dz;
    FDC_CUDA(c, c->dfac.ensure(nvox));
    FDC_CUDA(c, fdc::launch_dose_factor(c->density.p,
                                        fdc::kMeVToJ / (fdc::kTallyUnitsPerMeV * c->dx * c->dy * c->dz * 1e-3), nvox,
                                        c->dfac.p, nullptr));
    FDC_CUDA(c, cudaStreamSynchronize(nullptr));
    c->x0 = ph->x0;
    c->y0 = ph->y0;
    c->z0 = ph->z0;
    c->nvox = nvox;
    c->ph_loaded = true;
    return FDC_OK;
}

}  // extern "C"

namespace {

// fdc_run_ex; force_upload copies the beam in even when the device holds it.
int run_impl(fdc_ctx *c, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
             const fdc_run_opts *opts_in, const fdc_outputs *out_in, void *stream, bool force_upload) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->db_loaded || !c->ph_loaded) return fail(c, FDC_ERR_NOT_LOADED, "database and phantom must be loaded");
    fdc_run_opts opts;
    std::memset(&opts, 0, sizeof opts);
    if (opts_in) opts = *opts_in;
    fdc_outputs out;
    std::memset(&out, 0, sizeof out);
    if (out_in) out = *out_in;
    BeamInfo bi;
    int rc = check_beam(c, beam, &bi);
    if (rc) return rc;
    if (opts.history_offset > bi.total) return fail(c, FDC_ERR_INVALID, "history offset beyond the beam");
    unsigned long long n = n_histories ? n_histories : bi.total - opts.history_offset;
    if (n > bi.total - opts.history_offset) return fail(c, FDC_ERR_INVALID, "more histories than the beam holds");
    if (opts.track_group < 0 || opts.scaling_mode < 0 || opts.scaling_mode > 1 || opts.n_batches < 0 ||
        opts.fp64_geometry < 0 || opts.fp64_geometry > 1 || opts.no_rotation < 0 || opts.no_rotation > 1)
        return fail(c, FDC_ERR_INVALID, "invalid run options");
    const int n_batches = opts.n_batches < 2 ? 1 : opts.n_batches;
    if (n_batches > 1 && (unsigned long long)n_batches > n) return fail(c, FDC_ERR_INVALID, "more batches than histories");
    if ((out.batch_sum || out.batch_sumsq) && n_batches < 2)
        return fail(c, FDC_ERR_INVALID, "batch outputs need n_batches >= 2");
    // fixed-point headroom: every history of one launch into one voxel
    const unsigned long long per_launch = (n + n_batches - 1) / n_batches;
    if (c->max_track_units > 0 &&
        (double)per_launch * (double)c->max_track_units > 9.0e18)
        return fail(c, FDC_ERR_OVERFLOW, "too many histories per launch for the int64 tally");
    fdc_schedule sched;
    rc = resolve_schedule(c, &opts.schedule, run_variant(c, opts, out.history_sumsq != nullptr), &sched);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    FDC_CUDA(c, cudaSetDevice(c->device));

    const int n_tallies = out.layer_dose ? bi.n_layers : 1;
    const long long tsize = (long long)n_tallies * c->nvox;
    FDC_CUDA(c, c->tally.ensure(tsize));
    if (n_batches > 1) FDC_CUDA(c, c->accum.ensure(tsize));
    if (out.history_sumsq) FDC_CUDA(c, c->sumsq.ensure(tsize));
    rc = upload_beam(c, beam, st, force_upload);
    if (rc) return rc;
    fdc::ReplayArgs a = base_args(c);
    a.tally = (unsigned long long *)c->tally.p;
    a.per_layer = n_tallies > 1 ? 1 : 0;
    a.n_spots = beam->n_spots;
    a.seed = seed;
    a.track_group = opts.track_group > 1 ? opts.track_group : 1;
    a.rotate = opts.no_rotation ? 0 : 1;
    a.scaling_mode = opts.scaling_mode;
    a.chunk = sched.chunk;
    a.h_begin = opts.history_offset;
    a.n = n;
    a.sumsq = out.history_sumsq ? (unsigned long long *)c->sumsq.p : nullptr;
    const double scale = fdc::kMeVToJ / (fdc::kTallyUnitsPerMeV * c->dx * c->dy * c->dz * 1e-3);

    // The whole run as one sequence of stream operations: zero the counters
    // and tallies, per batch one replay launch (plus the fold of the batch
    // into the FP64 sums), then the dose.
    auto issue = [&](cudaStream_t s) -> int {
        FDC_CUDA(c, cudaMemsetAsync(c->counters.p, 0, sizeof(DeviceCounters), s));
        FDC_CUDA(c, cudaMemsetAsync(c->tally.p, 0, sizeof(long long) * tsize, s));
        if (a.sumsq) FDC_CUDA(c, cudaMemsetAsync(c->sumsq.p, 0, sizeof(long long) * tsize, s));
        if (n_batches > 1) {
            FDC_CUDA(c, cudaMemsetAsync(c->accum.p, 0, sizeof(long long) * tsize, s));
            if (out.batch_sum) FDC_CUDA(c, cudaMemsetAsync(out.batch_sum, 0, sizeof(double) * c->nvox, s));
            if (out.batch_sumsq) FDC_CUDA(c, cudaMemsetAsync(out.batch_sumsq, 0, sizeof(double) * c->nvox, s));
        }
        if (c->timing) FDC_CUDA(c, cudaEventRecord(c->ev[0], s));
        fdc::ReplayArgs ab = a;
        for (int b = 0; b < n_batches; ++b) {
            const unsigned long long lo = n * (unsigned long long)b / n_batches;
            const unsigned long long hi = n * (unsigned long long)(b + 1) / n_batches;
            ab.h_begin = opts.history_offset + lo;
            ab.n = hi - lo;
            FDC_CUDA(c, cudaMemsetAsync(c->work.p, 0, sizeof(unsigned long long), s));
            if (ab.n) FDC_CUDA(c, fdc::launch_replay(ab, sched, opts.fp64_geometry, c->sm_count, s));
            if (n_batches > 1) {
                fdc::FinalizeArgs f;
                std::memset(&f, 0, sizeof f);
                f.tally = c->tally.p;
                f.n_tallies = n_tallies;
                f.nvox = c->nvox;
                f.density = c->density.p;
                f.factor = c->dfac.p;
                f.scale = scale;
                f.batch_sum = out.batch_sum;
                f.batch_sumsq = out.batch_sumsq;
                f.accum = c->accum.p;
                f.zero_after = 1;
                FDC_CUDA(c, fdc::launch_finalize(f, c->sm_count, s));
            }
        }
        if (c->timing) FDC_CUDA(c, cudaEventRecord(c->ev[1], s));
        if (c->timing) FDC_CUDA(c, cudaEventRecord(c->ev[2], s));
        if (out.dose || out.layer_dose || out.tally || out.history_sumsq) {
            fdc::FinalizeArgs f;
            std::memset(&f, 0, sizeof f);
            f.tally = n_batches > 1 ? c->accum.p : c->tally.p;
            f.sumsq = a.sumsq ? c->sumsq.p : nullptr;
            f.hist_sumsq = out.history_sumsq;
            f.n_tallies = n_tallies;
            f.nvox = c->nvox;
            f.density = c->density.p;
            f.factor = c->dfac.p;
            f.scale = scale;
            f.dose = out.dose;
            f.layer_dose = out.layer_dose;
            f.tally_out = (long long *)out.tally;
            FDC_CUDA(c, fdc::launch_finalize(f, c->sm_count, s));
        }
        if (c->timing) FDC_CUDA(c, cudaEventRecord(c->ev[3], s));
        return FDC_OK;
    };

    c->timed = false;
    // timed runs issue their launches directly: events recorded inside a
    // stream capture only order the capture and cannot be read back
    if (opts.no_graph || c->timing) {
        rc = issue(st);
        if (rc) return rc;
    } else {
        // CUDA graph of the sequence, captured on the context's own stream and
        // relaunched on the caller's stream while the launch configuration
        // (every kernel argument, buffer and schedule) stays the same.
        GraphKey key;
        std::memset(&key, 0, sizeof key);
        key.a = a;
        key.sched = sched;
        key.out = out;
        key.n_batches = n_batches;
        key.n_tallies = n_tallies;
        key.fp64 = opts.fp64_geometry;
        key.timing = c->timing ? 1 : 0;
        if (!c->graph_exec || std::memcmp(&key, &c->graph_key, sizeof key) != 0) {
            if (!c->cap_stream) FDC_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            FDC_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = issue(c->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ec != cudaSuccess) return cuda_fail(c, ec, "cudaStreamEndCapture");
            bool updated = false;
            if (c->graph_exec) {
                cudaGraphExecUpdateResultInfo info;
                updated = cudaGraphExecUpdate(c->graph_exec, g, &info) == cudaSuccess;
                if (!updated) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(c->graph_exec);
                    c->graph_exec = nullptr;
                }
            }
            if (!updated) {
                cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, g, 0);
                if (ei != cudaSuccess) {
                    cudaGraphDestroy(g);
                    c->graph_exec = nullptr;
                    return cuda_fail(c, ei, "cudaGraphInstantiate");
                }
            }
            cudaGraphDestroy(g);
            c->graph_key = key;
        }
        FDC_CUDA(c, cudaGraphLaunch(c->graph_exec, st));
    }
    if (c->timing) c->timed = true;
    c->last_fp64 = opts.fp64_geometry;
    return FDC_OK;
}

}  // namespace

extern "C" {

int fdc_run_ex(fdc_ctx *c, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
               const fdc_run_opts *opts, const fdc_outputs *out, void *stream) {
    return run_impl(c, beam, n_histories, seed, opts, out, stream, false);
}

int fdc_run(fdc_ctx *c, const fdc_beam *beam, uint64_t n_histories, uint64_t seed, double *dose_out,
            void *stream) {
    if (!c) return FDC_ERR_INVALID;
    if (!dose_out) return fail(c, FDC_ERR_INVALID, "dose_out is null");
    fdc_outputs out;
    std::memset(&out, 0, sizeof out);
    out.dose = dose_out;
    return fdc_run_ex(c, beam, n_histories, seed, nullptr, &out, stream);
}

int fdc_dose_from_tally(fdc_ctx *c, const int64_t *tally, double *dose_out, void *stream) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->ph_loaded) return fail(c, FDC_ERR_NOT_LOADED, "phantom must be loaded");
    if (!tally || !dose_out) return fail(c, FDC_ERR_INVALID, "dose_from_tally: null pointer");
    FDC_CUDA(c, cudaSetDevice(c->device));
    fdc::FinalizeArgs f;
    std::memset(&f, 0, sizeof f);
    f.tally = (long long *)tally;  // read only: zero_after stays 0
    f.n_tallies = 1;
    f.nvox = c->nvox;
    f.density = c->density.p;
    f.factor = c->dfac.p;
    f.scale = fdc::kMeVToJ / (fdc::kTallyUnitsPerMeV * c->dx * c->dy * c->dz * 1e-3);
    f.dose = dose_out;
    FDC_CUDA(c, fdc::launch_finalize(f, c->sm_count, (cudaStream_t)stream));
    return FDC_OK;
}

int fdc_sync(fdc_ctx *c, void *stream, fdc_counters *counters) {
    if (!c) return FDC_ERR_INVALID;
    FDC_CUDA(c, cudaSetDevice(c->device));
    FDC_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
    DeviceCounters h;
    FDC_CUDA(c, cudaMemcpy(&h, c->counters.p, sizeof h, cudaMemcpyDeviceToHost));
    if (counters) std::memcpy(counters, &h, sizeof h);
    if (h.status) return fail(c, h.status, "device status %d at history %llu", h.status, h.bad_history);
    return FDC_OK;
}

int fdc_run_host(fdc_ctx *c, const fdc_beam *beam, uint64_t n_histories, uint64_t seed, const fdc_run_opts *opts,
                 double *dose_host) {
    if (!c) return FDC_ERR_INVALID;
    if (!dose_host) return fail(c, FDC_ERR_INVALID, "dose_host is null");
    if (!c->ph_loaded) return fail(c, FDC_ERR_NOT_LOADED, "phantom must be loaded");
    FDC_CUDA(c, cudaSetDevice(c->device));
    FDC_CUDA(c, c->scratch_dose.ensure(c->nvox));
    fdc_outputs out;
    std::memset(&out, 0, sizeof out);
    out.dose = c->scratch_dose.p;
    // the beam is this call's input: always copy it in
    int rc = run_impl(c, beam, n_histories, seed, opts, &out, nullptr, true);
    if (rc) return rc;
    FDC_CUDA(c, cudaMemcpyAsync(dose_host, c->scratch_dose.p, sizeof(double) * c->nvox, cudaMemcpyDeviceToHost, nullptr));
    return fdc_sync(c, nullptr, nullptr);
}

int fdc_batch_stats(fdc_ctx *c, const double *batch_sum, const double *batch_sumsq, int32_t n_batches,
                    double frac, double *mean, double *sigma, double *mean_rel, void *stream) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->ph_loaded) return fail(c, FDC_ERR_NOT_LOADED, "phantom must be loaded");
    if (!batch_sum || !batch_sumsq || !mean || !sigma || n_batches < 2 || !(frac >= 0.0))
        return fail(c, FDC_ERR_INVALID, "batch stats: bad arguments");
    FDC_CUDA(c, cudaSetDevice(c->device));
    const int parts = std::max(1, std::min<int>(c->sm_count * 2, (int)((c->nvox + 255) / 256)));
    FDC_CUDA(c, c->stats_part.ensure(3 * parts + 1));
    cudaStream_t st = (cudaStream_t)stream;
    FDC_CUDA(c, fdc::launch_batch_stats(batch_sum, batch_sumsq, n_batches, 0, c->nvox, frac, mean, sigma,
                                        c->stats_part.p, parts, c->stats_part.p + 3 * parts, st));
    double r = 0;
    FDC_CUDA(c, cudaMemcpyAsync(&r, c->stats_part.p + 3 * parts, sizeof r, cudaMemcpyDeviceToHost, st));
    FDC_CUDA(c, cudaStreamSynchronize(st));
    if (mean_rel) *mean_rel = r;
    return FDC_OK;
}

int fdc_history_stats(fdc_ctx *c, const double *dose_sum, const double *history_sumsq, uint64_t n_histories,
                      double frac, double *mean, double *sigma, double *mean_rel, void *stream) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->ph_loaded) return fail(c, FDC_ERR_NOT_LOADED, "phantom must be loaded");
    if (!dose_sum || !history_sumsq || !mean || !sigma || n_histories < 2 || !(frac >= 0.0))
        return fail(c, FDC_ERR_INVALID, "history stats: bad arguments");
    FDC_CUDA(c, cudaSetDevice(c->device));
    const int parts = std::max(1, std::min<int>(c->sm_count * 2, (int)((c->nvox + 255) / 256)));
    FDC_CUDA(c, c->stats_part.ensure(3 * parts + 1));
    cudaStream_t st = (cudaStream_t)stream;
    FDC_CUDA(c, fdc::launch_batch_stats(dose_sum, history_sumsq, (long long)n_histories, 1, c->nvox, frac, mean,
                                        sigma, c->stats_part.p, parts, c->stats_part.p + 3 * parts, st));
    double r = 0;
    FDC_CUDA(c, cudaMemcpyAsync(&r, c->stats_part.p + 3 * parts, sizeof r, cudaMemcpyDeviceToHost, st));
    FDC_CUDA(c, cudaStreamSynchronize(st));
    if (mean_rel) *mean_rel = r;
    return FDC_OK;
}

int fdc_autotune(fdc_ctx *c, const fdc_beam *beam, uint64_t n_histories, uint64_t seed,
                 const fdc_run_opts *opts_in, fdc_schedule *best) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->db_loaded || !c->ph_loaded) return fail(c, FDC_ERR_NOT_LOADED, "database and phantom must be loaded");
    FDC_CUDA(c, cudaSetDevice(c->device));
    FDC_CUDA(c, c->scratch_dose.ensure(c->nvox));
    fdc_run_opts base;
    std::memset(&base, 0, sizeof base);
    if (opts_in) base = *opts_in;
    base.n_batches = 0;
    std::memset(&base.schedule, 0, sizeof base.schedule);
    const fdc::ReplayVariant var = run_variant(c, base, false);
    // candidates: the built-in default first, then warps x CTAs x chunk x
    // aggregate, each CTA count bounded by the occupancy of the instantiation
    // that candidate launches
    std::vector<fdc_schedule> cand;
    {
        const bool was_valid = c->tuned_valid;
        c->tuned_valid = false;
        fdc_schedule d;
        int rc0 = resolve_schedule(c, nullptr, var, &d);
        c->tuned_valid = was_valid;
        if (rc0) return rc0;
        cand.push_back(d);
    }
    for (int w : {4, 8}) {
        for (int ag : {2, 1}) {
            fdc::ReplayVariant v = var;
            v.aggregate = ag;
            const int maxc = fdc::replay_max_ctas_per_sm(w, v);
            std::vector<int> ctas = {maxc};
            if (maxc > 1) ctas.push_back(maxc - 1);
            if (maxc > 3) ctas.push_back(maxc / 2);
            for (int ct : ctas)
                for (int ch : {1, 2, 8}) cand.push_back(fdc_schedule{ct, w, ch, ag});
        }
    }
    fdc_outputs out;
    std::memset(&out, 0, sizeof out);
    out.dose = c->scratch_dose.p;
    const bool timing_before = c->timing;
    int rc = fdc_set_timing(c, 1);
    if (rc) return rc;
    fdc_schedule best_s = cand[0];
    double best_ms = std::numeric_limits<double>::max();
    // one warm-up launch of the first candidate, then per candidate the best
    // of three replay-kernel times (CUDA events around the launch)
    for (size_t i = 0; i < cand.size() && !rc; ++i) {
        fdc_run_opts o = base;
        o.no_graph = 1;
        o.schedule = cand[i];
        double ms_min = std::numeric_limits<double>::max();
        for (int rep = 0; rep < (i == 0 ? 4 : 3) && !rc; ++rep) {
            rc = fdc_run_ex(c, beam, n_histories, seed, &o, &out, nullptr);
            if (rc) break;
            double rms = 0, fms = 0;
            rc = fdc_last_kernel_ms(c, &rms, &fms);
            if (rc) break;
            if (i == 0 && rep == 0) continue;
            ms_min = std::min(ms_min, rms);
        }
        if (!rc && ms_min < best_ms) {
            best_ms = ms_min;
            best_s = cand[i];
        }
    }
    c->timing = timing_before;
    c->timed = false;
    if (rc) return rc;
    rc = fdc_sync(c, nullptr, nullptr);
    if (rc) return rc;
    c->tuned = best_s;
    c->tuned_variant = var;
    c->tuned_valid = true;
    if (best) *best = best_s;
    return FDC_OK;
}

int fdc_set_timing(fdc_ctx *c, int32_t enable) {
    if (!c) return FDC_ERR_INVALID;
    FDC_CUDA(c, cudaSetDevice(c->device));
    for (auto &e : c->ev)
        if (!e) FDC_CUDA(c, cudaEventCreate(&e));
    c->timing = enable != 0;
    c->timed = false;
    return FDC_OK;
}

int fdc_last_kernel_ms(fdc_ctx *c, double *replay_ms, double *finalize_ms) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->timed) return fail(c, FDC_ERR_INVALID, "no timed run (enable fdc_set_timing first)");
    FDC_CUDA(c, cudaEventSynchronize(c->ev[3]));
    float a = 0, b = 0;
    FDC_CUDA(c, cudaEventElapsedTime(&a, c->ev[0], c->ev[1]));
    FDC_CUDA(c, cudaEventElapsedTime(&b, c->ev[2], c->ev[3]));
    if (replay_ms) *replay_ms = a;
    if (finalize_ms) *finalize_ms = b;
    return FDC_OK;
}

int fdc_probe_atomics(uint64_t *slots, uint64_t n_slots, uint64_t n_ops, double *ms, void *stream) {
    if (!slots || !n_slots || !ms) return FDC_ERR_INVALID;
    int dev = 0, sms = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FDC_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FDC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FDC_ERR_CUDA;
    }
    int rc = FDC_OK;
    if (cudaMemsetAsync(slots, 0, sizeof(uint64_t) * n_slots, st) != cudaSuccess ||
        cudaEventRecord(e0, st) != cudaSuccess ||
        fdc::launch_probe_atomics((unsigned long long *)slots, n_slots, n_ops, sms, st) != cudaSuccess ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        rc = FDC_ERR_CUDA;
    float t = 0;
    if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = FDC_ERR_CUDA;
    *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int fdc_run_noalloc(fdc_ctx *c, const fdc_beam *beam, uint64_t n_histories, uint64_t seed, double *dose_out,
                    fdc_counters *counters_dev, void *stream) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->db_loaded || !c->ph_loaded) return fail(c, FDC_ERR_NOT_LOADED, "database and phantom must be loaded");
    if (!dose_out) return fail(c, FDC_ERR_INVALID, "dose_out is null");
    BeamInfo bi;
    int rc = check_beam(c, beam, &bi);
    if (rc) return rc;
    if (c->nvox > FDC_NOALLOC_MAX_VOXELS)
        return fail(c, FDC_ERR_INVALID, "run_noalloc: %lld voxels exceed the static scratch limit of %d",
                    c->nvox, FDC_NOALLOC_MAX_VOXELS);
    if (beam->n_spots > FDC_NOALLOC_MAX_SPOTS)
        return fail(c, FDC_ERR_INVALID, "run_noalloc: %d spots exceed the static scratch limit of %d",
                    beam->n_spots, FDC_NOALLOC_MAX_SPOTS);
    const unsigned long long n = n_histories ? n_histories : bi.total;
    if (n > bi.total) return fail(c, FDC_ERR_INVALID, "more histories than the beam holds");
    if (c->max_track_units > 0 && (double)n * (double)c->max_track_units > 9.0e18)
        return fail(c, FDC_ERR_OVERFLOW, "too many histories per launch for the int64 tally");
    fdc_run_opts o0;
    std::memset(&o0, 0, sizeof o0);
    fdc_schedule sched;
    rc = resolve_schedule(c, nullptr, run_variant(c, o0, false), &sched);
    if (rc) return rc;
    FDC_CUDA(c, cudaSetDevice(c->device));
    fdc::NoallocScratch sc;
    FDC_CUDA(c, fdc::noalloc_scratch(c->device, &sc));
    cudaStream_t st = (cudaStream_t)stream;
    // inputs into the scratch; zero what accumulates
    FDC_CUDA(c, cudaMemcpyAsync(sc.spots, beam->spots, sizeof(fdc_spot) * beam->n_spots, cudaMemcpyHostToDevice, st));
    FDC_CUDA(c, fdc::launch_spot_prefix(sc.spots, beam->n_spots, sc.spot_cum, st));
    FDC_CUDA(c, cudaMemsetAsync(sc.tally, 0, sizeof(unsigned long long) * c->nvox, st));
    FDC_CUDA(c, cudaMemsetAsync(sc.counters, 0, sizeof(DeviceCounters), st));
    FDC_CUDA(c, cudaMemsetAsync(sc.work, 0, sizeof(unsigned long long), st));
    fdc::ReplayArgs a = base_args(c);
    a.spots = sc.spots;
    a.spot_cum = sc.spot_cum;
    a.n_spots = beam->n_spots;
    a.tally = sc.tally;
    a.per_layer = 0;
    a.seed = seed;
    a.track_group = 1;
    a.rotate = 1;
    a.scaling_mode = 0;
    a.chunk = sched.chunk;
    a.h_begin = 0;
    a.n = n;
    a.work = sc.work;
    a.counters = sc.counters;
    if (n) FDC_CUDA(c, fdc::launch_replay(a, sched, 0, c->sm_count, st));
    fdc::FinalizeArgs f;
    std::memset(&f, 0, sizeof f);
    f.tally = (long long *)sc.tally;
    f.n_tallies = 1;
    f.nvox = c->nvox;
    f.density = c->density.p;
    f.factor = c->dfac.p;
    f.scale = fdc::kMeVToJ / (fdc::kTallyUnitsPerMeV * c->dx * c->dy * c->dz * 1e-3);
    f.dose = dose_out;
    FDC_CUDA(c, fdc::launch_finalize(f, c->sm_count, st));
    if (counters_dev)
        FDC_CUDA(c, cudaMemcpyAsync(counters_dev, sc.counters, sizeof(DeviceCounters), cudaMemcpyDeviceToDevice, st));
    return FDC_OK;
}

int fdc_debug_philox(uint64_t key0, uint64_t key1, const uint64_t *ctr, uint64_t n, uint64_t *out, void *stream) {
    if (!ctr || !out) return FDC_ERR_INVALID;
    if (!n) return FDC_OK;
    return fdc::launch_debug_philox(key0, key1, (const unsigned long long *)ctr, n, (unsigned long long *)out,
                                    (cudaStream_t)stream) == cudaSuccess
               ? FDC_OK
               : FDC_ERR_CUDA;
}

int fdc_debug_sample(fdc_ctx *c, const fdc_beam *beam, uint64_t seed, uint64_t h_begin, uint64_t n,
                     int32_t track_group, int32_t no_rotation, float *xyEpsi, int64_t *btk, void *stream) {
    if (!c) return FDC_ERR_INVALID;
    if (!c->db_loaded) return fail(c, FDC_ERR_NOT_LOADED, "database must be loaded");
    if (!xyEpsi || !btk || track_group < 0) return fail(c, FDC_ERR_INVALID, "debug_sample: bad arguments");
    BeamInfo bi;
    int rc = check_beam(c, beam, &bi);
    if (rc) return rc;
    if (h_begin > bi.total || n > bi.total - h_begin) return fail(c, FDC_ERR_INVALID, "history range beyond the beam");
    if (!n) return FDC_OK;
    FDC_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    rc = upload_beam(c, beam, st, false);
    if (rc) return rc;
    fdc::ReplayArgs a = base_args(c);
    a.n_spots = beam->n_spots;
    a.seed = seed;
    a.h_begin = h_begin;
    a.n = n;
    a.track_group = track_group > 1 ? track_group : 1;
    a.rotate = no_rotation ? 0 : 1;
    FDC_CUDA(c, fdc::launch_debug_sample(a, xyEpsi, (long long *)btk, st));
    return FDC_OK;
}

}  // extern "C"
