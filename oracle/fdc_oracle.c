/*
 * fdc_oracle.c -- plain, sequential, FP64 CPU track repeater.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the
 * GPU dose engine.  It shares no code, header, table or helper with the CUDA
 * path, and only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it.  It is written for clarity, not speed: one history
 * at a time, in the order the method describes.
 *
 * What it computes (Yepes, Mirkovic & Taddei, "A GPU implementation of a
 * track-repeating algorithm for proton radiotherapy dose calculations"):
 *
 *   Sec. 2.2  A database holds pre-generated proton tracks in water, broken
 *             into steps; each step stores its length, energy loss and
 *             direction change.  A track is re-traced through a
 *             heterogeneous phantom by scaling each step length and each
 *             scattering angle with the material it crosses.
 *   Sec. 2.3  Per incident proton (phase-space entry): task 1 picks the
 *             database history and the step where re-tracing starts; task 2
 *             re-traces the history through the voxel phantom.  Deposited
 *             energy is tallied in a grid with the phantom's voxels, and
 *             converted to dose by dividing by the voxel mass at the end.
 *             One database history serves several incident protons at
 *             different entry positions.
 *   Sec. 2.4  Eq. (2) history-by-history uncertainty needs per-history sums
 *             of squares; those are produced here exactly (per history, not
 *             per deposit), and, as a second output, per voxel visit (the
 *             squares of what a history leaves in a voxel before moving on).
 *
 * Readings of what the paper leaves open (the engine follows the same ones):
 *   - per-step record: (dE, len, theta, phi, esec); theta/phi is the
 *     deflection applied at the END of the step, relative to the direction
 *     of the step, with azimuth measured in the frame defined below;
 *   - step scaling: the water step length is consumed voxel by voxel as
 *     water-equivalent length, geometric length g in voxel v consuming
 *     g * rho_v * s_rel[m_v]; the energy loss is spread over the segments in
 *     proportion to the water-equivalent length each one consumes (mode 0).
 *     Mode 1 (ablation) scales the whole step by the voxel where it starts;
 *   - angle scaling: theta_m = theta_w * sqrt(sum_i w_i k_theta[m_i]^2),
 *     w_i the water-equivalent fraction of the step in voxel i;
 *   - esec is deposited in the voxel where the step ends;
 *   - each reuse of a track is rotated rigidly about the beam axis by an
 *     angle psi drawn per proton;
 *   - start step: first step whose residual energy is <= the proton energy;
 *   - leaving the grid ends the history; the energy it still carried is
 *     counted as escaped.
 *
 * Random numbers: Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11,
 * "Parallel random numbers: as easy as 1, 2, 3"), key = (seed, 0),
 * counter = (history or group index, purpose, 0, 0).
 *
 * Pins (tests/test_oracle_pins.py): Philox against an independent
 * implementation; sampling moments; hand-computed tiny phantoms; the water
 * identity (depth dose equals the database's chords); 3-D brute force of
 * single histories; energy conservation; Bragg-Kleeman ranges in slabs;
 * sharding, per-layer partition and thread reentrancy.  The dose of a full
 * heterogeneous phantom has no pin beyond these special cases: parity
 * unpinned there (the paper prints no voxel values).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_NOMEM 4
#define OR_ERR_LOOP 5

/* ------------------------------------------------------------------ */
/* Inputs (layouts mirrored by the Python wrapper with ctypes).        */

typedef struct {
    int32_t n_energies;
    const float *energy;        /* [n_energies] MeV, increasing */
    const int64_t *track_begin; /* [n_energies+1] */
    const int64_t *step_begin;  /* [n_tracks+1] */
    const float *dE, *len, *theta, *phi, *esec;
} or_db;

typedef struct {
    int32_t nx, ny, nz, n_mat;
    double dx, dy, dz, x0, y0, z0;
    const uint8_t *material;    /* [nz][ny][nx] */
    const float *density;       /* [nz][ny][nx] g/cm^3 */
    const float *s_rel;         /* [n_mat] */
    const float *k_theta;       /* [n_mat] */
} or_phantom;

typedef struct {
    double x, y, energy, sigma_e, a, b;
    int32_t profile, layer;
    uint64_t n_histories;
} or_spot;

typedef struct {
    double *edep;      /* [n_layers_out][nvox] MeV, accumulated (caller zeroes) */
    double *hh_sumsq;  /* optional [nvox]: sum over histories of (history's energy in v)^2 */
    double replayed;   /* sum over histories of the energy of the replayed steps */
    double escaped;    /* part of it that left the grid */
    uint64_t n_histories, n_steps, n_segments;
    double *hv_sumsq;  /* optional [nvox]: sum over voxel visits of (visit's energy)^2, a visit
                          being a maximal run of one history's consecutive deposits into v */
} or_out;

/* ------------------------------------------------------------------ */
/* Philox4x64-10                                                        */

static void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * c[0];
        unsigned __int128 p1 = (unsigned __int128)M1 * c[2];
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c[1] ^ k0;
        uint64_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void fdco_philox4x64_10(const uint64_t *ctr, const uint64_t *key, uint64_t *out, int64_t n)
{
    /* n independent blocks: ctr is [n][4], key [2], out [n][4] */
    for (int64_t i = 0; i < n; ++i) philox4x64_10(ctr + 4 * i, key, out + 4 * i);
}

/* uniform on (0,1): 53 high bits, centred in their cell (never 0 or 1) */
static double u01(uint64_t r) { return ((double)(r >> 11) + 0.5) * 0x1p-53; }

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------ */
/* Task 1: phase-space entry, database history and start step (Sec. 2.3) */

typedef struct {
    int spot, layer;
    float x, y, E, psi;   /* the per-proton state is single precision */
    int bin;
    int64_t track;
    int64_t k0;           /* first step to replay (== n_steps: nothing) */
    int64_t n;            /* steps in the track */
} or_start;

static int find_spot(const or_spot *spots, int n_spots, uint64_t h)
{
    /* the global history index runs over the spots in order */
    uint64_t acc = 0;
    for (int s = 0; s < n_spots; ++s) {
        acc += spots[s].n_histories;
        if (h < acc) return s;
    }
    return -1;
}

static void sample_history(const or_db *db, const or_spot *spots, int n_spots, uint64_t seed,
                           uint64_t h, int track_group, int rotate, or_start *st)
{
    const uint64_t key[2] = {seed, 0};
    uint64_t ca[4] = {h, 1, 0, 0}, cb[4] = {h, 2, 0, 0};
    uint64_t cc[4] = {h / (uint64_t)track_group, 3, 0, 0};
    uint64_t A[4], B[4], C[4];
    philox4x64_10(ca, key, A);
    philox4x64_10(cb, key, B);
    philox4x64_10(cc, key, C);

    int s = find_spot(spots, n_spots, h);
    const or_spot *sp = &spots[s];
    st->spot = s;
    st->layer = sp->layer;

    /* transverse entry position */
    double x, y;
    if (sp->profile == 0) {            /* Gaussian, sigma = a (Box-Muller) */
        double r = sqrt(-2.0 * log(u01(A[0])));
        double ang = TWO_PI * u01(A[1]);
        x = sp->x + sp->a * (r * cos(ang));
        y = sp->y + sp->a * (r * sin(ang));
    } else if (sp->profile == 1) {     /* rectangle a x b */
        x = sp->x + sp->a * (u01(A[0]) - 0.5);
        y = sp->y + sp->b * (u01(A[1]) - 0.5);
    } else {                            /* disk of radius a */
        double r = sp->a * sqrt(u01(A[0]));
        double ang = TWO_PI * u01(A[1]);
        x = sp->x + r * cos(ang);
        y = sp->y + r * sin(ang);
    }
    /* energy */
    double E = sp->energy;
    if (sp->sigma_e > 0.0) {
        double r = sqrt(-2.0 * log(u01(A[2])));
        double n0 = r * cos(TWO_PI * u01(A[3]));
        E = sp->energy + sp->sigma_e * n0;
    }
    double psi = rotate ? TWO_PI * u01(B[0]) : 0.0;
    st->x = (float)x;
    st->y = (float)y;
    st->E = (float)E;
    st->psi = (float)psi;

    /* database history: nearest bin energy >= E (top bin if none) */
    int b = db->n_energies - 1;
    for (int i = 0; i < db->n_energies; ++i)
        if (db->energy[i] >= st->E) { b = i; break; }
    st->bin = b;
    uint64_t nb = (uint64_t)(db->track_begin[b + 1] - db->track_begin[b]);
    uint64_t j = (uint64_t)(((unsigned __int128)C[0] * nb) >> 64);
    st->track = db->track_begin[b] + (int64_t)j;

    /* start step: first k with residual energy E_res,k <= E, where
       E_res,k = E_bin - sum_{i<k} (dE_i + esec_i), summed in FP64 in step
       order and rounded to single precision (the precision of E). */
    int64_t s0 = db->step_begin[st->track], n = db->step_begin[st->track + 1] - s0;
    st->n = n;
    st->k0 = n;
    if (st->E > 0.0f) {
        double used = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            float eres = (float)((double)db->energy[b] - used);
            if (eres <= st->E) { st->k0 = k; break; }
            used += (double)db->dE[s0 + k] + (double)db->esec[s0 + k];
        }
    }
}

int fdco_sample(const or_db *db, const or_spot *spots, int32_t n_spots, uint64_t seed,
                uint64_t h_begin, uint64_t n, int32_t track_group, int32_t rotate,
                float *xyEpsi /* [n][4] */, int64_t *bin_track_k0 /* [n][3] */)
{
    for (uint64_t i = 0; i < n; ++i) {
        or_start st;
        sample_history(db, spots, n_spots, seed, h_begin + i, track_group, rotate, &st);
        xyEpsi[4 * i + 0] = st.x;
        xyEpsi[4 * i + 1] = st.y;
        xyEpsi[4 * i + 2] = st.E;
        xyEpsi[4 * i + 3] = st.psi;
        bin_track_k0[3 * i + 0] = st.bin;
        bin_track_k0[3 * i + 1] = st.track;
        bin_track_k0[3 * i + 2] = st.k0;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Per-history scratch for exact eq. (2) sums: a small hash map from     */
/* voxel index to the energy the current history left there.           */

typedef struct {
    int64_t *keys;
    double *vals;
    int64_t *used;
    int64_t n_used, cap;
} hmap;

static int hmap_init(hmap *m, int64_t cap)
{
    m->cap = cap;
    m->n_used = 0;
    m->keys = (int64_t *)malloc(sizeof(int64_t) * cap);
    m->vals = (double *)calloc(cap, sizeof(double));
    m->used = (int64_t *)malloc(sizeof(int64_t) * cap);
    if (!m->keys || !m->vals || !m->used) return -1;
    for (int64_t i = 0; i < cap; ++i) m->keys[i] = -1;
    return 0;
}

static void hmap_free(hmap *m) { free(m->keys); free(m->vals); free(m->used); }

static int hmap_add(hmap *m, int64_t key, double v)
{
    int64_t i = (int64_t)(((uint64_t)key * 0x9E3779B97F4A7C15ULL) % (uint64_t)m->cap);
    for (int64_t probe = 0; probe < m->cap; ++probe) {
        if (m->keys[i] == key) { m->vals[i] += v; return 0; }
        if (m->keys[i] < 0) {
            if (2 * (m->n_used + 1) > m->cap) return -1;
            m->keys[i] = key;
            m->vals[i] = v;
            m->used[m->n_used++] = i;
            return 0;
        }
        i = (i + 1) % m->cap;
    }
    return -1;
}

static void hmap_flush(hmap *m, double *sumsq)
{
    for (int64_t u = 0; u < m->n_used; ++u) {
        int64_t i = m->used[u];
        sumsq[m->keys[i]] += m->vals[i] * m->vals[i];
        m->keys[i] = -1;
        m->vals[i] = 0.0;
    }
    m->n_used = 0;
}

/* ------------------------------------------------------------------ */
/* Per-visit squares (the reading of Sec. 2.3's second tally that squares */
/* what one history leaves in a voxel before it moves on): the energy of  */
/* the current visit is accumulated while deposits go to the same voxel   */
/* and squared when the next deposit goes elsewhere or the history ends.  */

typedef struct {
    int64_t v;      /* voxel of the current visit, -1 for none */
    double e;       /* its energy so far */
    double *sumsq;  /* [nvox] */
} or_visit;

static void visit_add(or_visit *vs, int64_t v, double e)
{
    if (!vs) return;
    if (v != vs->v) {
        if (vs->v >= 0) vs->sumsq[vs->v] += vs->e * vs->e;
        vs->v = v;
        vs->e = 0.0;
    }
    vs->e += e;
}

static void visit_end(or_visit *vs)
{
    if (!vs) return;
    if (vs->v >= 0) vs->sumsq[vs->v] += vs->e * vs->e;
    vs->v = -1;
    vs->e = 0.0;
}

/* ------------------------------------------------------------------ */
/* Direction change: rotate unit vector d by polar angle theta at azimuth */
/* phi.  Frame attached to d = (dx,dy,dz) with p = sqrt(dx^2+dy^2) > 0:  */
/*   e2 = (z x d)/p = (-dy, dx, 0)/p,  e1 = e2 x d = (dx dz, dy dz, -p^2)/p */
/* For d exactly along +z the frame is (x, y) rotated by psi, which makes */
/* every reuse of a track a rigid rotation of it about the beam axis; for */
/* d along -z it is (x, -y) rotated the same way.                          */

static void deflect(double d[3], double theta, double phi, double psi)
{
    double st = sin(theta), ct = cos(theta);
    double p = sqrt(d[0] * d[0] + d[1] * d[1]);
    double n[3];
    if (p > 0.0) {
        double cp = cos(phi), sp = sin(phi);
        double a = st * cp, b = st * sp;
        double e1[3] = {d[0] * d[2] / p, d[1] * d[2] / p, -p};
        double e2[3] = {-d[1] / p, d[0] / p, 0.0};
        for (int i = 0; i < 3; ++i) n[i] = a * e1[i] + b * e2[i] + ct * d[i];
    } else if (d[2] > 0.0) {
        double az = phi + psi;
        n[0] = st * cos(az);
        n[1] = st * sin(az);
        n[2] = ct;
    } else {
        double az = phi - psi;
        n[0] = st * cos(az);
        n[1] = -st * sin(az);
        n[2] = -ct;
    }
    d[0] = n[0]; d[1] = n[1]; d[2] = n[2];
}

/* ------------------------------------------------------------------ */
/* Task 2: re-trace one history (Sec. 2.2, 2.3).                        */

static int replay(const or_db *db, const or_phantom *ph, const or_start *st, int scaling_mode,
                  double *edep_layer, hmap *hm, or_visit *vs, or_out *out)
{
    const int64_t s0 = db->step_begin[st->track];
    const int nx = ph->nx, ny = ph->ny, nz = ph->nz;
    const double h[3] = {ph->dx, ph->dy, ph->dz};
    const double o[3] = {ph->x0, ph->y0, ph->z0};
    const int nn[3] = {nx, ny, nz};

    double replayed = 0.0;
    for (int64_t k = st->k0; k < st->n; ++k)
        replayed += (double)db->dE[s0 + k] + (double)db->esec[s0 + k];
    out->replayed += replayed;
    if (st->k0 >= st->n) return OR_OK;

    double p[3] = {(double)st->x, (double)st->y, o[2]};
    double d[3] = {0.0, 0.0, 1.0};
    int iv[3];
    /* entry: the proton starts on the upstream face z = z0 */
    if (!(p[0] >= o[0] && p[0] < o[0] + nx * h[0] && p[1] >= o[1] && p[1] < o[1] + ny * h[1])) {
        out->escaped += replayed;
        return OR_OK;
    }
    iv[0] = (int)floor((p[0] - o[0]) / h[0]);
    iv[1] = (int)floor((p[1] - o[1]) / h[1]);
    iv[2] = 0;
    if (iv[0] > nx - 1) iv[0] = nx - 1;
    if (iv[1] > ny - 1) iv[1] = ny - 1;

    const double psi = (double)st->psi;
    const int64_t seg_cap = (int64_t)nx + ny + nz + 8;

    for (int64_t k = st->k0; k < st->n; ++k) {
        const double dE = db->dE[s0 + k], len = db->len[s0 + k];
        const double esec = db->esec[s0 + k];
        out->n_steps++;

        /* parametric distances to the next face on each axis */
        double tmax[3], tdelta[3];
        int dir[3];
        for (int a = 0; a < 3; ++a) {
            if (d[a] > 0.0) {
                dir[a] = 1;
                tmax[a] = (o[a] + (iv[a] + 1) * h[a] - p[a]) / d[a];
                tdelta[a] = h[a] / d[a];
            } else if (d[a] < 0.0) {
                dir[a] = -1;
                tmax[a] = (o[a] + iv[a] * h[a] - p[a]) / d[a];
                tdelta[a] = -h[a] / d[a];
            } else {
                dir[a] = 0;
                tmax[a] = INFINITY;
                tdelta[a] = INFINITY;
            }
            if (tmax[a] < 0.0) tmax[a] = 0.0;
        }

        /* step scaling: water-equivalent length still to consume */
        double rem = len;
        double t = 0.0;       /* geometric distance along d in this step */
        double acc_k2 = 0.0;  /* sum of wet_i * k_theta_i^2 */
        int64_t v = iv[0] + (int64_t)nx * (iv[1] + (int64_t)ny * iv[2]);
        double S_fixed = 0.0, k2_fixed = 0.0;
        if (scaling_mode == 1) {
            int m = ph->material[v];
            S_fixed = (double)ph->density[v] * (double)ph->s_rel[m];
            k2_fixed = (double)ph->k_theta[m] * (double)ph->k_theta[m];
        }
        int64_t nseg = 0;
        for (;;) {
            if (++nseg > seg_cap) return OR_ERR_LOOP;
            out->n_segments++;
            v = iv[0] + (int64_t)nx * (iv[1] + (int64_t)ny * iv[2]);
            int m = ph->material[v];
            double S = scaling_mode == 1 ? S_fixed : (double)ph->density[v] * (double)ph->s_rel[m];
            double k2 = scaling_mode == 1 ? k2_fixed : (double)ph->k_theta[m] * (double)ph->k_theta[m];
            int a = 0;                          /* nearest face; ties: x, then y, then z */
            if (tmax[1] < tmax[a]) a = 1;
            if (tmax[2] < tmax[a]) a = 2;
            double seg = tmax[a] - t;
            if (seg < 0.0) seg = 0.0;
            if (seg * S >= rem) {               /* the step ends inside voxel v */
                double e = dE * rem / len;
                edep_layer[v] += e;
                if (hm && e != 0.0 && hmap_add(hm, v, e)) return OR_ERR_NOMEM;
                visit_add(vs, v, e);
                acc_k2 += rem * k2;
                t += rem / S;
                rem = 0.0;
                break;
            }
            double wet = seg * S;
            double e = dE * wet / len;
            edep_layer[v] += e;
            if (hm && e != 0.0 && hmap_add(hm, v, e)) return OR_ERR_NOMEM;
            visit_add(vs, v, e);
            acc_k2 += wet * k2;
            rem -= wet;
            t = tmax[a];
            iv[a] += dir[a];
            if (iv[a] < 0 || iv[a] >= nn[a]) {  /* left the grid */
                double esc = dE * rem / len + esec;
                for (int64_t j = k + 1; j < st->n; ++j)
                    esc += (double)db->dE[s0 + j] + (double)db->esec[s0 + j];
                out->escaped += esc;
                return OR_OK;
            }
            tmax[a] += tdelta[a];
        }
        for (int i = 0; i < 3; ++i) p[i] += t * d[i];
        if (esec != 0.0) {
            edep_layer[v] += esec;
            if (hm && hmap_add(hm, v, esec)) return OR_ERR_NOMEM;
            visit_add(vs, v, esec);
        }
        /* angle scaling and direction change at the end of the step */
        double theta_m = (double)db->theta[s0 + k] * sqrt(acc_k2 / len);
        deflect(d, theta_m, (double)db->phi[s0 + k], psi);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */

static int check_inputs(const or_db *db, const or_phantom *ph, const or_spot *spots, int n_spots)
{
    if (!db || !ph || !spots || n_spots <= 0 || db->n_energies <= 0) return OR_ERR_INVALID;
    if (ph->nx <= 0 || ph->ny <= 0 || ph->nz <= 0 || ph->n_mat <= 0) return OR_ERR_INVALID;
    if (!(ph->dx > 0 && ph->dy > 0 && ph->dz > 0)) return OR_ERR_INVALID;
    for (int b = 0; b < db->n_energies; ++b)
        if (db->track_begin[b + 1] <= db->track_begin[b]) return OR_ERR_INVALID;
    int64_t n_tracks = db->track_begin[db->n_energies];
    for (int64_t t = 0; t < n_tracks; ++t) {
        for (int64_t s = db->step_begin[t]; s < db->step_begin[t + 1]; ++s)
            if (!(db->len[s] > 0.0f)) return OR_ERR_INVALID;
    }
    int64_t nvox = (int64_t)ph->nx * ph->ny * ph->nz;
    for (int64_t v = 0; v < nvox; ++v)
        if (ph->material[v] >= ph->n_mat) return OR_ERR_INVALID;
    for (int s = 0; s < n_spots; ++s)
        if (spots[s].profile < 0 || spots[s].profile > 2 || spots[s].layer < 0) return OR_ERR_INVALID;
    return OR_OK;
}

/* Replays histories [h_begin, h_end) of the beam and accumulates into out.
   per_layer != 0: out->edep is [n_layers][nvox] indexed by the spot's layer;
   otherwise [nvox].  rotate == 0 replays every track unrotated (psi = 0). */
typedef struct {
    uint64_t seed, h_begin, h_end;
    int32_t track_group, scaling_mode, per_layer, rotate;
} or_opts;

int fdco_run(const or_db *db, const or_phantom *ph, const or_spot *spots, int32_t n_spots,
             const or_opts *opt, or_out *out)
{
    const uint64_t seed = opt->seed, h_begin = opt->h_begin, h_end = opt->h_end;
    const int32_t track_group = opt->track_group, scaling_mode = opt->scaling_mode;
    const int32_t per_layer = opt->per_layer, rotate = opt->rotate;
    int rc = check_inputs(db, ph, spots, n_spots);
    if (rc) return rc;
    if (track_group < 1 || scaling_mode < 0 || scaling_mode > 1) return OR_ERR_INVALID;
    uint64_t total = 0;
    for (int s = 0; s < n_spots; ++s) total += spots[s].n_histories;
    if (h_end > total || h_begin > h_end) return OR_ERR_INVALID;
    const int64_t nvox = (int64_t)ph->nx * ph->ny * ph->nz;
    hmap hm;
    int use_hm = out->hh_sumsq != NULL;
    or_visit visit = {-1, 0.0, out->hv_sumsq};
    or_visit *vs = out->hv_sumsq ? &visit : NULL;
    if (use_hm && hmap_init(&hm, 1 << 16)) return OR_ERR_NOMEM;
    rc = OR_OK;
    for (uint64_t hh = h_begin; hh < h_end; ++hh) {
        or_start st;
        sample_history(db, spots, n_spots, seed, hh, track_group, rotate, &st);
        double *edep = out->edep + (per_layer ? (int64_t)st.layer * nvox : 0);
        rc = replay(db, ph, &st, scaling_mode, edep, use_hm ? &hm : NULL, vs, out);
        if (rc) break;
        if (use_hm) hmap_flush(&hm, out->hh_sumsq);
        visit_end(vs);
        out->n_histories++;
    }
    if (use_hm) hmap_free(&hm);
    return rc;
}

/* Sec. 2.3: energy (MeV) to absorbed dose (Gy) by dividing by voxel mass. */
void fdco_dose(const or_phantom *ph, const double *edep, double *dose)
{
    const double MEV_TO_J = 1.602176634e-13;
    const double vol_cm3 = ph->dx * ph->dy * ph->dz;
    const int64_t nvox = (int64_t)ph->nx * ph->ny * ph->nz;
    for (int64_t v = 0; v < nvox; ++v) {
        double mass_kg = (double)ph->density[v] * vol_cm3 * 1e-3;
        dose[v] = mass_kg > 0.0 ? edep[v] * MEV_TO_J / mass_kg : 0.0;
    }
}
