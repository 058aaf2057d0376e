/*
 * halobox.c - seeded, index-addressable synthetic N-body snapshot.
 *
 * Stand-in for the Millennium snapshots of Ivkin et al. (arXiv:1711.00975,
 * Sec. 4.1), which are not available here.  A box of side L holds a mixture
 * of Plummer-profile halos (a fraction `halo_frac` of the particles) and a
 * uniform background.  Halo masses follow a power law dN/dM ~ M^-slope on
 * [m_min, m_max]; particle counts are proportional to the drawn masses
 * (largest-remainder rounding so they sum exactly to round(halo_frac*N));
 * the Plummer scale radius is r_scale*(M/m_pivot)^(1/3), truncated at
 * trunc*a.  Positions wrap periodically into [0, L).
 *
 * Stream order: stream position i holds generation index j = P(i), where P is
 * a seeded bijection of [0, N) (a cycle-walking balanced Feistel network), so
 * the stream is "not sorted in any way" (Sec. 2.1) yet any slice [i0, i1) can
 * be produced independently - chunks of an out-of-core stream are generated
 * on demand.
 *
 * This file produces INPUTS only.  It contains none of the sketch method's
 * arithmetic (no quantisation, no sampling hash, no sketch hash); its random
 * numbers come from a murmur3-style 64-bit finaliser, a different generator
 * from the splitmix64 the method uses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HB_STREAM_MASS 1ULL
#define HB_STREAM_CENTRE 2ULL
#define HB_STREAM_PART 3ULL
#define HB_STREAM_BG 4ULL
#define HB_STREAM_PERM 5ULL

typedef struct {
    uint64_t n;        /* total particles                              */
    double box;        /* side length L                                */
    uint64_t n_halo;   /* number of halos                              */
    double halo_frac;  /* fraction of particles in halos               */
    double m_min, m_max, slope;   /* power law dN/dM ~ M^-slope       */
    double r_scale;    /* a = r_scale * (M / m_pivot)^(1/3)            */
    double m_pivot;
    double trunc;      /* profile truncated at trunc * a               */
    uint64_t seed;
    int32_t permute;   /* 1: seeded permutation of the stream order    */
    int32_t pad;
} hb_config;

typedef struct {
    hb_config cfg;
    uint64_t n_in_halos;  /* sum of counts                              */
    double *centre;       /* 3 * n_halo                                 */
    double *mass;         /* n_halo                                     */
    double *a;            /* scale radius, n_halo                       */
    uint64_t *count;      /* particles per halo                         */
    uint64_t *offset;     /* n_halo + 1 prefix sums                     */
    uint64_t *jtab;       /* halo index at j = q * jstep, narrows search */
    uint64_t jstep;
    uint64_t jtab_len;
    uint32_t half_bits;   /* Feistel half width                         */
    uint64_t round_key[4];
} hb_box;

static inline uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

static inline uint64_t hb_rand(uint64_t seed, uint64_t stream, uint64_t ctr) {
    uint64_t s = fmix64(seed ^ (stream * 0xD1B54A32D192ED03ULL) ^ 0x5851F42D4C957F2DULL);
    return fmix64(s ^ (ctr * 0x8CB92BA72F3D8DD7ULL + 0x632BE59BD9B4E019ULL));
}

/* uniform double strictly inside (0, 1) */
static inline double hb_u01(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1p-53; }

typedef struct { double frac; uint64_t idx; } frac_idx;

static int cmp_frac(const void *pa, const void *pb) {
    const frac_idx *a = (const frac_idx *)pa, *b = (const frac_idx *)pb;
    if (a->frac > b->frac) return -1;
    if (a->frac < b->frac) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

void hb_free(hb_box *b) {
    if (!b) return;
    free(b->centre); free(b->mass); free(b->a); free(b->count); free(b->offset); free(b->jtab);
    free(b);
}

/* Build the halo catalogue.  Returns 0 on success. */
int hb_build(const hb_config *cfg, hb_box **out) {
    *out = NULL;
    if (cfg->n == 0 || !(cfg->box > 0) || cfg->halo_frac < 0 || cfg->halo_frac > 1) return 1;
    hb_box *b = (hb_box *)calloc(1, sizeof(hb_box));
    if (!b) return 2;
    b->cfg = *cfg;
    uint64_t H = cfg->n_halo;
    uint64_t n_h_total = (uint64_t)llround(cfg->halo_frac * (double)cfg->n);
    if (H == 0) n_h_total = 0;
    if (n_h_total > cfg->n) n_h_total = cfg->n;
    b->centre = (double *)malloc(sizeof(double) * 3 * (H ? H : 1));
    b->mass = (double *)malloc(sizeof(double) * (H ? H : 1));
    b->a = (double *)malloc(sizeof(double) * (H ? H : 1));
    b->count = (uint64_t *)calloc(H ? H : 1, sizeof(uint64_t));
    b->offset = (uint64_t *)calloc(H + 1, sizeof(uint64_t));
    if (!b->centre || !b->mass || !b->a || !b->count || !b->offset) { hb_free(b); return 2; }

    double e = 1.0 - cfg->slope;   /* inverse CDF of the power law */
    double lo = pow(cfg->m_min, e), hi = pow(cfg->m_max, e);
    double msum = 0.0;
    for (uint64_t h = 0; h < H; ++h) {
        double u = hb_u01(hb_rand(cfg->seed, HB_STREAM_MASS, h));
        double m = (fabs(e) < 1e-12) ? cfg->m_min * pow(cfg->m_max / cfg->m_min, u)
                                     : pow(lo + u * (hi - lo), 1.0 / e);
        b->mass[h] = m;
        msum += m;
        for (int d = 0; d < 3; ++d)
            b->centre[3 * h + d] = cfg->box * hb_u01(hb_rand(cfg->seed, HB_STREAM_CENTRE, 3 * h + d));
        b->a[h] = cfg->r_scale * cbrt(m / cfg->m_pivot);
    }
    /* largest-remainder apportionment of n_h_total by mass */
    if (H > 0 && n_h_total > 0) {
        frac_idx *fr = (frac_idx *)malloc(sizeof(frac_idx) * H);
        if (!fr) { hb_free(b); return 2; }
        uint64_t assigned = 0;
        for (uint64_t h = 0; h < H; ++h) {
            double q = (double)n_h_total * b->mass[h] / msum;
            double f = floor(q);
            b->count[h] = (uint64_t)f;
            assigned += (uint64_t)f;
            fr[h].frac = q - f;
            fr[h].idx = h;
        }
        uint64_t rem = n_h_total > assigned ? n_h_total - assigned : 0;
        if (rem > 0) {
            qsort(fr, H, sizeof(frac_idx), cmp_frac);
            for (uint64_t r = 0; r < rem && r < H; ++r) b->count[fr[r].idx] += 1;
        }
        free(fr);
    }
    uint64_t acc = 0;
    for (uint64_t h = 0; h < H; ++h) { b->offset[h] = acc; acc += b->count[h]; }
    b->offset[H] = acc;
    b->n_in_halos = acc;
    /* coarse table of halo indices so the per-particle search is short */
    b->jstep = acc / (1ULL << 20) + 1;
    b->jtab_len = acc / b->jstep + 2;
    b->jtab = (uint64_t *)malloc(sizeof(uint64_t) * b->jtab_len);
    if (!b->jtab) { hb_free(b); return 2; }
    {
        uint64_t h = 0;
        for (uint64_t q = 0; q < b->jtab_len; ++q) {
            uint64_t j = q * b->jstep;
            while (h + 1 < H && b->offset[h + 1] <= j) ++h;
            b->jtab[q] = h;
        }
    }

    uint32_t bits = 1;
    while (bits < 64 && (1ULL << bits) < cfg->n) ++bits;
    if (bits & 1) ++bits;
    b->half_bits = bits / 2;
    for (int r = 0; r < 4; ++r) b->round_key[r] = hb_rand(cfg->seed, HB_STREAM_PERM, (uint64_t)r);
    *out = b;
    return 0;
}

/* one pass of the 4-round balanced Feistel network on [0, 4^half_bits) */
static inline uint64_t feistel(const hb_box *b, uint64_t x) {
    uint32_t hb = b->half_bits;
    uint64_t mask = (hb >= 64) ? ~0ULL : ((1ULL << hb) - 1);
    uint64_t L = (x >> hb) & mask, R = x & mask;
    for (int r = 0; r < 4; ++r) {
        uint64_t F = fmix64(R ^ b->round_key[r]) & mask;
        uint64_t nL = R;
        R = L ^ F;
        L = nL;
    }
    return (L << hb) | R;
}

/* generation index held at stream position i */
uint64_t hb_stream_index(const hb_box *b, uint64_t i) {
    if (!b->cfg.permute) return i;
    uint64_t j = feistel(b, i);
    while (j >= b->cfg.n) j = feistel(b, j);   /* cycle walking */
    return j;
}

static inline float wrap_to_float(double v, double L) {
    v = fmod(v, L);
    if (v < 0) v += L;
    float f = (float)v;
    if (f >= (float)L) f = 0.0f;   /* rounding up to L wraps to 0 */
    if (f < 0.0f) f = 0.0f;
    return f;
}

static inline void gen_one(const hb_box *b, uint64_t j, float *out) {
    const hb_config *c = &b->cfg;
    if (j < b->n_in_halos) {
        /* halo h with offset[h] <= j < offset[h+1] */
        uint64_t q = j / b->jstep;
        uint64_t lo = b->jtab[q];
        uint64_t hi = (q + 1 < b->jtab_len) ? b->jtab[q + 1] + 1 : c->n_halo;
        if (hi > c->n_halo) hi = c->n_halo;
        while (hi - lo > 1) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (b->offset[mid] <= j) lo = mid; else hi = mid;
        }
        uint64_t h = lo;
        double a = b->a[h];
        double T = c->trunc;
        double mt = pow(T * T / (T * T + 1.0), 1.5);   /* enclosed mass fraction at T*a */
        double u1 = hb_u01(hb_rand(c->seed, HB_STREAM_PART, 3 * j)) * mt;
        double u2 = hb_u01(hb_rand(c->seed, HB_STREAM_PART, 3 * j + 1));
        double u3 = hb_u01(hb_rand(c->seed, HB_STREAM_PART, 3 * j + 2));
        double r = a / sqrt(pow(u1, -2.0 / 3.0) - 1.0);
        double ct = 2.0 * u2 - 1.0;
        double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double ph = 2.0 * M_PI * u3;
        out[0] = wrap_to_float(b->centre[3 * h + 0] + r * st * cos(ph), c->box);
        out[1] = wrap_to_float(b->centre[3 * h + 1] + r * st * sin(ph), c->box);
        out[2] = wrap_to_float(b->centre[3 * h + 2] + r * ct, c->box);
    } else {
        for (int d = 0; d < 3; ++d)
            out[d] = wrap_to_float(c->box * hb_u01(hb_rand(c->seed, HB_STREAM_BG, 3 * j + d)), c->box);
    }
}

/* Positions of stream positions [i0, i0+count) as float32 xyz, AoS. */
int hb_generate(const hb_box *b, uint64_t i0, uint64_t count, float *xyz, int nthreads) {
    if (i0 > b->cfg.n || count > b->cfg.n - i0) return 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static, 65536) num_threads(nthreads)
#endif
    for (int64_t q = 0; q < (int64_t)count; ++q) {
        uint64_t j = hb_stream_index(b, i0 + (uint64_t)q);
        gen_one(b, j, xyz + 3 * (uint64_t)q);
    }
    (void)nthreads;
    return 0;
}

uint64_t hb_n_in_halos(const hb_box *b) { return b->n_in_halos; }

/* Copy the catalogue out (any pointer may be NULL). */
void hb_catalogue(const hb_box *b, double *centre, double *mass, double *a, uint64_t *count) {
    uint64_t H = b->cfg.n_halo;
    if (centre) memcpy(centre, b->centre, sizeof(double) * 3 * H);
    if (mass) memcpy(mass, b->mass, sizeof(double) * H);
    if (a) memcpy(a, b->a, sizeof(double) * H);
    if (count) memcpy(count, b->count, sizeof(uint64_t) * H);
}
