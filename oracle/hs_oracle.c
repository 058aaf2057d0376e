/*
 * hs_oracle.c - TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU restatement of the one-pass Count
 * Sketch path of Ivkin et al., "Scalable Streaming Tools for Analyzing N-body
 * Simulations" (arXiv:1711.00975).  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg use it; the CUDA library never links,
 * includes or calls anything here, and nothing here comes from the CUDA
 * library.  Build with -ffp-contract=off so the float32 multiply of the cell
 * quantisation is a single IEEE-754 rounding, as on the device.
 *
 * What it computes, in the paper's order:
 *   - mesh reduction (Sec. 2.1): particle -> regular-mesh cell ID;
 *   - Bernoulli sampling of particles by a hash of the particle index
 *     (Sec. 3.1, the sampling paragraph);
 *   - Count Sketch Add (Sec. 2.2): for every row i, M[i, h_{i,b}(s)] += h_{i,s}(s);
 *   - Estimate (Sec. 2.2): median over rows of M[i, h_{i,b}(j)] * h_{i,s}(j);
 *   - Count Sketch with Full Search (Algorithm 1): estimate every cell of the
 *     dictionary and keep the k largest;
 *   - the exact algorithm of Sec. 4.2 (one counter per occupied cell, k
 *     heaviest), the ground truth of recall.
 *
 * Readings taken where the paper is silent, ambiguous or garbled:
 *   - hash family: vector multiply-shift over the three cell coordinates,
 *     v = (a0*cx + a1*cy + a2*cz + b) mod 2^64, bucket = top log2W bits of v,
 *     sign bit = the next bit (1 -> -1) (strongly universal, Thorup 2015,
 *     "High Speed Hashing for Integers and Strings", vector multiply-shift);
 *   - seeds: successive splitmix64 outputs from hash_seed, row by row, in the
 *     order a0, a1, a2, b;
 *   - cell: c = floor(fl32(x * inv_cell)) reduced periodically into [0, G),
 *     key = cx + G*(cy + G*cz); particles whose scaled coordinate is not a
 *     finite value in [-2^31, 2^31) are skipped;
 *   - sampling: keep particle g iff the splitmix64 output at position g of the
 *     sequence seeded by sample_seed is below floor(rate * 2^64); rate >= 1
 *     keeps every particle without hashing;
 *   - median: lower median (sorted index floor((t-1)/2));
 *   - ranking: estimate descending, then key ascending; exactly min(k, G^3)
 *     entries; counters are int32 with two's-complement wrap-around.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_GAMMA 0x9E3779B97F4A7C15ULL
#define OR_INVALID_KEY 0xFFFFFFFFFFFFFFFFULL

/* ---- splitmix64 (Steele, Lea, Flood 2014), from its published definition ---- */

static uint64_t or_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* advance the state by the golden gamma and return the mixed output */
uint64_t or_splitmix64_next(uint64_t *state) {
    *state += OR_GAMMA;
    return or_mix(*state);
}

/* output number g (0-based) of the generator seeded with `seed` */
uint64_t or_splitmix64_at(uint64_t seed, uint64_t g) {
    uint64_t s = seed + (g + 1) * OR_GAMMA;
    return or_mix(s);
}

/* Row seeds: out[4r + 0..3] = a0, a1, a2, b of row r. */
void or_derive_seeds(uint64_t hash_seed, uint32_t t, uint64_t *out) {
    uint64_t st = hash_seed;
    for (uint32_t i = 0; i < 4 * t; ++i) out[i] = or_splitmix64_next(&st);
}

/* ---- mesh reduction (Sec. 2.1) ---- */

uint32_t or_grid_size(double box, double cell) { return (uint32_t)llround(box / cell); }
float or_inv_cell(double cell) { return (float)(1.0 / cell); }

/* One coordinate: 1 and the cell index in [0, G), or 0 when the particle is skipped. */
static int or_axis(float x, float inv, uint32_t G, uint32_t *c) {
    float p = x * inv;                      /* one float32 rounding */
    float f = floorf(p);
    if (!(f >= -2147483648.0f && f < 2147483648.0f)) return 0;
    int64_t i = (int64_t)f;
    int64_t g = (int64_t)G;
    int64_t m = i % g;
    if (m < 0) m += g;                      /* periodic box */
    *c = (uint32_t)m;
    return 1;
}

int or_cell(float x, float y, float z, float inv, uint32_t G, uint32_t *c3) {
    return or_axis(x, inv, G, &c3[0]) && or_axis(y, inv, G, &c3[1]) && or_axis(z, inv, G, &c3[2]);
}

uint64_t or_key_of(const uint32_t *c3, uint32_t G) {
    return (uint64_t)c3[0] + (uint64_t)G * ((uint64_t)c3[1] + (uint64_t)G * (uint64_t)c3[2]);
}

void or_key_decode(uint64_t key, uint32_t G, uint32_t *c3) {
    c3[0] = (uint32_t)(key % G);
    c3[1] = (uint32_t)((key / G) % G);
    c3[2] = (uint32_t)(key / ((uint64_t)G * G));
}

void or_keys(const float *xyz, uint64_t n, float inv, uint32_t G, uint64_t *keys) {
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t c[3];
        keys[i] = or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c) ? or_key_of(c, G)
                                                                                 : OR_INVALID_KEY;
    }
}

/* ---- sampling (Sec. 3.1) ---- */

uint64_t or_sample_threshold(double rate) {
    if (!(rate < 1.0)) return 0;           /* unused: keep all */
    return (uint64_t)ldexp(rate, 64);
}

int or_keep(uint64_t g, uint64_t sample_seed, double rate) {
    if (rate >= 1.0) return 1;
    return or_splitmix64_at(sample_seed, g) < or_sample_threshold(rate);
}

/* ---- Count Sketch hashes (Sec. 2.2) ---- */

void or_hash_row(const uint64_t *s4, const uint32_t *c3, uint32_t log2w, uint32_t *bucket,
                 int32_t *sign) {
    uint64_t v = s4[0] * (uint64_t)c3[0] + s4[1] * (uint64_t)c3[1] + s4[2] * (uint64_t)c3[2] + s4[3];
    *bucket = (uint32_t)(v >> (64 - log2w));
    *sign = ((v >> (63 - log2w)) & 1ULL) ? -1 : 1;
}

/* Add(M, s) for one cell (Sec. 2.2), int32 counters with wrap-around. */
static void or_add(int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                   const uint32_t *c3) {
    uint64_t W = 1ULL << log2w;
    for (uint32_t r = 0; r < t; ++r) {
        uint32_t b;
        int32_t s;
        or_hash_row(seeds + 4 * r, c3, log2w, &b, &s);
        uint32_t *cell = (uint32_t *)&C[r * W + b];
        *cell = *cell + (uint32_t)s;
    }
}

/*
 * Processing the stream (Algorithm 1): particles [0, n) of this call have
 * global indices g0 + i.  nthreads > 1 gives each thread a private copy of the
 * counters and sums them at the end; integer addition commutes, so the result
 * equals the sequential loop bit for bit.
 */
int or_sketch_update(int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                     const float *xyz, uint64_t n, uint64_t g0, float inv, uint32_t G,
                     uint64_t sample_seed, double rate, int nthreads) {
    uint64_t W = 1ULL << log2w;
    uint64_t total = (uint64_t)t * W;
    if (nthreads <= 1) {
        for (uint64_t i = 0; i < n; ++i) {
            if (!or_keep(g0 + i, sample_seed, rate)) continue;
            uint32_t c[3];
            if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c)) continue;
            or_add(C, t, log2w, seeds, c);
        }
        return 0;
    }
#ifdef _OPENMP
    int nt = nthreads;
    uint32_t **priv = (uint32_t **)calloc((size_t)nt, sizeof(uint32_t *));
    if (!priv) return 1;
    for (int k = 0; k < nt; ++k) {
        priv[k] = (uint32_t *)calloc(total, sizeof(uint32_t));
        if (!priv[k]) {
            for (int q = 0; q < k; ++q) free(priv[q]);
            free(priv);
            return 1;
        }
    }
#pragma omp parallel num_threads(nt)
    {
        int me = omp_get_thread_num();
        int32_t *P = (int32_t *)priv[me];
        uint64_t lo = n * (uint64_t)me / (uint64_t)nt, hi = n * (uint64_t)(me + 1) / (uint64_t)nt;
        for (uint64_t i = lo; i < hi; ++i) {
            if (!or_keep(g0 + i, sample_seed, rate)) continue;
            uint32_t c[3];
            if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c)) continue;
            or_add(P, t, log2w, seeds, c);
        }
    }
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t j = 0; j < (int64_t)total; ++j) {
        uint32_t acc = (uint32_t)C[j];
        for (int k = 0; k < nt; ++k) acc += priv[k][j];
        C[j] = (int32_t)acc;
    }
    for (int k = 0; k < nt; ++k) free(priv[k]);
    free(priv);
    return 0;
#else
    return or_sketch_update(C, t, log2w, seeds, xyz, n, g0, inv, G, sample_seed, rate, 1);
#endif
}

/* ---- Estimate (Sec. 2.2) ---- */

static int32_t or_lower_median(int32_t *v, uint32_t t) {
    for (uint32_t i = 1; i < t; ++i) {          /* insertion sort */
        int32_t x = v[i];
        uint32_t j = i;
        while (j > 0 && v[j - 1] > x) { v[j] = v[j - 1]; --j; }
        v[j] = x;
    }
    return v[(t - 1) / 2];
}

int32_t or_estimate_cell(const int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                         const uint32_t *c3) {
    uint64_t W = 1ULL << log2w;
    int32_t v[64];
    for (uint32_t r = 0; r < t; ++r) {
        uint32_t b;
        int32_t s;
        or_hash_row(seeds + 4 * r, c3, log2w, &b, &s);
        v[r] = (int32_t)((uint32_t)C[r * W + b] * (uint32_t)s);   /* wraps like int32 */
    }
    return or_lower_median(v, t);
}

/* per-row estimates of one key (test aid) */
void or_row_estimates(const int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                      uint64_t key, uint32_t G, int32_t *out) {
    uint64_t W = 1ULL << log2w;
    uint32_t c[3];
    or_key_decode(key, G, c);
    for (uint32_t r = 0; r < t; ++r) {
        uint32_t b;
        int32_t s;
        or_hash_row(seeds + 4 * r, c, log2w, &b, &s);
        out[r] = (int32_t)((uint32_t)C[r * W + b] * (uint32_t)s);
    }
}

void or_estimate(const int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                 const uint64_t *keys, uint64_t m, uint32_t G, int32_t *out) {
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t c[3];
        or_key_decode(keys[i], G, c);
        out[i] = or_estimate_cell(C, t, log2w, seeds, c);
    }
}

/* ---- top-k by (estimate desc, key asc) ---- */

typedef struct { int32_t est; uint64_t key; } or_entry;

/* a ranks after b */
static int or_worse(const or_entry *a, const or_entry *b) {
    return a->est < b->est || (a->est == b->est && a->key > b->key);
}

/* heap with the worst entry at the root */
static void or_sift_down(or_entry *h, uint64_t n, uint64_t i) {
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, w = i;
        if (l < n && or_worse(&h[l], &h[w])) w = l;
        if (r < n && or_worse(&h[r], &h[w])) w = r;
        if (w == i) return;
        or_entry tmp = h[i]; h[i] = h[w]; h[w] = tmp;
        i = w;
    }
}

static void or_sift_up(or_entry *h, uint64_t i) {
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!or_worse(&h[i], &h[p])) return;
        or_entry tmp = h[i]; h[i] = h[p]; h[p] = tmp;
        i = p;
    }
}

static void or_offer(or_entry *h, uint64_t *n, uint64_t k, or_entry e) {
    if (*n < k) { h[*n] = e; or_sift_up(h, *n); ++*n; }
    else if (or_worse(&h[0], &e)) { h[0] = e; or_sift_down(h, *n, 0); }
}

static int or_cmp_rank(const void *pa, const void *pb) {
    const or_entry *a = (const or_entry *)pa, *b = (const or_entry *)pb;
    if (a->est != b->est) return a->est > b->est ? -1 : 1;
    return (a->key < b->key) ? -1 : (a->key > b->key);
}

/*
 * Querying the data structure (Algorithm 1, CSFS): Estimate every cell
 * j in [key_lo, key_hi) of the dictionary and keep the k best.  Returns the
 * number written (min(k, key_hi - key_lo)), sorted by rank.  With nthreads > 1
 * each thread scans a contiguous key range with its own heap; the union of the
 * per-range top-k contains the global top-k.
 */
uint64_t or_topk_range(const int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                       uint32_t G, uint64_t key_lo, uint64_t key_hi, uint32_t k,
                       uint64_t *keys_out, int32_t *est_out, int nthreads) {
    if (key_hi <= key_lo || k == 0) return 0;
    uint64_t span = key_hi - key_lo;
    int nt = nthreads < 1 ? 1 : nthreads;
#ifndef _OPENMP
    nt = 1;
#endif
    or_entry *all = (or_entry *)malloc(sizeof(or_entry) * (uint64_t)k * (uint64_t)nt);
    uint64_t *cnt = (uint64_t *)calloc((size_t)nt, sizeof(uint64_t));
    if (!all || !cnt) { free(all); free(cnt); return 0; }
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int me = 0;
#ifdef _OPENMP
        me = omp_get_thread_num();
#endif
        or_entry *h = all + (uint64_t)k * (uint64_t)me;
        uint64_t n = 0;
        uint64_t lo = key_lo + span * (uint64_t)me / (uint64_t)nt;
        uint64_t hi = key_lo + span * (uint64_t)(me + 1) / (uint64_t)nt;
        for (uint64_t key = lo; key < hi; ++key) {
            uint32_t c[3];
            or_key_decode(key, G, c);
            or_entry e;
            e.est = or_estimate_cell(C, t, log2w, seeds, c);
            e.key = key;
            or_offer(h, &n, k, e);
        }
        cnt[me] = n;
    }
    /* gather the per-range lists and rank them */
    uint64_t tot = 0;
    for (int q = 0; q < nt; ++q) {
        memmove(all + tot, all + (uint64_t)k * (uint64_t)q, sizeof(or_entry) * cnt[q]);
        tot += cnt[q];
    }
    qsort(all, tot, sizeof(or_entry), or_cmp_rank);
    uint64_t out = tot < k ? tot : k;
    for (uint64_t i = 0; i < out; ++i) { keys_out[i] = all[i].key; est_out[i] = all[i].est; }
    free(all);
    free(cnt);
    return out;
}

uint64_t or_topk_full(const int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                      uint32_t G, uint32_t k, uint64_t *keys_out, int32_t *est_out, int nthreads) {
    uint64_t n = (uint64_t)G * G * G;
    return or_topk_range(C, t, log2w, seeds, G, 0, n, k, keys_out, est_out, nthreads);
}

/* ---- exact algorithm (Sec. 4.2): one counter per occupied cell ---- */

typedef struct {
    uint64_t *keys;   /* key + 1, 0 = empty */
    uint32_t *cnt;
    uint64_t cap;     /* power of two */
    uint64_t used;
} or_map;

static uint64_t or_slot(uint64_t key, uint64_t mask) {
    return or_mix(key ^ 0x2545F4914F6CDD1DULL) & mask;
}

static int or_map_grow(or_map *m);

static int or_map_add(or_map *m, uint64_t key, uint32_t inc) {
    if ((m->used + 1) * 2 > m->cap && or_map_grow(m)) return 1;
    uint64_t mask = m->cap - 1, s = or_slot(key, mask);
    for (;;) {
        if (m->keys[s] == 0) { m->keys[s] = key + 1; m->cnt[s] = inc; ++m->used; return 0; }
        if (m->keys[s] == key + 1) { m->cnt[s] += inc; return 0; }
        s = (s + 1) & mask;
    }
}

static int or_map_grow(or_map *m) {
    or_map n;
    n.cap = m->cap ? m->cap * 2 : 1024;
    n.used = 0;
    n.keys = (uint64_t *)calloc(n.cap, sizeof(uint64_t));
    n.cnt = (uint32_t *)calloc(n.cap, sizeof(uint32_t));
    if (!n.keys || !n.cnt) { free(n.keys); free(n.cnt); return 1; }
    for (uint64_t i = 0; i < m->cap; ++i)
        if (m->keys[i]) {
            uint64_t mask = n.cap - 1, s = or_slot(m->keys[i] - 1, mask);
            while (n.keys[s]) s = (s + 1) & mask;
            n.keys[s] = m->keys[i];
            n.cnt[s] = m->cnt[i];
            ++n.used;
        }
    free(m->keys);
    free(m->cnt);
    *m = n;
    return 0;
}

static int or_cmp_key(const void *pa, const void *pb) {
    const or_entry *a = (const or_entry *)pa, *b = (const or_entry *)pb;
    return (a->key < b->key) ? -1 : (a->key > b->key);
}

/*
 * Exact counts of the kept particles' cells.  Returns the number of distinct
 * cells D; when D <= cap, keys_out/cnt_out hold them sorted by key.
 */
uint64_t or_exact_counts(const float *xyz, uint64_t n, uint64_t g0, float inv, uint32_t G,
                         uint64_t sample_seed, double rate, uint64_t *keys_out, uint32_t *cnt_out,
                         uint64_t cap) {
    or_map m = {0, 0, 0, 0};
    if (or_map_grow(&m)) return 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (!or_keep(g0 + i, sample_seed, rate)) continue;
        uint32_t c[3];
        if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c)) continue;
        if (or_map_add(&m, or_key_of(c, G), 1)) break;
    }
    uint64_t D = m.used;
    if (D <= cap) {
        or_entry *e = (or_entry *)malloc(sizeof(or_entry) * (D ? D : 1));
        if (e) {
            uint64_t q = 0;
            for (uint64_t i = 0; i < m.cap; ++i)
                if (m.keys[i]) { e[q].key = m.keys[i] - 1; e[q].est = (int32_t)m.cnt[i]; ++q; }
            qsort(e, D, sizeof(or_entry), or_cmp_key);
            for (uint64_t i = 0; i < D; ++i) { keys_out[i] = e[i].key; cnt_out[i] = (uint32_t)e[i].est; }
            free(e);
        }
    }
    free(m.keys);
    free(m.cnt);
    return D;
}

/* ======================================================================
 * Learned router (an addition to the paper's method; the paper finds heavy
 * cells with the Count Sketch alone).  Coarse cell = fine cell / R per axis.
 * ====================================================================== */

#define OR_MLP_IN 27
#define OR_MLP_H 64
#define OR_MLP_PARAMS (OR_MLP_H * OR_MLP_IN + OR_MLP_H + OR_MLP_H * OR_MLP_H + OR_MLP_H + OR_MLP_H + 1)

/* sample counts of the coarse cells (feature pass) */
void or_coarse_hist(const float *xyz, uint64_t n, uint64_t g0, float inv, uint32_t G, uint32_t R,
                    uint64_t feature_seed, double feature_rate, int32_t *counts) {
    uint32_t Gc = G / R;
    for (uint64_t i = 0; i < n; ++i) {
        if (!or_keep(g0 + i, feature_seed, feature_rate)) continue;
        uint32_t c[3];
        if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c)) continue;
        uint64_t ck = (uint64_t)(c[0] / R) + (uint64_t)Gc * ((uint64_t)(c[1] / R) + (uint64_t)Gc * (c[2] / R));
        counts[ck] += 1;
    }
}

/* bf16 bit pattern of a float: round to nearest, ties to even */
uint16_t or_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

static float or_from_bf16(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* feature of a count: bf16(float(log10(1 + n))) */
uint16_t or_feature_of(int32_t n) { return or_bf16((float)log10(1.0 + (double)n)); }

/* 27 features of each coarse key: neighbour (dx, dy, dz) at (dz+1)*9 + (dy+1)*3 + (dx+1) */
void or_features(const int32_t *counts, uint32_t Gc, const uint64_t *keys, uint64_t m, uint16_t *out) {
    for (uint64_t s = 0; s < m; ++s) {
        int64_t x = (int64_t)(keys[s] % Gc), y = (int64_t)((keys[s] / Gc) % Gc),
                z = (int64_t)(keys[s] / ((uint64_t)Gc * Gc));
        int f = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++f) {
                    int64_t xx = (x + dx + Gc) % Gc, yy = (y + dy + Gc) % Gc, zz = (z + dz + Gc) % Gc;
                    out[s * OR_MLP_IN + f] = or_feature_of(counts[xx + (int64_t)Gc * (yy + (int64_t)Gc * zz)]);
                }
    }
}

/* Forward pass in the kernel's precision: bf16 weights, inputs and hidden
 * activations; each neuron a float32 fmaf chain in index order from its bias. */
void or_mlp_forward_f32(const float *P, const uint16_t *feats, uint64_t m, float *logits) {
    float w[OR_MLP_PARAMS];
    for (int i = 0; i < OR_MLP_PARAMS; ++i) w[i] = or_from_bf16(or_bf16(P[i]));
    const float *w1 = w, *b1 = w1 + OR_MLP_H * OR_MLP_IN, *w2 = b1 + OR_MLP_H,
                *b2 = w2 + OR_MLP_H * OR_MLP_H, *w3 = b2 + OR_MLP_H, *b3 = w3 + OR_MLP_H;
    for (uint64_t s = 0; s < m; ++s) {
        float x[OR_MLP_IN], h1[OR_MLP_H], h2[OR_MLP_H];
        for (int i = 0; i < OR_MLP_IN; ++i) x[i] = or_from_bf16(feats[s * OR_MLP_IN + i]);
        for (int j = 0; j < OR_MLP_H; ++j) {
            float a = b1[j];
            for (int i = 0; i < OR_MLP_IN; ++i) a = fmaf(w1[j * OR_MLP_IN + i], x[i], a);
            h1[j] = or_from_bf16(or_bf16(a > 0.0f ? a : 0.0f));
        }
        for (int j = 0; j < OR_MLP_H; ++j) {
            float a = b2[j];
            for (int i = 0; i < OR_MLP_H; ++i) a = fmaf(w2[j * OR_MLP_H + i], h1[i], a);
            h2[j] = or_from_bf16(or_bf16(a > 0.0f ? a : 0.0f));
        }
        float z = b3[0];
        for (int i = 0; i < OR_MLP_H; ++i) z = fmaf(w3[i], h2[i], z);
        logits[s] = z;
    }
}

static int or_routed(const uint8_t *routed, const uint32_t *c3, uint32_t R, uint32_t Gc) {
    uint64_t ck = (uint64_t)(c3[0] / R) + (uint64_t)Gc * ((uint64_t)(c3[1] / R) + (uint64_t)Gc * (c3[2] / R));
    return routed[ck] != 0;
}

/*
 * The learned update: each kept particle in a routed coarse cell increments
 * its fine cell's exact count; every other kept particle is added to the
 * sketch (Add, Sec. 2.2).  routed: one byte per coarse cell.  Returns the
 * number of distinct routed fine cells; when <= cap, keys/counts hold them
 * sorted by key.
 */
uint64_t or_learned_update(int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                           const float *xyz, uint64_t n, uint64_t g0, float inv, uint32_t G,
                           uint64_t sample_seed, double rate, const uint8_t *routed, uint32_t R,
                           uint64_t *keys_out, uint32_t *cnt_out, uint64_t cap) {
    uint32_t Gc = G / R;
    or_map m = {0, 0, 0, 0};
    if (or_map_grow(&m)) return 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (!or_keep(g0 + i, sample_seed, rate)) continue;
        uint32_t c[3];
        if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c)) continue;
        if (or_routed(routed, c, R, Gc)) or_map_add(&m, or_key_of(c, G), 1);
        else or_add(C, t, log2w, seeds, c);
    }
    uint64_t D = m.used;
    if (D <= cap) {
        or_entry *e = (or_entry *)malloc(sizeof(or_entry) * (D ? D : 1));
        uint64_t q = 0;
        for (uint64_t i = 0; i < m.cap; ++i)
            if (m.keys[i]) { e[q].key = m.keys[i] - 1; e[q].est = (int32_t)m.cnt[i]; ++q; }
        qsort(e, D, sizeof(or_entry), or_cmp_key);
        for (uint64_t i = 0; i < D; ++i) { keys_out[i] = e[i].key; cnt_out[i] = (uint32_t)e[i].est; }
        free(e);
    }
    free(m.keys);
    free(m.cnt);
    return D;
}

/* CSFS over the cells of [key_lo, key_hi) that are not in routed coarse cells */
uint64_t or_topk_unrouted(const int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                          uint32_t G, const uint8_t *routed, uint32_t R, uint32_t k,
                          uint64_t *keys_out, int32_t *est_out) {
    uint64_t n = (uint64_t)G * G * G;
    uint32_t Gc = G / R;
    or_entry *h = (or_entry *)malloc(sizeof(or_entry) * (k ? k : 1));
    uint64_t cnt = 0;
    for (uint64_t key = 0; key < n; ++key) {
        uint32_t c[3];
        or_key_decode(key, G, c);
        if (or_routed(routed, c, R, Gc)) continue;
        or_entry e;
        e.est = or_estimate_cell(C, t, log2w, seeds, c);
        e.key = key;
        or_offer(h, &cnt, k, e);
    }
    qsort(h, cnt, sizeof(or_entry), or_cmp_rank);
    for (uint64_t i = 0; i < cnt; ++i) { keys_out[i] = h[i].key; est_out[i] = h[i].est; }
    free(h);
    return cnt;
}

/* ======================================================================
 * Count Sketch Hierarchical (Algorithm 3, CSHi; the "GPU hierarchy" variant
 * of Sec. 3): a second sketch M1 counts super-items, a cell's super-item
 * being the F x F x F block holding it (super coords = cell coords / F on a
 * grid of G / F).  The query finds the c*k best super-items by M1's
 * estimates, then ranks every cell inside them by M2's estimates.
 * ====================================================================== */

/* Add(M1, super-item of s_i) for every kept particle (Algorithm 3, processing the stream) */
void or_sketch_update_super(int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                            const float *xyz, uint64_t n, uint64_t g0, float inv, uint32_t G,
                            uint32_t F, uint64_t sample_seed, double rate) {
    for (uint64_t i = 0; i < n; ++i) {
        if (!or_keep(g0 + i, sample_seed, rate)) continue;
        uint32_t c[3];
        if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c)) continue;
        uint32_t q[3] = {c[0] / F, c[1] / F, c[2] / F};
        or_add(C, t, log2w, seeds, q);
    }
}

/*
 * Querying (Algorithm 3 with the top-(c*k) rule of the GPU hierarchy): the
 * m_super = min(c*k, (G/F)^3) best super-items of M1 (CSFS over the super
 * dictionary), then the k best cells of those super-items by M2, ranked by
 * (estimate desc, key asc).  Returns the number written.
 */
uint64_t or_topk_hier(const int32_t *C2, uint32_t t2, uint32_t log2w2, const uint64_t *seeds2,
                      const int32_t *C1, uint32_t t1, uint32_t log2w1, const uint64_t *seeds1,
                      uint32_t G, uint32_t F, uint32_t k, uint32_t c_mult,
                      uint64_t *keys_out, int32_t *est_out, int nthreads) {
    uint32_t Gs = G / F;
    uint64_t ns = (uint64_t)Gs * Gs * Gs;
    uint64_t m = (uint64_t)c_mult * k;
    if (m > ns) m = ns;
    if (k == 0 || m == 0) return 0;
    uint64_t *skeys = (uint64_t *)malloc(sizeof(uint64_t) * m);
    int32_t *sest = (int32_t *)malloc(sizeof(int32_t) * m);
    or_entry *h = (or_entry *)malloc(sizeof(or_entry) * k);
    if (!skeys || !sest || !h) { free(skeys); free(sest); free(h); return 0; }
    uint64_t got = or_topk_range(C1, t1, log2w1, seeds1, Gs, 0, ns, (uint32_t)m, skeys, sest, nthreads);
    uint64_t cnt = 0;
    for (uint64_t s = 0; s < got; ++s) {
        uint32_t q[3];
        or_key_decode(skeys[s], Gs, q);
        for (uint32_t lz = 0; lz < F; ++lz)
            for (uint32_t ly = 0; ly < F; ++ly)
                for (uint32_t lx = 0; lx < F; ++lx) {
                    uint32_t c[3] = {q[0] * F + lx, q[1] * F + ly, q[2] * F + lz};
                    or_entry e;
                    e.est = or_estimate_cell(C2, t2, log2w2, seeds2, c);
                    e.key = or_key_of(c, G);
                    or_offer(h, &cnt, k, e);
                }
    }
    qsort(h, cnt, sizeof(or_entry), or_cmp_rank);
    for (uint64_t i = 0; i < cnt; ++i) { keys_out[i] = h[i].key; est_out[i] = h[i].est; }
    free(skeys);
    free(sest);
    free(h);
    return cnt;
}

/*
 * The hierarchical query of a learned sketch: the c*k best super-items of M1
 * (which counts every kept particle), then the k best cells inside them that
 * are not in routed coarse cells (routed: one byte per coarse cell of R^3
 * cells), by M2's estimates.  The exact counts of routed cells are merged by
 * the caller.
 */
uint64_t or_topk_hier_unrouted(const int32_t *C2, uint32_t t2, uint32_t log2w2, const uint64_t *seeds2,
                               const int32_t *C1, uint32_t t1, uint32_t log2w1, const uint64_t *seeds1,
                               uint32_t G, uint32_t F, uint32_t k, uint32_t c_mult,
                               const uint8_t *routed, uint32_t R,
                               uint64_t *keys_out, int32_t *est_out, int nthreads) {
    uint32_t Gs = G / F, Gc = G / R;
    uint64_t ns = (uint64_t)Gs * Gs * Gs;
    uint64_t m = (uint64_t)c_mult * k;
    if (m > ns) m = ns;
    if (k == 0 || m == 0) return 0;
    uint64_t *skeys = (uint64_t *)malloc(sizeof(uint64_t) * m);
    int32_t *sest = (int32_t *)malloc(sizeof(int32_t) * m);
    or_entry *h = (or_entry *)malloc(sizeof(or_entry) * k);
    if (!skeys || !sest || !h) { free(skeys); free(sest); free(h); return 0; }
    uint64_t got = or_topk_range(C1, t1, log2w1, seeds1, Gs, 0, ns, (uint32_t)m, skeys, sest, nthreads);
    uint64_t cnt = 0;
    for (uint64_t s = 0; s < got; ++s) {
        uint32_t q[3];
        or_key_decode(skeys[s], Gs, q);
        for (uint32_t lz = 0; lz < F; ++lz)
            for (uint32_t ly = 0; ly < F; ++ly)
                for (uint32_t lx = 0; lx < F; ++lx) {
                    uint32_t c[3] = {q[0] * F + lx, q[1] * F + ly, q[2] * F + lz};
                    if (or_routed(routed, c, R, Gc)) continue;
                    or_entry e;
                    e.est = or_estimate_cell(C2, t2, log2w2, seeds2, c);
                    e.key = or_key_of(c, G);
                    or_offer(h, &cnt, k, e);
                }
    }
    qsort(h, cnt, sizeof(or_entry), or_cmp_rank);
    for (uint64_t i = 0; i < cnt; ++i) { keys_out[i] = h[i].key; est_out[i] = h[i].est; }
    free(skeys);
    free(sest);
    free(h);
    return cnt;
}

/* ---- threaded forms of the learned-router oracle (for 10^9-particle checks) ----
 * Same arithmetic as the single-threaded functions above: the forward pass is
 * independent per sample, and the update's private counters and maps are
 * integer sums, so the results are equal bit for bit. */

void or_mlp_forward_f32_mt(const float *P, const uint16_t *feats, uint64_t m, float *logits,
                           int nthreads) {
#ifdef _OPENMP
    int nt = nthreads < 1 ? 1 : nthreads;
#pragma omp parallel num_threads(nt)
    {
        int me = omp_get_thread_num(), k = omp_get_num_threads();
        uint64_t lo = m * (uint64_t)me / (uint64_t)k, hi = m * (uint64_t)(me + 1) / (uint64_t)k;
        if (hi > lo) or_mlp_forward_f32(P, feats + lo * OR_MLP_IN, hi - lo, logits + lo);
    }
#else
    (void)nthreads;
    or_mlp_forward_f32(P, feats, m, logits);
#endif
}

uint64_t or_learned_update_mt(int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                              const float *xyz, uint64_t n, uint64_t g0, float inv, uint32_t G,
                              uint64_t sample_seed, double rate, const uint8_t *routed, uint32_t R,
                              uint64_t *keys_out, uint32_t *cnt_out, uint64_t cap, int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 1)
#endif
        return or_learned_update(C, t, log2w, seeds, xyz, n, g0, inv, G, sample_seed, rate, routed,
                                 R, keys_out, cnt_out, cap);
#ifdef _OPENMP
    const uint64_t total = (uint64_t)t << log2w;
    const uint32_t Gc = G / R;
    const int nt = nthreads;
    uint32_t **priv = (uint32_t **)calloc((size_t)nt, sizeof(uint32_t *));
    or_map *maps = (or_map *)calloc((size_t)nt, sizeof(or_map));
    int bad = !priv || !maps;
    for (int k = 0; k < nt && !bad; ++k) {
        priv[k] = (uint32_t *)calloc(total, sizeof(uint32_t));
        bad = !priv[k] || or_map_grow(&maps[k]);
    }
    if (!bad) {
#pragma omp parallel num_threads(nt)
        {
            int me = omp_get_thread_num();
            uint64_t lo = n * (uint64_t)me / (uint64_t)nt, hi = n * (uint64_t)(me + 1) / (uint64_t)nt;
            for (uint64_t i = lo; i < hi; ++i) {
                if (!or_keep(g0 + i, sample_seed, rate)) continue;
                uint32_t c[3];
                if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, G, c)) continue;
                if (or_routed(routed, c, R, Gc)) or_map_add(&maps[me], or_key_of(c, G), 1);
                else or_add((int32_t *)priv[me], t, log2w, seeds, c);
            }
        }
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t j = 0; j < (int64_t)total; ++j) {
            uint32_t acc = (uint32_t)C[j];
            for (int k = 0; k < nt; ++k) acc += priv[k][j];
            C[j] = (int32_t)acc;
        }
        for (int k = 1; k < nt; ++k)
            for (uint64_t i = 0; i < maps[k].cap; ++i)
                if (maps[k].keys[i]) or_map_add(&maps[0], maps[k].keys[i] - 1, maps[k].cnt[i]);
    }
    uint64_t D = 0;
    if (!bad) {
        D = maps[0].used;
        if (D <= cap) {
            or_entry *e = (or_entry *)malloc(sizeof(or_entry) * (D ? D : 1));
            uint64_t q = 0;
            for (uint64_t i = 0; i < maps[0].cap; ++i)
                if (maps[0].keys[i]) { e[q].key = maps[0].keys[i] - 1; e[q].est = (int32_t)maps[0].cnt[i]; ++q; }
            qsort(e, D, sizeof(or_entry), or_cmp_key);
            for (uint64_t i = 0; i < D; ++i) { keys_out[i] = e[i].key; cnt_out[i] = (uint32_t)e[i].est; }
            free(e);
        }
    }
    for (int k = 0; k < nt; ++k) {
        if (priv) free(priv[k]);
        if (maps) { free(maps[k].keys); free(maps[k].cnt); }
    }
    free(priv);
    free(maps);
    return D;
#endif
}

/* ======================================================================
 * Packed particle records (the evaluation setup of Sec. 4: "every 64 bits
 * contains 3 coordinates for one particle").  Reading: 21 bits per
 * coordinate, q = floor(fl32(x * fl32(2^21 / L))) reduced periodically into
 * [0, 2^21), x in bits 0-20, y in 21-41, z in 42-62; bit 63 marks a particle
 * whose coordinates were not finite (skipped).  The cell of a record on a mesh
 * of G cells per axis is (q * G) >> 21 per axis.
 * ====================================================================== */

#define OR_PACK_BITS 21
#define OR_PACK_LEVELS (1u << OR_PACK_BITS)
#define OR_PACK_INVALID (1ull << 63)

void or_pack(const float *xyz, uint64_t n, double box, uint64_t *out) {
    float inv = (float)((double)OR_PACK_LEVELS / box);
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        if (!or_cell(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], inv, OR_PACK_LEVELS, q)) {
            out[i] = OR_PACK_INVALID;
            continue;
        }
        out[i] = (uint64_t)q[0] | ((uint64_t)q[1] << OR_PACK_BITS) | ((uint64_t)q[2] << (2 * OR_PACK_BITS));
    }
}

int or_cell_packed(uint64_t p, uint32_t G, uint32_t *c3) {
    if (p & OR_PACK_INVALID) return 0;
    const uint64_t m = OR_PACK_LEVELS - 1;
    for (int a = 0; a < 3; ++a) c3[a] = (uint32_t)((((p >> (OR_PACK_BITS * a)) & m) * (uint64_t)G) >> OR_PACK_BITS);
    return 1;
}

/* Processing a packed stream (Algorithm 1): cells of the records, divided by F
 * per axis for a super-item sketch (F = 1: the cells themselves). */
int or_sketch_update_packed(int32_t *C, uint32_t t, uint32_t log2w, const uint64_t *seeds,
                            const uint64_t *packed, uint64_t n, uint64_t g0, uint32_t G, uint32_t F,
                            uint64_t sample_seed, double rate, int nthreads) {
    const uint64_t total = (uint64_t)t << log2w;
    int nt = nthreads < 1 ? 1 : nthreads;
#ifndef _OPENMP
    nt = 1;
#endif
    uint32_t **priv = (uint32_t **)calloc((size_t)nt, sizeof(uint32_t *));
    if (!priv) return 1;
    for (int k = 0; k < nt; ++k) {
        priv[k] = (uint32_t *)calloc(total, sizeof(uint32_t));
        if (!priv[k]) {
            for (int q = 0; q < k; ++q) free(priv[q]);
            free(priv);
            return 1;
        }
    }
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int me = 0;
#ifdef _OPENMP
        me = omp_get_thread_num();
#endif
        uint64_t lo = n * (uint64_t)me / (uint64_t)nt, hi = n * (uint64_t)(me + 1) / (uint64_t)nt;
        for (uint64_t i = lo; i < hi; ++i) {
            if (!or_keep(g0 + i, sample_seed, rate)) continue;
            uint32_t c[3];
            if (!or_cell_packed(packed[i], G, c)) continue;
            c[0] /= F;
            c[1] /= F;
            c[2] /= F;
            or_add((int32_t *)priv[me], t, log2w, seeds, c);
        }
    }
    for (uint64_t j = 0; j < total; ++j) {
        uint32_t acc = (uint32_t)C[j];
        for (int k = 0; k < nt; ++k) acc += priv[k][j];
        C[j] = (int32_t)acc;
    }
    for (int k = 0; k < nt; ++k) free(priv[k]);
    free(priv);
    return 0;
}
