/*
 * halosketch.h - C ABI of the GB300 (sm_103a) Count Sketch halo finder.
 *
 * The library implements the data-parallel hot path of Ivkin et al.,
 * "Scalable Streaming Tools for Analyzing N-body Simulations: Finding Halos
 * and Investigating Excursion Sets in One Pass" (arXiv:1711.00975):
 *
 *   particle xyz --(mesh reduction, Sec. 2.1)--> cell key
 *                --(Bernoulli sampling by an index hash, Sec. 3.1)-->
 *                --(Count Sketch Add, Sec. 2.2)--> t x W int32 counters
 *   counters --(Estimate = median of rows, Sec. 2.2; full search over every
 *               cell, Algorithm 1 "CSFS")--> top-k heaviest cells.
 *
 * It answers the top-k form of the Heavy Hitter problem (Sec. 2.1, Problem 1:
 * the k most frequent cells are the (alpha_k, l1)-heavy items).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an hs_status; none aborts.  On failure the thread's
 *    last error message is available from hs_last_error().
 *  - The caller owns all input and output buffers; the library owns the
 *    counters and its scratch memory.
 *  - Buffers may be device memory or host memory (pageable or pinned) unless
 *    the entry point says otherwise; the library inspects each pointer.
 *  - Work is ordered on the CUDA stream given to sketch_create (the legacy
 *    default stream when NULL).  Calls on one handle are not thread-safe.
 *  - Particles are float32 xyz triples, array-of-structures
 *    [x0, y0, z0, x1, y1, z1, ...], 12 bytes per particle.
 *  - Cells: G = round(box / cell) per axis, inv_cell = (float)(1.0 / cell)
 *    (computed in double, rounded once to float).  The cell coordinate on each
 *    axis is floor(fl32(x * inv_cell)) reduced periodically into [0, G); a
 *    particle whose scaled coordinate is not a finite value in
 *    [-2^31, 2^31) is skipped.  key = cx + G * (cy + G * cz) (uint64).
 *  - Row r of the sketch hashes a cell with vector multiply-shift:
 *    v = (a0*cx + a1*cy + a2*cz + b) mod 2^64, bucket = v >> (64 - log2W),
 *    sign = -1 if bit (63 - log2W) of v is set, else +1.  (a0, a1, a2, b) of
 *    row r are splitmix64 outputs 4r .. 4r+3 of the generator seeded with
 *    hash_seed.
 *  - Sampling: particle number g of the stream (g counts every particle ever
 *    passed to sketch_update on this handle, from 0) is kept iff rate >= 1 or
 *    splitmix64 output number g of the generator seeded with sample_seed is
 *    below floor(rate * 2^64).
 *  - Estimate(key) = lower median over rows of sign_r(key) * C[r][bucket_r(key)]
 *    (int32, two's-complement wrap-around; counters wrap the same way).
 *  - Ranking: estimate descending, then key ascending.
 */
#ifndef HALOSKETCH_H
#define HALOSKETCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hs_sketch hs_sketch; /* opaque, owned by the library */

typedef enum {
    HS_OK = 0,
    HS_ERR_ARG = 1,        /* invalid argument: null pointer, bad size or range   */
    HS_ERR_CUDA = 2,       /* a CUDA runtime call or kernel launch failed          */
    HS_ERR_OOM = 3,        /* device or host allocation failed                     */
    HS_ERR_TABLE_FULL = 4, /* a bounded-probe hash table ran out of probes         */
    HS_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up                   */
    HS_ERR_STATE = 6       /* handle in a state that does not allow the call       */
} hs_status;

/* Flags of hs_params.  The full search picks, per pass, the cheaper of two
 * exact methods - scanning every cell with a shared-memory filter, or
 * enumerating the cells of hot buckets through a directory of mesh lines;
 * these flags force one (for testing; both give the same result). */
#define HS_FLAG_SEARCH_SCAN 1u
#define HS_FLAG_SEARCH_DIRECTORY 2u
/* The update adds each kept particle's t counter increments either directly
 * with global atomics or, for large calls, by binning them and accumulating
 * each bin in shared memory (the bins are drained into the counters before
 * any read of the counters); these flags force one (same counters). */
#define HS_FLAG_UPDATE_DIRECT 4u
#define HS_FLAG_UPDATE_BINNED 8u
/* The directory of mesh lines keeps each slot's first records inline beside
 * its offset when that saves a dependent read (large directories with about
 * two lines per slot); this flag keeps them for every mesh (for testing; same
 * result). */
#define HS_FLAG_DIR_INLINE 16u

/* Sketch parameters.  rows in [1, 32]; log2_width in [1, 30]; box > 0 and
 * cell > 0 with 1 <= round(box / cell) <= 2^21; flags: 0, or at most one
 * HS_FLAG_SEARCH_* and at most one HS_FLAG_UPDATE_* value, plus optionally
 * HS_FLAG_DIR_INLINE. */
typedef struct {
    uint32_t rows;        /* t: number of independent rows (Sec. 2.2)         */
    uint32_t log2_width;  /* b = W = 2^log2_width counters per row            */
    double box;           /* side of the periodic simulation box              */
    double cell;          /* mesh cell size (Sec. 2.1)                         */
    uint64_t hash_seed;   /* seeds the row hash functions                     */
    uint64_t sample_seed; /* seeds the sampling hash                          */
    uint32_t flags;       /* HS_FLAG_* bits (0 = automatic choices)           */
    uint32_t reserved;    /* must be 0                                        */
} hs_params;

/* Read-only description of a handle. */
typedef struct {
    uint32_t rows;
    uint32_t log2_width;
    uint32_t grid;        /* G                                               */
    float inv_cell;
    uint64_t width;       /* W                                               */
    uint64_t n_cells;     /* G^3, the size of the dictionary                 */
    uint64_t n_seen;      /* particles passed to sketch_update so far        */
} hs_info;

/* Counters kept by the library for benchmarking. */
typedef struct {
    uint64_t kernel_launches;   /* every kernel this handle launched          */
    uint64_t update_launches;   /* launches of the update kernel              */
    double update_ms;           /* summed device time of update launches       */
    uint64_t search_launches;   /* launches of the full-search kernel          */
    double search_ms;           /* summed device time of full-search launches  */
    double topk_ms;             /* summed device time of whole top-k queries   */
    uint64_t topk_calls;
    uint64_t last_candidates;   /* candidates collected by the last query      */
    int32_t last_threshold;     /* pruning threshold of the last query's pass  */
    uint32_t last_passes;       /* full-search passes of the last query        */
    uint64_t flush_launches;    /* launches accumulating binned increments     */
    double flush_ms;            /* their summed device time (part of update_ms)*/
    uint64_t h2d_bytes;         /* bytes staged from host buffers              */
    double h2d_ms;              /* summed device time of those copies          */
    uint64_t host_path_volumes; /* batch: volumes the last top-k answered one by
                                   one instead of in its single graph           */
} hs_stats;

/*
 * Initialization (Algorithm 1): allocate a t x W matrix of int32 counters
 * filled with zeros on the current CUDA device and bind the handle to
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * HS_ERR_ARG for invalid parameters or out == NULL; HS_ERR_OOM if device
 * memory is short.  *out is set only on success.
 */
hs_status sketch_create(const hs_params *params, void *cuda_stream, hs_sketch **out);

/*
 * Processing the stream (Algorithm 1; per item: Add of Sec. 2.2 after the mesh
 * reduction of Sec. 2.1 and the sampling of Sec. 3.1).  Adds n particles
 * (xyz, 3n floats) with global indices n_seen .. n_seen + n - 1, then
 * n_seen += n.  sample_rate in (0, 1]; rate 1 keeps every particle.
 * Device xyz: asynchronous on the handle's stream; the buffer must stay valid
 * until that work completes.  Page-locked host xyz (cudaHostAlloc,
 * cudaHostRegister) of a sketch without a hierarchy: read by the update
 * kernels over the host link directly, asynchronous like device memory.  Other
 * host xyz: copied in chunks through the library's staging buffers (three
 * device buffers of 2^24 particles: copies on the handle's own copy stream run
 * ahead of the updates of earlier pieces); the call returns after the last
 * copy is issued (pageable memory may be reused on return; page-locked memory
 * after sketch_wait_copies).  n == 0 is a no-op.
 * HS_ERR_ARG for a null handle, a null xyz with n > 0, or a rate outside (0, 1].
 */
hs_status sketch_update(hs_sketch *h, const float *xyz, uint64_t n, double sample_rate);

/*
 * Count Sketch Hierarchical (Algorithm 3, CSHi; the paper's "GPU hierarchy"):
 * a second sketch M1 of 2^super_log2_width counters per row (same rows and
 * sample seed, hash seed + 1) counts super-items, the super_factor^3 blocks of
 * cells, at every sketch_update; topk_extract then finds the c_mult * k best
 * super-items by M1's full search and ranks the cells inside them by this
 * sketch (M2), so the query costs c_mult * k * super_factor^3 estimates
 * instead of G^3.  Needs a fresh plain sketch (nothing added, no router), a
 * mesh G < 2^16 divisible by super_factor in [2, 64].  Point queries, counters
 * and merges of M2 are unchanged; reset, seek, flush and merge act on both.
 */
hs_status sketch_set_hierarchy(hs_sketch *h, uint32_t super_factor, uint32_t super_log2_width,
                               uint32_t c_mult);
/* M1 of a hierarchical sketch (NULL without a hierarchy); owned by h. */
hs_status sketch_super(hs_sketch *h, hs_sketch **out);

/*
 * Packed particle records (the data layout of the paper's evaluation, Sec. 4:
 * 64 bits hold the three coordinates of one particle).  Each coordinate is
 * q = floor(fl32(x * fl32(2^21 / box))) reduced periodically into [0, 2^21)
 * (the mesh reduction of Sec. 2.1 on a 2^21-cell mesh); x in bits 0-20, y in
 * 21-41, z in 42-62; bit 63 set marks coordinates that were not finite (the
 * record is skipped).  On the sketch's mesh of G cells per axis the record's
 * cell is (q * G) >> 21 per axis, which can differ by one cell from the cell of
 * the float32 position for particles within box / 2^21 of a cell boundary.
 *
 * pack_positions writes n records for n float32 xyz triples (device arrays;
 * asynchronous on cuda_stream).  sketch_update_packed is sketch_update for
 * records (8 bytes a particle instead of 12; host or device; plain and
 * hierarchical sketches, HS_ERR_ARG for a learned sketch).
 */
hs_status pack_positions(const float *xyz, uint64_t n, double box, void *cuda_stream,
                         uint64_t *records);
hs_status sketch_update_packed(hs_sketch *h, const uint64_t *records, uint64_t n,
                               double sample_rate);

/* Block until every host -> device copy issued by sketch_update has completed,
 * so the host buffers may be reused, without waiting for the updates (an
 * out-of-core stream refills one pinned chunk while the GPU consumes another). */
hs_status sketch_wait_copies(hs_sketch *h);

/*
 * Estimate (Sec. 2.2) for m cell keys: est[i] = median over rows of
 * sign_r(keys[i]) * C[r][bucket_r(keys[i])].  keys and est may each be host or
 * device memory.  Synchronous: returns once est is written.  A key >= G^3
 * gives HS_ERR_ARG (its est entry is 0; the others are still written).
 */
hs_status sketch_query(hs_sketch *h, const uint64_t *keys, uint64_t m, int32_t *est);

/*
 * Querying the data structure of Count Sketch with Full Search (Algorithm 1,
 * the "GPU without heap" design of Sec. 3.1): estimate every cell of the
 * dictionary [0, G^3) and return the min(k, G^3) best by (estimate desc,
 * key asc).  keys (uint64) and est (int32) receive *n_out entries in rank
 * order; they are HOST arrays of at least k entries.  Synchronous.  The result
 * is exactly that of enumerating every cell (the search prunes only cells
 * that provably cannot reach the k-th estimate).  HS_ERR_ARG for k == 0 or
 * null pointers.
 */
hs_status topk_extract(hs_sketch *h, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out);

/* Free the counters, scratch and staging buffers of h (NULL is a no-op). */
hs_status sketch_destroy(hs_sketch *h);

/* ---- extensions ---- */

/* Set the global index of the next particle (a shard of a longer stream that
 * starts at particle number n_seen keeps its sampling decisions; Sec. 5's sum of
 * sketches then reproduces the whole stream's sketch).  Counters are kept. */
hs_status sketch_seek(hs_sketch *h, uint64_t n_seen);

/* Zero the counters and n_seen (asynchronous on the handle's stream). */
hs_status sketch_reset(hs_sketch *h);

/* Copy the t x W counters (row-major, int32) to out (host or device); synchronous. */
hs_status sketch_counters(hs_sketch *h, int32_t *out);

/* Replace the counters with t x W int32 values from in (host or device); synchronous.
 * n_seen is unchanged. */
hs_status sketch_load_counters(hs_sketch *h, const int32_t *in);

/* Sketches built with the same parameters sum to the sketch of the union of
 * their streams (Sec. 5): dst.C += src.C element-wise (int32 wrap-around) and
 * dst.n_seen += src.n_seen.  HS_ERR_ARG if the parameters differ.  Ordered on
 * dst's stream after src's pending work. */
hs_status sketch_merge(hs_sketch *dst, hs_sketch *src);

/* Describe h. */
hs_status sketch_info(const hs_sketch *h, hs_info *out);

/* Apply binned, not yet accumulated increments to the counters (asynchronous
 * on the handle's stream).  Every call that reads the counters does this
 * itself; it is exposed so a caller can time the whole update. */
hs_status sketch_flush(hs_sketch *h);

/* Block until the handle's stream has finished its work. */
hs_status sketch_synchronize(hs_sketch *h);

/* Read (and with reset != 0, clear) the handle's benchmarking counters;
 * synchronises the handle's stream first. */
hs_status sketch_stats(hs_sketch *h, hs_stats *out, int reset);

/* Benchmark aid with no counterpart in the paper: the rate (operations per
 * second) of random 32-bit atomic adds into a fresh device table of n_counters
 * (a power of two) counters, total_ops adds in one launch.  This is the
 * second roofline of the update (besides the particle stream's HBM bytes):
 * t adds per kept particle resolve in L2.  Allocates and frees its table. */
hs_status hs_measure_red_rate(uint64_t n_counters, uint64_t total_ops, double *ops_per_s);

/*
 * Point queries that allocate nothing.  No counterpart in the paper: this is
 * for callers that cannot call cudaMalloc when they query - processes whose
 * device memory belongs to another allocator or is held to a fixed budget,
 * and query loops that must not pay for an allocation (a cudaMalloc may
 * synchronise the device).  Same results as sketch_query (keys and est host
 * or device arrays, in any combination; a key >= G^3 gives HS_ERR_ARG with
 * its est entry 0), through the same estimate kernel, but every temporary
 * lives in one static device array of the library, sized for
 * HS_NOALLOC_QUERY_MAX keys (about 3 MiB, held on every GPU that loads the
 * library until the process exits).  m > HS_NOALLOC_QUERY_MAX gives
 * HS_ERR_ARG: split the query.  The sketch's device must be current.
 * The call is synchronous: it waits on the handle's stream to read back the
 * bad-key flag (and est, for a host array).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress), which may load the
 * library's device code.  All calls share the array, which keeps the previous
 * call's contents (the call clears its own flag); calls that overlap on the
 * GPU - from several host threads or handles - race on it.  Pending binned
 * increments are applied first, as by every reader.
 */
#define HS_NOALLOC_QUERY_MAX 262144u
hs_status sketch_query_noalloc(hs_sketch *h, const uint64_t *keys, uint64_t m, int32_t *est);

/* ---- batches of independent sub-volumes (many small snapshots or sub-boxes) ----
 *
 * A batch holds n_volumes independent Count Sketches with the same rows, width
 * and hash seeds; volume v has its own box (boxes[v], mesh G_v =
 * round(boxes[v] / cell) <= 65535), its own particle stream (global indices
 * from 0 per volume; sample_seed shared) and its own top-k.  batch_update
 * processes the particles of all volumes, concatenated in one DEVICE buffer
 * with volume v at particles [offsets[v], offsets[v+1]) (offsets: host array of
 * n_volumes+1 entries, offsets[0] = 0), in one persistent scatter launch and one
 * accumulation launch, replayed as a CUDA graph while xyz, the total count and
 * the rate stay the same.  Every call is Add (Sec. 2.2) per particle of every
 * volume; results equal n_volumes separate sketches.  The batch's stream must
 * not be the legacy default stream (NULL creates a private stream).
 */
typedef struct hs_batch hs_batch;

/* Scatter configuration chosen by batch_autotune. */
typedef struct {
    uint32_t rounds;         /* tiles of 3072 particles staged between flushes    */
    uint32_t slot;           /* shared-memory ring depth (codes per bin)          */
    uint32_t configs_tried;  /* 0: the process's earlier choice for this shape    */
    float best_ms;           /* its time for the tuning data                      */
    uint32_t window_volumes; /* consecutive volumes whose bins have rings         */
} hs_tune;

/* params: rows, log2_width, cell, hash_seed, sample_seed, flags as for
 * sketch_create (params->box is ignored; boxes[v] gives each volume's box). */
hs_status batch_create(const hs_params *params, uint32_t n_volumes, const double *boxes,
                       void *cuda_stream, hs_batch **out);
hs_status batch_update(hs_batch *b, const float *xyz, const uint64_t *offsets, double sample_rate);
/* Top-k of every volume (Algorithm 1 per volume): volume v's min(k, G_v^3)
 * entries go to keys/est[v*k ...] (HOST arrays of n_volumes*k), their number to
 * n_out[v], ranked (estimate desc, key asc) as topk_extract ranks them.
 * Synchronous.  With k <= 4096 every volume is searched on the device in one
 * captured graph (replayed while k stays the same; the per-volume directories
 * are built on the first call); a volume outside its fixed capacities (fewer
 * distinct probe cells than k, too many hot buckets or candidates) is answered
 * by the per-volume search instead, counted in hs_stats.host_path_volumes.
 * HS_FLAG_SEARCH_SCAN sends every volume to the per-volume search. */
hs_status batch_topk(hs_batch *b, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out);
/* Counters of one volume (rows x W int32, host or device out); synchronous. */
hs_status batch_counters(hs_batch *b, uint32_t volume, int32_t *out);
hs_status batch_reset(hs_batch *b);
hs_status batch_volume_info(const hs_batch *b, uint32_t volume, hs_info *out);
hs_status batch_stats(hs_batch *b, hs_stats *out, int reset);
/* Time the scatter's ring window and depth (the widest window whose rings
 * hold a tile's codes; a window of one volume with its deepest ring, a half and
 * a quarter of it) on the given particles and
 * keep the fastest for later updates.  The tuning runs update the sketches, so
 * the batch is reset afterwards.  The choice is kept for the process, keyed by
 * (device, log2_width, rows, sample_rate): a later call for the same shape
 * applies it without running (configs_tried = 0) and leaves the batch as it is. */
hs_status batch_autotune(hs_batch *b, const float *xyz, const uint64_t *offsets,
                         double sample_rate, hs_tune *out);
hs_status batch_destroy(hs_batch *b);

/* ---- learned router (an addition to the paper's method) ----
 *
 * A small MLP predicts, from coarse-mesh densities, which coarse cells hold
 * heavy fine cells; the fine cells of those coarse cells are counted exactly
 * (the exact algorithm of Sec. 4.2 restricted to them) and every other
 * particle goes to the Count Sketch (Sec. 2.2).  The top-k merges the exact
 * counts with the sketch's full search over the cells that are not routed.
 *
 * MLP: 27 -> 64 -> 64 -> 1 with ReLU; HS_MLP_PARAMS float32 parameters in the
 * order w1[64][27], b1[64], w2[64][64], b2[64], w3[64], b3.  The forward pass
 * rounds weights, biases, inputs and hidden activations to bf16 and
 * accumulates each neuron as a float32 fused multiply-add chain over its
 * inputs in index order, starting from the bias.  Features are bf16 bit
 * patterns, 27 per sample.  Loss: weighted binary cross-entropy on the logit,
 * sum(w (softplus(z) - y z)) / sum(w).
 */
#define HS_MLP_PARAMS 6017
typedef struct hs_mlp hs_mlp;
hs_status mlp_create(uint64_t seed, void *cuda_stream, hs_mlp **out);
hs_status mlp_set_params(hs_mlp *m, const float *params);   /* host or device; resets Adam */
hs_status mlp_get_params(hs_mlp *m, float *params);
/* logits[i] of features[i*27 .. i*27+26]; arrays host or device; synchronous */
hs_status mlp_forward(hs_mlp *m, const uint16_t *features, uint64_t n, float *logits);
/* summed (not averaged) gradient of sum(w (softplus(z) - y z)) and that loss;
 * grad: HS_MLP_PARAMS floats.  The bf16 roundings pass gradients unchanged.
 * Every sum runs in a fixed order (per block of 128 samples, then over the
 * blocks in order), so equal inputs give equal gradients bit for bit and a
 * training run repeats exactly. */
hs_status mlp_gradient(hs_mlp *m, const uint16_t *features, const float *y, const float *w,
                       uint64_t n, float *grad, float *loss);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on the weight-averaged loss;
 * *loss (if not NULL) receives that average. */
hs_status mlp_train_step(hs_mlp *m, const uint16_t *features, const float *y, const float *w,
                         uint64_t n, float lr, float *loss);
hs_status mlp_destroy(hs_mlp *m);

/* ---- exact counts (Sec. 4.2, the exact algorithm) ----
 *
 * One counter per occupied cell of the box/cell mesh, in an open-addressing
 * table of 2^log2_slots (uint64 key, int32 count) entries in device memory
 * (12 bytes a slot; linear probing from a 64-bit mix of the key, at most 64
 * slots per key).  The reads below fail with HS_ERR_TABLE_FULL when some key
 * found no free slot (size the table about 2x the distinct cells or more).
 * Used as the ground truth of top-k recall and for the router's training labels.
 * All calls are ordered on cuda_stream; the reads are synchronous. */
typedef struct hs_exact hs_exact;
hs_status exact_create(double box, double cell, uint32_t log2_slots, void *cuda_stream,
                       hs_exact **out);
/* count n particles (device xyz; cells as in sketch_update, invalid ones skipped) */
hs_status exact_add(hs_exact *E, const float *xyz, uint64_t n);
/* up to cap (key, count) pairs in table order (host or device); *n_out = distinct
 * cells; cap 0: count only */
hs_status exact_list(hs_exact *E, uint64_t *keys, int32_t *counts, uint64_t cap, uint64_t *n_out);
/* the min(k, distinct) heaviest cells ranked by (count desc, key asc) */
hs_status exact_topk(hs_exact *E, uint32_t k, uint64_t *keys, int32_t *counts, uint32_t *n_out);
/* counts[i] = exact count of keys[i] (0 if never seen); host or device arrays */
hs_status exact_query(hs_exact *E, const uint64_t *keys, uint64_t m, int32_t *counts);
hs_status exact_reset(hs_exact *E);
hs_status exact_destroy(hs_exact *E);
/* one-shot: exact_create + exact_add + exact_list + exact_destroy */
hs_status exact_counts(const float *xyz, uint64_t n, double box, double cell, uint32_t log2_slots,
                       void *cuda_stream, uint64_t *keys, int32_t *counts, uint64_t cap,
                       uint64_t *n_out);

/* Learned sketch: params describe the sketch of the cells that are not routed;
 * coarse cells are R x R x R fine cells (R = coarse_factor, 1..64; the mesh must
 * be a multiple of R and below 2^16).  The exact part has the memory of an
 * open-addressing table of 2^table_log2 slots of (uint64 key, int32 count),
 * 12 * 2^table_log2 bytes, held as dense blocks of R^3 int32 counters, one per
 * routed coarse cell: at most B = floor(3 * 2^table_log2 / R^3) coarse cells are
 * routed, so the exact part never overflows.  The features use a sample of the
 * particles kept with probability feature_rate by a splitmix64 index hash
 * seeded with feature_seed (indices 0.. of the particles given to
 * learned_prepare). */
typedef struct hs_learned hs_learned;
hs_status learned_create(const hs_params *params, uint32_t coarse_factor, uint32_t table_log2,
                         uint64_t feature_seed, double feature_rate, void *cuda_stream,
                         hs_learned **out);
/* B and the bytes of the dense blocks (either pointer may be NULL) */
hs_status learned_capacity(hs_learned *L, uint64_t *max_routed, uint64_t *table_bytes);
/* Sample pass -> coarse counts -> 27 features of every coarse cell with a
 * sample: bf16(float(log10(1 + count))) of the cell and its 26 periodic
 * neighbours, neighbour (dx, dy, dz) at index (dz+1)*9 + (dy+1)*3 + (dx+1) ->
 * MLP -> a coarse cell is routed iff its logit > 0 and it is among the B cells
 * of largest logit (ties: smaller coarse key first).  xyz host or device (host
 * memory goes through the sketch's staging buffers).  Zeroes the exact
 * counters; call it before the updates (a fresh or reset sketch).
 * learned_prepare(xyz, n) = learned_sample(xyz, n) + learned_route. */
hs_status learned_prepare(hs_learned *L, const float *xyz, uint64_t n, hs_mlp *mlp,
                          uint64_t *n_routed);
/* The sample pass in pieces (an out-of-core stream): each call adds the
 * sampled particles of xyz[0, n) to the coarse counts, their indices following
 * those of the previous calls since the last learned_route. */
hs_status learned_sample(hs_learned *L, const float *xyz, uint64_t n);
/* Features, MLP and routing from the coarse counts of the learned_sample
 * calls so far (then the next learned_sample starts new counts). */
hs_status learned_route(hs_learned *L, hs_mlp *mlp, uint64_t *n_routed);
/* Each kept particle of a routed coarse cell increments its fine cell's exact
 * count; every other kept particle is added to the sketch (sketch_update). */
hs_status learned_update(hs_learned *L, const float *xyz, uint64_t n, double sample_rate);
/* The k best of: sketch estimates of cells that are not routed (full search,
 * Algorithm 1, or the hierarchical query when sketch_set_hierarchy was called
 * on learned_sketch before learned_prepare) and exact counts of the fine cells
 * of routed coarse cells with a particle; ranked by (value desc, key asc);
 * HOST outputs. */
hs_status learned_topk(hs_learned *L, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out);
/* the non-zero exact counts (fine key, count), in block order; cap 0: count only */
hs_status learned_table(hs_learned *L, uint64_t *keys, int32_t *counts, uint64_t cap,
                        uint64_t *n_out);
/* the routed coarse keys, ascending */
hs_status learned_routed(hs_learned *L, uint64_t *coarse_keys, uint64_t cap, uint64_t *n_out);
/* the coarse cells with a sample (keys) and their logits, in list order */
hs_status learned_logits(hs_learned *L, uint64_t *coarse_keys, float *logits, uint64_t cap,
                         uint64_t *n_out);
hs_status learned_features(hs_learned *L, uint16_t *features, uint64_t cap, uint64_t *n_out);
hs_status learned_coarse_counts(hs_learned *L, int32_t *out);
hs_status learned_sketch(hs_learned *L, hs_sketch **out);
/* zero the sketch and the exact counters (the routing is kept) */
hs_status learned_reset(hs_learned *L);
hs_status learned_destroy(hs_learned *L);

/* Message of the calling thread's last failed call ("" if none). */
const char *hs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HALOSKETCH_H */
