// hs_kernels.h - host-side launchers of the library's kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hs_device.cuh"

namespace hs {

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`, calling the runtime only when the limit grows (launch paths
// run this before every launch; cudaFuncSetAttribute itself is not free).
cudaError_t ensure_smem_limit(const void *kernel, size_t bytes);
template <typename K>
inline cudaError_t ensure_smem_limit(K *kernel, size_t bytes) {
    return ensure_smem_limit(reinterpret_cast<const void *>(kernel), bytes);
}

// ---- update mode (k_update.cu) ----
cudaError_t launch_update(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                          int32_t *C, double rate, uint64_t sample_seed, uint64_t *probe,
                          uint64_t probe_base, uint64_t probe_cap, uint32_t band_lo,
                          uint32_t band_hi, int max_blocks,
                          cudaStream_t s);
// ---- update mode with shared-memory accumulation (k_binned.cu) ----
// One sub-volume of a batch: particles [start, next start) of the concatenated
// buffer, its own stream index g0, mesh (G, inv_cell) and first bin.
struct VolumeDesc {
    uint64_t start;
    uint64_t g0;
    uint64_t probe_base;
    float inv_cell;
    uint32_t G;
    uint32_t bin0;
    uint32_t pad;
};
// Shared-memory layout of the binned scatter: per bin a ring of `slot` 16-bit
// codes in two halves, flushed a half at a time between block barriers;
// per-warp queues of kept cells for sampled calls.
struct BinLayout {
    uint32_t S;        // log2 counters per bin
    uint32_t nbins;    // rows * W / 2^S
    uint32_t slot;     // ring entries per bin (0: binning unavailable)
    uint32_t half;     // flush granule in entries (slot / 2, a multiple of 8)
    uint32_t rows_per_pass;   // rows one scatter launch stages (all: one pass)
    size_t smem;       // dynamic shared memory of the scatter kernel (no queues)
};
// single_pass: every row in one launch or not at all (batches: a volume's bins
// are offset within one launch)
BinLayout bin_layout(const SketchDesc &d, size_t smem_budget, bool single_pass = false);
constexpr uint32_t kMaxBinGroups = 128;
constexpr uint32_t kScatterTile = 3072;   // particles of one scatter tile (768 threads x 4)
// Global side of the binned update.  Each scatter block owns one region per
// bin.  Bins come in groups of bpg bins whose regions have the same capacity
// (one group for a sketch, one per volume for a batch): region (bin j, block b)
// of group g = j / bpg starts at code gbase[g] + (b bpg + j - g bpg) gcap[g],
// so a block writes into one span of the group.  fill[j * nblocks + b]
// codes of it are written (whole halves; the unused entries of a last,
// partial half hold pairs of codes that cancel).
struct BinStore {
    uint16_t *codes;
    uint32_t *fill;            // per (bin, block), codes written since the last accumulation
    const uint64_t *gbase;     // per group
    const uint32_t *gcap;      // per group: codes per region (a multiple of 16)
    uint32_t nblocks;          // scatter blocks (regions per bin)
    uint32_t bpg;              // bins per group
    uint32_t ngroups;          // <= kMaxBinGroups
};
// where routed particles go: one dense block of R^3 int32 counters per routed
// coarse cell, blocks in coarse-key order; the block of routed cell ck is
// prefix[ck / 32] + (number of routed cells below ck in its bitmap word)
struct RouteTarget {
    RouteFilter filter;
    const uint32_t *prefix;   // exclusive prefix count of routed cells per bitmap word
    int32_t *blocks;
};
// xyz: float32 positions, or 64-bit packed records when packed != 0 (plain and
// super-item sketches only).  Launches B.nblocks blocks.  rounds: tiles of
// 3072 particles a block stages between flush phases (0: chosen from the rate);
// slot: ring depth (0: the largest that fits shared memory).
cudaError_t launch_bin_scatter(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                               int32_t *C, double rate, uint64_t sample_seed, uint64_t *probe,
                               uint64_t probe_base, uint64_t probe_cap, const BinLayout &L,
                               const BinStore &B, cudaStream_t s,
                               const VolumeDesc *vols = nullptr, uint32_t nvol = 0,
                               uint32_t probe_per_vol = 0, const RouteTarget *route = nullptr,
                               int packed = 0, uint32_t rounds = 0, uint32_t slot = 0,
                               uint32_t *tile_vols = nullptr,
                               const unsigned long long *n_dev = nullptr, uint64_t n_base = 0,
                               uint32_t wvols_cap = 0);
// packed: 0 float32 xyz, 1 packed position records, 2 cell records (from
// launch_compact_cells; n is then a bound and the launch takes the records
// [n_base, min(n_base + n, *n_dev)) of the buffer starting n_base before xyz)
// Rings of a batch's scatter: the bins of a window of `wvols` consecutive
// volumes (a power of two) have rings of `slot` entries; tiles holding
// particles of later volumes move the window.  slot_cap: 0 or a smaller ring;
// wvols_cap: 0 (4) or a smaller window.
struct BatchRing {
    uint32_t wvols, nslots, slot;
};
BatchRing batch_ring(const BinLayout &L, const SketchDesc &d, uint32_t ngroups, double rate,
                     uint32_t slot_cap, uint32_t wvols_cap = 0);
// Compaction of a stream piece for several passes over it: every particle is
// sampled (index g0 + i) and quantised once on d's mesh (d.F == 1; packed:
// xyz holds packed position records, decoded as the packed scatter does); the
// cells of kept, valid particles are appended to `cells` (cx | cy << 21 |
// cz << 42, in no particular order) and counted in *count (reset by the
// caller).  The probes of the sketch (probe, G) and of its super-item sketch
// (sprobe, mesh G / F) record every particle of their windows [base, end).
struct CompactProbe {
    uint64_t *probe;
    uint64_t base, end;
    uint32_t F;            // 1: the fine mesh; > 1: blocks of F^3 cells
    uint32_t fmagic;       // ceil(2^32 / F)
    uint32_t G;            // mesh of the keys
};
cudaError_t launch_compact_cells(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                                 double rate, uint64_t sample_seed, const CompactProbe &p0,
                                 const CompactProbe &p1, uint64_t *cells,
                                 unsigned long long *count, int blocks, cudaStream_t s,
                                 int packed = 0);
// C[bin range] += the codes of every region, then fill = 0
cudaError_t launch_bin_accumulate(const BinLayout &L, const BinStore &B, int32_t *C,
                                  cudaStream_t s);

// ---- learned router (k_learned.cu) ----
cudaError_t launch_coarse_hist(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                               uint32_t R, uint32_t Gc, uint64_t seed, double rate,
                               int32_t *counts, cudaStream_t s);
cudaError_t launch_coarse_list(const int32_t *counts, uint64_t ncoarse, uint64_t *list,
                               unsigned long long *n_list, uint64_t cap, cudaStream_t s);
cudaError_t launch_features(const int32_t *counts, uint32_t Gc, const uint64_t *list, uint64_t m,
                            const uint16_t *ftab, uint32_t ftab_n, uint16_t *feats,
                            cudaStream_t s);
cudaError_t launch_mlp_forward(const float *P, const uint16_t *feats, uint64_t m, float *logits,
                               cudaStream_t s);
// grad = summed gradient, loss[0] = sum w * bce, loss[1] = sum w, each summed in a
// fixed order (reproducible); part: mlp_grad_scratch_floats(m) floats of scratch
size_t mlp_grad_scratch_floats(uint64_t m);
cudaError_t launch_mlp_grad(const float *P, const uint16_t *feats, const float *y, const float *w,
                            uint64_t m, float *grad, float *loss, float *part, cudaStream_t s);
cudaError_t launch_adam(float *P, float *M, float *V, const float *grad, const float *gscale,
                        float lr, int step, cudaStream_t s);
cudaError_t launch_logit_rank(const float *logits, uint64_t m, int32_t *rank,
                              unsigned long long *n_pos, cudaStream_t s);
struct SelectState;
cudaError_t launch_route(const uint64_t *list, const int32_t *rank, uint64_t m,
                         const SelectState *sel, int use_sel, uint32_t *bits, cudaStream_t s);
cudaError_t launch_exclusive_scan(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *scratch,
                                  cudaStream_t s, int *launches);
cudaError_t launch_word_popc(const uint32_t *bits, uint64_t words, uint32_t *out, cudaStream_t s);
cudaError_t launch_route_list(const uint64_t *list, uint64_t m, const uint32_t *bits,
                              const uint32_t *prefix, uint64_t *rlist, cudaStream_t s);
cudaError_t launch_block_list(const int32_t *blocks, const uint64_t *rlist, uint64_t nblocks,
                              uint32_t R, uint32_t Gc, uint32_t G, uint64_t *out_keys,
                              int32_t *out_counts, unsigned long long *n_out, uint64_t cap,
                              cudaStream_t s);
cudaError_t launch_exact_count(const float *xyz, uint64_t n, const SketchDesc &d,
                               unsigned long long *keys, int32_t *counts, uint64_t slots,
                               uint32_t *overflow, cudaStream_t s);
cudaError_t launch_table_list(const unsigned long long *keys, const int32_t *counts, uint64_t slots,
                              uint64_t *out_keys, int32_t *out_counts, unsigned long long *n_out,
                              uint64_t cap, cudaStream_t s);
cudaError_t launch_exact_query(const unsigned long long *tkeys, const int32_t *tcounts,
                               uint64_t slots, const uint64_t *keys, uint64_t m, int32_t *counts,
                               cudaStream_t s);

// dst[i] += src[i] (int32 wrap-around), the merge of two sketches
cudaError_t launch_update_packed(const uint64_t *rec, uint64_t n, uint64_t g0,
                                 const SketchDesc &d, int32_t *C, double rate,
                                 uint64_t sample_seed, uint64_t *probe, uint64_t probe_base,
                                 uint64_t probe_cap, int max_blocks, cudaStream_t s);
cudaError_t launch_pack(const float *xyz, uint64_t n, double box, uint64_t *out, cudaStream_t s);
cudaError_t launch_add_counters(int32_t *dst, const int32_t *src, uint64_t n, cudaStream_t s);
cudaError_t launch_red_rate(uint32_t *table, uint64_t n_counters, uint64_t ops_per_thread,
                            int blocks, cudaStream_t s);

// ---- estimate mode (k_search.cu) ----
enum SearchMode : uint32_t { kGE = 0, kGT = 1, kEQ = 2 };

struct SearchOut {
    uint64_t *key;
    int32_t *est;
    unsigned long long *count;   // entries appended (may exceed cap)
    uint64_t cap;
};

// bits per row of the hot-bucket bitmap that fits the shared-memory budget
uint32_t bitmap_log2_bits(uint32_t rows, uint32_t log2w, size_t smem_budget_bytes);
// bitmap[r][sb] = 1 iff some counter of super-bucket sb in row r has |C| >= theta_hot
cudaError_t launch_hot_bitmap(const int32_t *C, const SketchDesc &d, uint32_t nb,
                              int32_t theta_hot, uint32_t *bitmap, int max_blocks, cudaStream_t s);
// estimate every cell of lines [line_lo, line_hi) (line = cy + G*cz) and append
// the cells whose estimate passes (mode, theta)
cudaError_t launch_full_search(const int32_t *C, const SketchDesc &d, int32_t theta,
                               SearchMode mode, const uint32_t *bitmap, uint32_t nb, int prune,
                               uint64_t line_lo, uint64_t line_hi, SearchOut out, int blocks,
                               cudaStream_t s, RouteFilter skip = RouteFilter{nullptr, 0, 0, 0});
// est[i] = Estimate(keys[i]); keys >= G^3 give 0 and set *bad
// Second layer of the hierarchical query: estimate every cell of the ns listed
// super-items (F^3 cells each, super grid Gs per axis) and append those that
// pass theta with keys in [key_lo, key_hi) to out.
cudaError_t launch_expand(const int32_t *C, const SketchDesc &d, const uint64_t *skeys, uint64_t ns,
                          uint32_t F, uint32_t Gs, int32_t theta, SearchMode mode, uint64_t key_lo,
                          uint64_t key_hi, SearchOut out, int max_blocks, cudaStream_t s,
                          int *launches, RouteFilter skip = RouteFilter{nullptr, 0, 0, 0});
cudaError_t launch_point_query(const int32_t *C, const SketchDesc &d, const uint64_t *keys,
                               uint64_t m, int32_t *est, uint32_t *bad, cudaStream_t s);
// distinct valid keys of probe[0..m) via an open-addressing set of 2^log2_slots slots
cudaError_t launch_probe_distinct(const uint64_t *probe, uint64_t m, uint64_t *slots,
                                  uint32_t log2_slots, uint64_t *distinct,
                                  unsigned long long *n_distinct, uint32_t *overflow,
                                  cudaStream_t s);

// ---- output-sensitive full search (k_dir.cu) ----
// one mesh line of a row's directory: cy | cz << 16 (directories exist for
// G < 2^16 only); the line's value L is recomputed from it when queried
typedef uint32_t DirRecord;
// A row's directory lives in one allocation of dir_bytes(G, D): (2^D + 1)
// uint32 slot offsets, then (16-byte aligned) 2^D inline slots of up to 4
// records.  The inline slots save a dependent DRAM read when the directory is
// too large for L2 (G^2 >= 2^23 lines) and slots hold about 2 lines or fewer
// (G^2 <= 2^(D+1)), or always when forced; otherwise only the offsets are kept.
inline bool dir_has_inline(uint32_t G, uint32_t D, bool force) {
    const uint64_t lines = (uint64_t)G * G;
    return force || (lines >= (1ull << 23) && lines <= (2ull << D));
}
inline size_t dir_offsets_bytes(uint32_t D) { return (((size_t)1 << D) * 4 + 4 + 15) & ~(size_t)15; }
inline size_t dir_bytes(uint32_t G, uint32_t D, bool force) {
    return dir_offsets_bytes(D) + (dir_has_inline(G, D, force) ? ((size_t)16 << D) : 0);
}
inline const uint4 *dir_inline(const uint32_t *offsets, uint32_t D) {
    return reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(offsets) +
                                           dir_offsets_bytes(D));
}
inline uint4 *dir_inline(uint32_t *offsets, uint32_t D) {
    return reinterpret_cast<uint4 *>(reinterpret_cast<char *>(offsets) + dir_offsets_bytes(D));
}
// directory of the G^2 lines of row r bucketed by the top D bits of L, with
// inline slots when `inl` (dir_has_inline of the allocation)
cudaError_t launch_dir_build(const SketchDesc &d, int r, uint32_t D, bool inl, uint32_t *offsets,
                             uint32_t *cursor, DirRecord *rec, uint32_t *scan_scratch,
                             int max_blocks, cudaStream_t s, int *launches);
// signed hot maps of every row for threshold theta >= 1 (W >= 32): bits holds
// rows x W/32 words of the positive map (C >= theta), then of the negative
// map (C <= -theta)
cudaError_t launch_signed_bits(const int32_t *C, const SketchDesc &d, int32_t theta, uint32_t *bits,
                               int max_blocks, cudaStream_t s);
// row r's hot buckets from the signed maps, as bucket << 1 | sign bit
cudaError_t launch_hot_list(const uint32_t *bits, const SketchDesc &d, int r, uint32_t *list,
                            unsigned long long *count, uint64_t cap, int max_blocks,
                            cudaStream_t s);
// cells first hot in row r, with at least `need` hot rows and a passing
// estimate (hot: the row's signed count can reach theta: the signed maps);
// hot: row r's list from launch_hot_list
cudaError_t launch_dir_query(const int32_t *C, const SketchDesc &d, int r, uint32_t D, bool inl,
                             const uint32_t *offsets, const DirRecord *rec, const uint32_t *hot,
                             uint64_t n_hot, const uint32_t *bits, int32_t theta, SearchMode mode,
                             uint64_t line_lo, uint64_t line_hi, SearchOut out, int max_blocks,
                             cudaStream_t s, RouteFilter skip = RouteFilter{nullptr, 0, 0, 0});

// ---- top-k of a batch of sketches in one launch sequence (k_batch_topk.cu) ----
struct BatchTopkVol {     // one volume's query, filled by the host before each launch
    uint64_t m_probe;     // probe entries recorded (at most probe_per_vol)
    uint32_t G;           // mesh cells a side
    uint32_t kk;          // min(k, G^3)
    uint32_t use;         // 0: the host's general path answers this volume
    uint32_t D;           // its directories have 2^D slots (D >= log2 W: a
                          // bucket's lines are the records of a run of slots)
    uint64_t gmagic;      // div_magic(G): x / G as one high multiply
};
struct BatchTopkBufs {    // device buffers; per-volume arrays are volume-major
    const BatchTopkVol *vol;
    uint32_t nvol, F;     // F: rows enumerated by the directory search
    uint32_t k;           // output stride per volume
    uint32_t hot_cap;     // hot buckets listed per (volume, row)
    uint32_t cand_cap;    // candidates per volume
    uint32_t set_log2;    // probe set slots per volume = 2^set_log2
    uint64_t probe_per_vol;
    const uint64_t *probe;        // nvol x probe_per_vol probe keys
    unsigned long long *set;      // nvol x 2^set_log2
    uint64_t *dkey;               // distinct probe cells, nvol x probe_per_vol
    int32_t *dest;
    uint32_t *dcnt;               // nvol
    int32_t *theta;               // nvol
    uint32_t *status;             // nvol: 0, or why the host must answer the volume
    uint32_t *scan;               // nvol: 1 when the volume's cells are scanned
    uint32_t *bits;               // 2 x nvol x rows x W/32: positive, then negative hot maps
    uint32_t *hot;                // nvol x F x hot_cap
    uint32_t *hot_cnt;            // nvol x F
    unsigned long long *pre;      // nvol x F + 1 work prefix
    const uint32_t *const *dir_off;   // nvol x F directory slot offsets
    const DirRecord *const *dir_rec;  // nvol x F directory records
    uint64_t *ckey;               // nvol x cand_cap candidates
    int32_t *cest;
    uint32_t *ccnt;               // nvol
    uint64_t *okey;               // nvol x k results in rank order
    int32_t *oest;
    uint32_t *on;                 // nvol: results written
};
// counters C: nvol x rows x W int32 (W >= 32); every launch on stream s
cudaError_t launch_batch_topk(const int32_t *C, const SketchDesc &d, const BatchTopkBufs &b,
                              int num_sms, cudaStream_t s, int *launches);
size_t batch_topk_final_smem(uint32_t k);

// ---- ranking (k_select.cu) ----
struct SelectState {
    uint32_t hi;        // decided digits of the estimate part
    uint32_t pad;
    uint64_t lo;        // decided digits of the key part
    uint64_t k_rem;     // rank (1-based) still to find among matching entries
};

// Find the k-th best (estimate desc, key asc) entry of (key, est)[0..m) by a
// most-significant-digit radix select; leaves the threshold in *state.
// key_bits: keys are < 2^key_bits.  hist: 256 uint64 of scratch.
cudaError_t launch_select_kth(const uint64_t *key, const int32_t *est, uint64_t m, uint64_t k,
                              uint32_t key_bits, SelectState *state, unsigned long long *hist,
                              int blocks, cudaStream_t s, int *launches);
// Entries ranked at or above the threshold, written in rank order to
// out_key/out_est (exactly min(k, m) of them when the threshold came from
// launch_select_kth with the same k).  tmp_* hold min(k, m) entries of scratch
// (tmp_rank: min(k, m) uint32).
cudaError_t launch_take_sorted(const uint64_t *key, const int32_t *est, uint64_t m,
                               const SelectState *state, int all, uint64_t *tmp_key,
                               int32_t *tmp_est, unsigned long long *tmp_count, uint32_t *tmp_rank,
                               uint64_t n_take, uint64_t *out_key, int32_t *out_est, int blocks,
                               cudaStream_t s, int *launches);

}  // namespace hs
