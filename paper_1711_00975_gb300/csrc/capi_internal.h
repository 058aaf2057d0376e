// capi_internal.h - what the C ABI's translation units share: the sketch
// handle, error reporting, tuning constants and the internal steps of the
// update and the full search (defined in capi.cu).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/halosketch.h"
#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {
namespace capi {

// Record the calling thread's error message (hs_last_error) and return st.
hs_status fail(hs_status st, const char *fmt, ...);

#define HS_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? HS_ERR_OOM : HS_ERR_CUDA,        \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                         \
    } while (0)

// return st unless it is HS_OK
#define HS_TRY(call)                          \
    do {                                      \
        hs_status st_ = (call);               \
        if (st_ != HS_OK) return st_;         \
    } while (0)

constexpr uint64_t kProbeCap = 1ull << 20;        // keys of the first 2^20 particles
constexpr uint64_t kCellsMax = 1ull << 27;       // cell records buffered (1 GiB)
constexpr uint32_t kProbeSlotsLog2 = 21;
constexpr uint64_t kStageParticles = 1ull << 24;  // 192 MiB per staging buffer
constexpr int kStageBuffers = 3;                    // copies run ahead through a drain
constexpr size_t kSearchSmemBudget = 192 * 1024;
constexpr size_t kBinSmemBudget = 224 * 1024;
constexpr uint64_t kBinBudgetBytes = 16ull << 30;  // global code regions of one sketch, at most
constexpr double kBinnedMinUpdates = 1 << 20;      // smaller calls add directly
constexpr uint64_t kMaxScanCells = 1ull << 40;      // largest full scan one top-k may run
constexpr uint32_t kBatchViews = 8;                 // volumes whose top-k run concurrently
constexpr size_t kMaxPendingEvents = 256;           // timing pairs kept before folding

struct EventPair {
    cudaEvent_t a, b;
};

// Global code regions of a binned update (see BinStore) and their host-side
// sizes.
struct BinBuffers {
    uint16_t *codes = nullptr;
    uint32_t *fill = nullptr;
    uint64_t *gbase = nullptr;
    uint32_t *gcap = nullptr;
    uint32_t nblocks = 0, bpg = 0, ngroups = 0;
    uint32_t min_cap = 0;       // smallest region capacity
    BinStore store() const { return BinStore{codes, fill, gbase, gcap, nblocks, bpg, ngroups}; }
};

// Region capacity (codes, a multiple of 16) for `mean` expected codes per
// region: 8 % and 8 standard deviations of margin, plus `pad_halves` partial
// halves (one per launch) of `half` entries.
uint32_t region_capacity(double mean, uint32_t half, double pad_halves);
// Allocate regions for groups of bpg bins, group g's regions of caps[g] codes
// (multiples of 16), nblocks per bin; fills zeroed.
hs_status alloc_bins(BinBuffers &bb, const std::vector<uint32_t> &caps, uint32_t bpg,
                     uint32_t nblocks, cudaStream_t s);
void free_bins(BinBuffers &bb);

}  // namespace capi
}  // namespace hs

using namespace hs;
using namespace hs::capi;

struct hs_sketch {
    hs_params p;
    SketchDesc d;
    uint64_t n_cells = 0;
    uint32_t key_bits = 0;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    int32_t *C = nullptr;
    uint64_t *probe = nullptr;
    uint64_t probe_cap = kProbeCap;   // probe slots
    uint64_t probe_base = 0;    // global index of probe slot 0
    uint64_t n_seen = 0;

    // staging for host particle buffers
    float *stage[kStageBuffers] = {};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[kStageBuffers] = {};
    cudaEvent_t ev_free[kStageBuffers] = {};

    // top-k scratch
    uint64_t cap = 0;               // candidate capacity
    uint64_t min_cap = 0;           // extra candidates a learned top-k appends
    hs_sketch *super = nullptr;     // hierarchy: sketch of F^3 super-items (Algorithm 3)
    uint64_t *cells = nullptr;      // compaction: cells of a call's kept particles
    uint64_t cells_cap = 0;
    uint64_t cells_bound = 0;       // records appended at most (particles compacted)
    unsigned long long *cells_cnt = nullptr;
    uint32_t super_mult = 0;        // hierarchy: c of the top-(c*k) super-items
    uint64_t *cand_key = nullptr;
    int32_t *cand_est = nullptr;
    unsigned long long *counters = nullptr;   // [0] candidates, [1] tmp, [2] distinct
    uint32_t *flags = nullptr;                // [0] bad key, [1] probe overflow
    uint32_t *bitmap = nullptr;
    uint32_t nb = 0;
    uint64_t *slots = nullptr;
    uint64_t *distinct = nullptr;
    int32_t *distinct_est = nullptr;
    SelectState *sel = nullptr;
    unsigned long long *hist = nullptr;
    uint64_t *tmp_key = nullptr;
    int32_t *tmp_est = nullptr;
    uint32_t *tmp_rank = nullptr;
    uint64_t *out_key = nullptr;
    int32_t *out_est = nullptr;
    uint64_t out_cap = 0;
    uint64_t *q_keys = nullptr;
    int32_t *q_est = nullptr;
    uint64_t q_cap = 0;

    // output-sensitive search: exact hot bitmap, hot-bucket lists, and one
    // directory of mesh lines per enumerated row (kept across queries)
    uint32_t *xbits = nullptr;
    uint32_t *hot_list = nullptr;
    unsigned long long *hot_cnt = nullptr;
    uint64_t hot_cap = 0;
    uint32_t dir_D = 0;
    uint32_t *dir_off[kMaxRows] = {};
    DirRecord *dir_rec[kMaxRows] = {};
    uint32_t *dir_cursor = nullptr;
    uint32_t *scan_scratch = nullptr;
    bool dir_failed = false;
    uint32_t dir_G[kMaxRows] = {};        // mesh the directory of row r was built for
    uint64_t dir_lines_cap[kMaxRows] = {};
    bool is_view = false;                 // counters and probe belong to a batch
    bool routing = false;                 // learned router: routed cells go to a table
    RouteTarget route{};

    // binned update: codes waiting in the global regions until the next drain
    BinLayout bl{};
    BinBuffers bb;
    double pending = 0;          // expected codes per region since the last drain
    double pending_limit = 0;    // drain before the expected fill passes this

    // benchmarking
    hs_stats stats;
    std::vector<EventPair> pending_update, pending_search, pending_flush, pending_copy, pool;
};

namespace hs {
namespace capi {

bool is_device_ptr(const void *p);
const void *pinned_device_view(const void *p);
hs_status check_params(const hs_params *p);
hs_status take_events(hs_sketch *h, EventPair *out);
void drain_timings(hs_sketch *h);
hs_status check_ranked(const uint64_t *keys, const int32_t *est, uint64_t n);
void free_topk_scratch(hs_sketch *h);
hs_status ensure_topk_scratch(hs_sketch *h, uint64_t k);
void free_dir(hs_sketch *h);
uint32_t enum_rows(const hs_sketch *h);
hs_status ensure_dir_scratch(hs_sketch *h);
bool ensure_dir(hs_sketch *h, int r);
hs_status ensure_staging(hs_sketch *h);
hs_status ensure_query_scratch(hs_sketch *h, uint64_t m);
hs_status drain(hs_sketch *h);
hs_status discard_pending(hs_sketch *h);
bool want_binned(hs_sketch *h, uint64_t n, double rate);
hs_status ensure_bins(hs_sketch *h, uint64_t n, double rate, uint64_t launches = 1);
hs_status launch_update_timed(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                              double rate, bool packed = false);
hs_status launch_update_direct(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                               double rate, bool packed = false);
bool want_compact(hs_sketch *h, uint64_t n, double rate, bool packed);
hs_status update_piece(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0, double rate,
                       bool packed, bool compact, uint64_t call_n);
hs_status update_finish(hs_sketch *h, double rate);
hs_status search_pass_dir(hs_sketch *h, int32_t theta, SearchMode mode, int64_t hot,
                          uint64_t line_lo, uint64_t line_hi, SearchOut out, bool *used);
hs_status search_pass(hs_sketch *h, int32_t theta, SearchMode mode, uint64_t line_lo,
                      uint64_t line_hi, unsigned long long count_base,
                      unsigned long long *count_out);
hs_status kth_estimate(hs_sketch *h, const uint64_t *key, const int32_t *est, uint64_t m,
                       uint64_t k, int32_t *theta);
hs_status finalize(hs_sketch *h, uint64_t m, uint64_t k);

}  // namespace capi
}  // namespace hs
