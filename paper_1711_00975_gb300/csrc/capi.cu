// capi.cu - the library's C ABI (include/halosketch.h): handle lifetime, the
// update path (device buffers directly, host buffers through double-buffered
// staging), point queries and the exact full-search top-k.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/halosketch.h"
#include "hs_device.cuh"
#include "hs_kernels.h"

using namespace hs;

namespace {

thread_local std::string g_last_error;

hs_status fail(hs_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define HS_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? HS_ERR_OOM : HS_ERR_CUDA,        \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                         \
    } while (0)

constexpr uint64_t kProbeCap = 1ull << 20;        // keys of the first 2^20 particles
constexpr uint32_t kProbeSlotsLog2 = 21;
constexpr uint64_t kStageParticles = 1ull << 24;  // 192 MiB per staging buffer
constexpr int kStageBuffers = 3;                    // copies run ahead through a drain
constexpr size_t kSearchSmemBudget = 192 * 1024;
constexpr size_t kBinSmemBudget = 224 * 1024;
constexpr uint64_t kBinBudgetBytes = 4ull << 30;   // global bins, at most
constexpr double kBinnedMinUpdates = 1 << 20;      // smaller calls add directly
constexpr uint64_t kMaxScanCells = 1ull << 40;      // largest full scan one top-k may run
constexpr uint32_t kBatchViews = 8;                 // volumes whose top-k run concurrently

struct EventPair {
    cudaEvent_t a, b;
};

}  // namespace

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

    // binned update: codes waiting in global bins until the next drain
    BinLayout bl{};
    uint16_t *bins = nullptr;
    uint32_t *bin_cursor = nullptr;
    uint32_t bin_cap = 0;
    uint4 *carry = nullptr;         // scatter rings carried from one launch to the next
    bool carry_valid = false;
    double pending = 0;          // kept particles binned since the last drain
    double pending_limit = 0;    // drain before the expected bin load passes this

    // benchmarking
    hs_stats stats;
    std::vector<EventPair> pending_update, pending_search, pending_flush, pool;
};

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

hs_status check_params(const hs_params *p) {
    if (!p) return fail(HS_ERR_ARG, "params is NULL");
    if (p->rows < 1 || p->rows > (uint32_t)kMaxRows)
        return fail(HS_ERR_ARG, "rows=%u outside [1, %d]", p->rows, kMaxRows);
    if (p->log2_width < 1 || p->log2_width > 30)
        return fail(HS_ERR_ARG, "log2_width=%u outside [1, 30]", p->log2_width);
    if (!(p->box > 0) || !(p->cell > 0) || !std::isfinite(p->box) || !std::isfinite(p->cell))
        return fail(HS_ERR_ARG, "box and cell must be positive and finite");
    double g = std::llround(p->box / p->cell);
    if (g < 1 || g > (double)(1u << 21))
        return fail(HS_ERR_ARG, "grid round(box/cell)=%.0f outside [1, 2^21]", g);
    const uint32_t known = HS_FLAG_SEARCH_SCAN | HS_FLAG_SEARCH_DIRECTORY | HS_FLAG_UPDATE_DIRECT |
                           HS_FLAG_UPDATE_BINNED;
    if ((p->flags & ~known) != 0 || p->reserved != 0)
        return fail(HS_ERR_ARG, "unknown flags or reserved != 0");
    if ((p->flags & HS_FLAG_SEARCH_SCAN) && (p->flags & HS_FLAG_SEARCH_DIRECTORY))
        return fail(HS_ERR_ARG, "at most one search method may be forced");
    if ((p->flags & HS_FLAG_UPDATE_DIRECT) && (p->flags & HS_FLAG_UPDATE_BINNED))
        return fail(HS_ERR_ARG, "at most one update method may be forced");
    return HS_OK;
}

EventPair take_events(hs_sketch *h) {
    if (!h->pool.empty()) {
        EventPair e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    EventPair e{nullptr, nullptr};
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
    return e;
}

// fold finished event pairs into the stats (caller has synchronised)
void drain_timings(hs_sketch *h) {
    for (auto &e : h->pending_update) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) h->stats.update_ms += ms;
        h->pool.push_back(e);
    }
    h->pending_update.clear();
    for (auto &e : h->pending_search) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) h->stats.search_ms += ms;
        h->pool.push_back(e);
    }
    h->pending_search.clear();
    for (auto &e : h->pending_flush) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            h->stats.flush_ms += ms;
            h->stats.update_ms += ms;
        }
        h->pool.push_back(e);
    }
    h->pending_flush.clear();
    cudaGetLastError();
}

void free_topk_scratch(hs_sketch *h) {
    void *ps[] = {h->cand_key, h->cand_est, h->counters, h->bitmap,  h->slots,
                  h->distinct, h->distinct_est, h->sel, h->hist,  h->tmp_key, h->tmp_est,
                  h->tmp_rank, h->out_key, h->out_est};
    for (void *p : ps)
        if (p) cudaFree(p);
    h->cand_key = nullptr;
    h->cand_est = nullptr;
    h->counters = nullptr;
    h->bitmap = nullptr;
    h->slots = nullptr;
    h->distinct = nullptr;
    h->distinct_est = nullptr;
    h->sel = nullptr;
    h->hist = nullptr;
    h->tmp_key = nullptr;
    h->tmp_est = nullptr;
    h->tmp_rank = nullptr;
    h->out_key = nullptr;
    h->out_est = nullptr;
    h->cap = 0;
    h->out_cap = 0;
}

hs_status ensure_topk_scratch(hs_sketch *h, uint64_t k) {
    uint64_t want_cap = std::max<uint64_t>(std::max<uint64_t>(1ull << 22, 8 * k), k + h->min_cap);
    if (h->cand_key && h->cap >= want_cap && h->out_cap >= k) return HS_OK;
    free_topk_scratch(h);
    h->cap = want_cap;
    h->out_cap = std::max<uint64_t>(k, 1);
    h->nb = bitmap_log2_bits(h->d.rows, h->d.log2w, kSearchSmemBudget);
    uint64_t words = (uint64_t)h->d.rows * std::max<uint64_t>((1ull << h->nb) >> 5, 1);
    HS_CUDA(cudaMalloc(&h->cand_key, h->cap * 8));
    HS_CUDA(cudaMalloc(&h->cand_est, h->cap * 4));
    HS_CUDA(cudaMalloc(&h->counters, 4 * sizeof(unsigned long long)));
    HS_CUDA(cudaMalloc(&h->bitmap, words * 4));
    HS_CUDA(cudaMalloc(&h->slots, (size_t)8 << kProbeSlotsLog2));
    HS_CUDA(cudaMalloc(&h->distinct, kProbeCap * 8));
    HS_CUDA(cudaMalloc(&h->distinct_est, kProbeCap * 4));
    HS_CUDA(cudaMalloc(&h->sel, sizeof(SelectState)));
    HS_CUDA(cudaMalloc(&h->hist, 256 * sizeof(unsigned long long)));
    HS_CUDA(cudaMalloc(&h->tmp_key, h->out_cap * 8));
    HS_CUDA(cudaMalloc(&h->tmp_est, h->out_cap * 4));
    HS_CUDA(cudaMalloc(&h->tmp_rank, h->out_cap * 4));
    HS_CUDA(cudaMalloc(&h->out_key, h->out_cap * 8));
    HS_CUDA(cudaMalloc(&h->out_est, h->out_cap * 4));
    return HS_OK;
}

void free_dir(hs_sketch *h) {
    void *ps[] = {h->xbits, h->hot_list, h->hot_cnt, h->dir_cursor, h->scan_scratch};
    for (void *p : ps)
        if (p) cudaFree(p);
    for (int r = 0; r < kMaxRows; ++r) {
        if (!h->is_view) {             // a view's directories belong to its batch
            if (h->dir_off[r]) cudaFree(h->dir_off[r]);
            if (h->dir_rec[r]) cudaFree(h->dir_rec[r]);
        }
        h->dir_off[r] = nullptr;
        h->dir_rec[r] = nullptr;
        h->dir_G[r] = 0;
        h->dir_lines_cap[r] = 0;
    }
    h->xbits = nullptr;
    h->hot_list = nullptr;
    h->hot_cnt = nullptr;
    h->dir_cursor = nullptr;
    h->scan_scratch = nullptr;
}

// rows whose hot buckets are enumerated: a passing cell is hot in one of them
uint32_t enum_rows(const hs_sketch *h) {
    uint32_t t = h->d.rows, need = t - (t - 1) / 2;
    return t - need + 1;
}

// scratch of the directory search (not the directories themselves)
hs_status ensure_dir_scratch(hs_sketch *h) {
    if (h->xbits) return HS_OK;
    uint64_t wpr = std::max<uint64_t>(h->d.W >> 5, 1);
    h->dir_D = std::min<uint32_t>(h->d.log2w, 26);
    h->hot_cap = std::min<uint64_t>(h->d.W, 1ull << 22);
    uint64_t nslots = 1ull << h->dir_D;
    HS_CUDA(cudaMalloc(&h->xbits, (size_t)h->d.rows * wpr * 4));
    HS_CUDA(cudaMalloc(&h->hot_list, (size_t)enum_rows(h) * h->hot_cap * 4));
    HS_CUDA(cudaMalloc(&h->hot_cnt, kMaxRows * sizeof(unsigned long long)));
    HS_CUDA(cudaMalloc(&h->dir_cursor, (nslots + 1) * 4));
    HS_CUDA(cudaMalloc(&h->scan_scratch, (nslots / 1024 + 4096) * 4));
    return HS_OK;
}

// build the directory of row r (once per mesh size; the buffers are reused
// when a batch view moves to a smaller mesh); false when memory is short
bool ensure_dir(hs_sketch *h, int r) {
    uint64_t lines = (uint64_t)h->d.G * h->d.G;
    if (h->dir_off[r] && h->dir_G[r] == h->d.G) return true;
    uint64_t nslots = 1ull << h->dir_D;
    if (h->dir_off[r] && h->dir_lines_cap[r] < lines) {
        cudaFree(h->dir_off[r]);
        cudaFree(h->dir_rec[r]);
        h->dir_off[r] = nullptr;
        h->dir_rec[r] = nullptr;
    }
    if (!h->dir_off[r]) {
        if (cudaMalloc(&h->dir_off[r], (nslots + 1) * 4) != cudaSuccess ||
            cudaMalloc(&h->dir_rec[r], lines * sizeof(DirRecord)) != cudaSuccess) {
            cudaGetLastError();
            if (h->dir_off[r]) cudaFree(h->dir_off[r]);
            h->dir_off[r] = nullptr;
            h->dir_rec[r] = nullptr;
            return false;
        }
        h->dir_lines_cap[r] = lines;
    }
    int launches = 0;
    cudaError_t e = launch_dir_build(h->d, r, h->dir_D, h->dir_off[r], h->dir_cursor, h->dir_rec[r],
                                     h->scan_scratch, h->num_sms * 8, h->stream, &launches);
    h->stats.kernel_launches += launches;
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->dir_off[r]);
        cudaFree(h->dir_rec[r]);
        h->dir_off[r] = nullptr;
        h->dir_rec[r] = nullptr;
        return false;
    }
    h->dir_G[r] = h->d.G;
    return true;
}

hs_status ensure_staging(hs_sketch *h) {
    if (h->stage[0]) return HS_OK;
    for (int i = 0; i < kStageBuffers; ++i) {
        HS_CUDA(cudaMalloc(&h->stage[i], kStageParticles * 12));
        HS_CUDA(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming));
        HS_CUDA(cudaEventCreateWithFlags(&h->ev_free[i], cudaEventDisableTiming));
    }
    HS_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    return HS_OK;
}

hs_status ensure_query_scratch(hs_sketch *h, uint64_t m) {
    if (h->q_cap >= m) return HS_OK;
    if (h->q_keys) cudaFree(h->q_keys);
    if (h->q_est) cudaFree(h->q_est);
    h->q_keys = nullptr;
    h->q_est = nullptr;
    h->q_cap = 0;
    uint64_t c = std::max<uint64_t>(m, 1 << 16);
    HS_CUDA(cudaMalloc(&h->q_keys, c * 8));
    HS_CUDA(cudaMalloc(&h->q_est, c * 4));
    h->q_cap = c;
    return HS_OK;
}

hs_status launch_update_direct(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                               double rate, bool packed = false);

// add every binned code to the counters (before anything reads them)
hs_status drain(hs_sketch *h) {
    if (h->pending <= 0) return HS_OK;
    EventPair ev = take_events(h);
    cudaEventRecord(ev.a, h->stream);
    if (h->carry_valid) {
        HS_CUDA(launch_carry_flush(h->bl, h->carry, (uint32_t)h->num_sms, h->bins, h->bin_cursor,
                                   h->bin_cap, h->C, h->stream));
        h->carry_valid = false;
        h->stats.kernel_launches += 1;
    }
    HS_CUDA(launch_bin_accumulate(h->bl, h->bins, h->bin_cursor, h->bin_cap, h->C, h->stream));
    cudaEventRecord(ev.b, h->stream);
    h->pending_flush.push_back(ev);
    h->stats.kernel_launches += 1;
    h->stats.flush_launches += 1;
    h->pending = 0;
    return HS_OK;
}

// drop binned codes that were never drained (reset / load)
hs_status discard_pending(hs_sketch *h) {
    if (h->pending > 0 && h->bin_cursor)
        HS_CUDA(cudaMemsetAsync(h->bin_cursor, 0, (size_t)h->bl.nbins * 4, h->stream));
    h->pending = 0;
    h->carry_valid = false;
    return HS_OK;
}

bool want_binned(hs_sketch *h, uint64_t n, double rate) {
    if (h->routing) return true;          // only the binned scatter routes
    if (h->p.flags & HS_FLAG_UPDATE_DIRECT) return false;
    if (h->bl.slot == 0) return false;
    if (h->p.flags & HS_FLAG_UPDATE_BINNED) return true;
    return (double)n * rate * h->d.rows >= kBinnedMinUpdates;
}

hs_status ensure_bins(hs_sketch *h, uint64_t n, double rate) {
    if (h->bins) return HS_OK;
    const double per_bin = (double)(1ull << (h->d.log2w - h->bl.S));   // bins per row
    uint64_t want = (uint64_t)(1.3 * (double)n * rate / per_bin) + 8192;
    uint64_t most = kBinBudgetBytes / (2ull * h->bl.nbins);
    uint64_t cap = std::min(want, most);
    cap = std::max<uint64_t>(cap, 4096);
    cap = std::min<uint64_t>(cap, 0xFFFFFFF0ull);
    cap = (cap + 15) & ~15ull;
    HS_CUDA(cudaMalloc(&h->carry, (size_t)h->num_sms * carry_words16(h->bl) * 16));
    HS_CUDA(cudaMalloc(&h->bins, (size_t)h->bl.nbins * cap * 2));
    HS_CUDA(cudaMalloc(&h->bin_cursor, (size_t)h->bl.nbins * 4));
    HS_CUDA(cudaMemsetAsync(h->bin_cursor, 0, (size_t)h->bl.nbins * 4, h->stream));
    h->bin_cap = (uint32_t)cap;
    // expected codes per bin = kept particles / bins per row; keep a margin of
    // 20 % and 6 standard deviations below the capacity
    double c = (double)cap;
    double safe = c - 6.0 * std::sqrt(c) - 4096.0;
    h->pending_limit = std::max(0.0, 0.8 * safe) * per_bin;
    return HS_OK;
}

// xyz: float32 positions, or packed 64-bit records when packed is set
hs_status launch_update_timed(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                              double rate, bool packed = false) {
    const size_t esz = packed ? 8 : 12;
    if (want_binned(h, n, rate)) {
        hs_status st = ensure_bins(h, n, rate);
        if (st != HS_OK) return st;
        if (h->routing && h->pending_limit < 1.0)
            return fail(HS_ERR_STATE, "routing needs bins of useful capacity");
        if (h->pending_limit >= 1.0) {
            // launches small enough that no bin is expected to fill
            uint64_t piece = (uint64_t)std::max(1.0, h->pending_limit / rate);
            for (uint64_t off = 0; off < n; off += piece) {
                uint64_t cnt = std::min(piece, n - off);
                if (h->pending + (double)cnt * rate > h->pending_limit) {
                    st = drain(h);
                    if (st != HS_OK) return st;
                }
                EventPair ev = take_events(h);
                cudaEventRecord(ev.a, h->stream);
                const float *src = reinterpret_cast<const float *>(
                    reinterpret_cast<const char *>(xyz) + off * esz);
                HS_CUDA(launch_bin_scatter(src, cnt, g0 + off, h->d, h->C, rate,
                                           h->p.sample_seed, h->probe, h->probe_base, kProbeCap,
                                           h->bl, h->bins, h->bin_cursor, h->bin_cap, h->num_sms,
                                           h->stream, nullptr, 0, 0, 1024,
                                           h->routing ? &h->route : nullptr, h->carry,
                                           h->carry_valid ? 1 : 0, 1, packed ? 1 : 0));
                h->carry_valid = true;
                cudaEventRecord(ev.b, h->stream);
                h->pending_update.push_back(ev);
                h->pending += (double)cnt * rate;
                h->stats.update_launches += 1;
                h->stats.kernel_launches += 1;
            }
            return HS_OK;
        }
    }
    return launch_update_direct(h, xyz, n, g0, rate, packed);
}

hs_status launch_update_direct(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                               double rate, bool packed) {
    EventPair ev = take_events(h);
    cudaEventRecord(ev.a, h->stream);
    if (packed)
        HS_CUDA(launch_update_packed(reinterpret_cast<const uint64_t *>(xyz), n, g0, h->d, h->C,
                                     rate, h->p.sample_seed, h->probe, h->probe_base, kProbeCap,
                                     h->num_sms * 8, h->stream));
    else
        HS_CUDA(launch_update(xyz, n, g0, h->d, h->C, rate, h->p.sample_seed, h->probe,
                              h->probe_base, kProbeCap, 0,
                              (uint32_t)h->d.W, h->num_sms * 8, h->stream));
    cudaEventRecord(ev.b, h->stream);
    h->pending_update.push_back(ev);
    h->stats.update_launches += 1;
    h->stats.kernel_launches += 1;
    return HS_OK;
}

// Directory search of one pass; *used = false when it does not apply (too
// many hot buckets, more work than the scan, or memory short).
hs_status search_pass_dir(hs_sketch *h, int32_t theta, SearchMode mode, int64_t hot,
                          uint64_t line_lo, uint64_t line_hi, SearchOut out, bool *used) {
    *used = false;
    const uint64_t G = h->d.G, lines = G * G;
    if (h->dir_failed || lines >= (1ull << 32)) return HS_OK;
    if (ensure_dir_scratch(h) != HS_OK) {
        cudaGetLastError();
        free_dir(h);
        h->dir_failed = true;
        return HS_OK;
    }
    const uint32_t F = enum_rows(h);
    HS_CUDA(launch_hot_bitmap(h->C, h->d, h->d.log2w, (int32_t)std::min<int64_t>(hot, INT32_MAX),
                              h->xbits, h->num_sms * 8, h->stream));
    HS_CUDA(cudaMemsetAsync(h->hot_cnt, 0, kMaxRows * sizeof(unsigned long long), h->stream));
    for (uint32_t r = 0; r < F; ++r)
        HS_CUDA(launch_hot_list(h->xbits, h->d, (int)r, h->hot_list + r * h->hot_cap,
                                &h->hot_cnt[r], h->hot_cap, h->num_sms * 8, h->stream));
    h->stats.kernel_launches += 1 + F;
    unsigned long long cnt[kMaxRows];
    HS_CUDA(cudaMemcpyAsync(cnt, h->hot_cnt, F * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    // relative costs, from GB300 timings: one scanned cell ~ 1 (about 1e10
    // cells/s); one (cx, hot bucket) query ~ 0.25 per directory slot it reads
    // (about 4e10 queries/s); building a directory ~ 1 per line.  The query
    // and build weights are kept about 4x above the measured ones.
    const double per_slot = (double)lines / (double)(1ull << h->dir_D);
    double cost_dir = 0, cost_scan = (double)G * G * G;
    for (uint32_t r = 0; r < F; ++r) {
        if (cnt[r] > h->hot_cap) return HS_OK;
        cost_dir += 1.0 * (double)G * (double)cnt[r] * (1.0 + per_slot);
        if (!h->dir_off[r] || h->dir_G[r] != h->d.G) cost_dir += 4.0 * (double)lines;
    }
    const uint32_t force = h->p.flags & (HS_FLAG_SEARCH_SCAN | HS_FLAG_SEARCH_DIRECTORY);
    if (force == HS_FLAG_SEARCH_SCAN) return HS_OK;
    if (force != HS_FLAG_SEARCH_DIRECTORY && cost_dir >= cost_scan) return HS_OK;
    for (uint32_t r = 0; r < F; ++r) {
        if (!ensure_dir(h, (int)r)) {
            free_dir(h);
            h->dir_failed = true;
            return HS_OK;
        }
    }
    EventPair ev = take_events(h);
    cudaEventRecord(ev.a, h->stream);
    for (uint32_t r = 0; r < F; ++r) {
        HS_CUDA(launch_dir_query(h->C, h->d, (int)r, h->dir_D, h->dir_off[r], h->dir_rec[r],
                                 h->hot_list + r * h->hot_cap, cnt[r], h->xbits, theta, mode,
                                 line_lo, line_hi, out, h->num_sms * 16, h->stream,
                                 h->route.filter));
    }
    cudaEventRecord(ev.b, h->stream);
    h->pending_search.push_back(ev);
    h->stats.search_launches += 1;
    h->stats.kernel_launches += F;
    *used = true;
    return HS_OK;
}

// One full-search pass over lines [line_lo, line_hi); appends after count_base.
// Returns the new candidate count (possibly above cap).
hs_status search_pass(hs_sketch *h, int32_t theta, SearchMode mode, uint64_t line_lo,
                      uint64_t line_hi, unsigned long long count_base,
                      unsigned long long *count_out) {
    int64_t hot = (int64_t)theta + (mode == kGT ? 1 : 0);
    int prune = hot >= 1;
    if (mode == kGT && theta == INT32_MAX) line_hi = line_lo;   // nothing above the largest int32
    HS_CUDA(cudaMemcpyAsync(&h->counters[0], &count_base, sizeof(count_base),
                            cudaMemcpyHostToDevice, h->stream));
    SearchOut out{h->cand_key, h->cand_est, &h->counters[0], h->cap};
    bool used = false;
    if (prune && line_hi > line_lo) {
        hs_status st = search_pass_dir(h, theta, mode, hot, line_lo, line_hi, out, &used);
        if (st != HS_OK) return st;
    }
    if (!used) {
        if (prune) {
            HS_CUDA(launch_hot_bitmap(h->C, h->d, h->nb,
                                      (int32_t)std::min<int64_t>(hot, INT32_MAX), h->bitmap,
                                      h->num_sms * 8, h->stream));
            h->stats.kernel_launches += 1;
        }
        // a scan touches every cell of the lines: refuse meshes whose scan would
        // run for minutes, and keep each launch to about 2^34 cells
        const uint64_t G = h->d.G;
        if ((line_hi - line_lo) * G > kMaxScanCells)
            return fail(HS_ERR_STATE,
                        "full scan of %llu cells refused (directory search unavailable at this "
                        "threshold); use the hierarchical query (sketch_set_hierarchy)",
                        (unsigned long long)((line_hi - line_lo) * G));
        const uint64_t seg = std::max<uint64_t>(1, (1ull << 34) / G);
        EventPair ev = take_events(h);
        cudaEventRecord(ev.a, h->stream);
        for (uint64_t l0 = line_lo; l0 < line_hi; l0 += seg) {
            HS_CUDA(launch_full_search(h->C, h->d, theta, mode, h->bitmap, h->nb, prune, l0,
                                       std::min(line_hi, l0 + seg), out, h->num_sms, h->stream,
                                       h->route.filter));
            h->stats.kernel_launches += 1;
        }
        cudaEventRecord(ev.b, h->stream);
        h->pending_search.push_back(ev);
        h->stats.search_launches += 1;
    }
    h->stats.last_passes += 1;
    h->stats.last_threshold = theta;
    unsigned long long c = 0;
    HS_CUDA(cudaMemcpyAsync(&c, &h->counters[0], sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    *count_out = c;
    return HS_OK;
}

// estimate of the k-th best entry of (key, est)[0..m)
hs_status kth_estimate(hs_sketch *h, const uint64_t *key, const int32_t *est, uint64_t m,
                       uint64_t k, int32_t *theta) {
    int launches = 0;
    HS_CUDA(launch_select_kth(key, est, m, k, h->key_bits, h->sel, h->hist, h->num_sms * 4,
                              h->stream, &launches));
    h->stats.kernel_launches += launches;
    SelectState st;
    HS_CUDA(cudaMemcpyAsync(&st, h->sel, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    *theta = (int32_t)(st.hi ^ 0x80000000u);
    return HS_OK;
}

// the k best of the m >= k candidates, in rank order, into h->out_*
hs_status finalize(hs_sketch *h, uint64_t m, uint64_t k) {
    int launches = 0;
    int all = m <= k;
    if (!all)
        HS_CUDA(launch_select_kth(h->cand_key, h->cand_est, m, k, h->key_bits, h->sel, h->hist,
                                  h->num_sms * 4, h->stream, &launches));
    uint64_t n_take = all ? m : k;
    HS_CUDA(launch_take_sorted(h->cand_key, h->cand_est, m, h->sel, all, h->tmp_key, h->tmp_est,
                               &h->counters[1], h->tmp_rank, n_take, h->out_key, h->out_est, h->num_sms * 4,
                               h->stream, &launches));
    h->stats.kernel_launches += launches;
    return HS_OK;
}

}  // namespace

extern "C" {

const char *hs_last_error(void) { return g_last_error.c_str(); }

hs_status sketch_create(const hs_params *params, void *cuda_stream, hs_sketch **out) {
    if (!out) return fail(HS_ERR_ARG, "out is NULL");
    hs_status st = check_params(params);
    if (st != HS_OK) return st;
    hs_sketch *h = new (std::nothrow) hs_sketch();
    if (!h) return fail(HS_ERR_OOM, "host allocation failed");
    h->p = *params;
    h->stream = (cudaStream_t)cuda_stream;
    std::memset(&h->stats, 0, sizeof(h->stats));
    SketchDesc &d = h->d;
    std::memset(&d, 0, sizeof(d));
    d.rows = params->rows;
    d.log2w = params->log2_width;
    d.G = (uint32_t)std::llround(params->box / params->cell);
    d.inv_cell = (float)(1.0 / params->cell);
    d.Gq = d.G;
    d.F = 1;
    d.W = 1ull << params->log2_width;
    for (uint32_t r = 0; r < d.rows; ++r) {   // splitmix64 outputs 4r .. 4r+3
        d.seed[r].a0 = splitmix64_at(params->hash_seed, 4 * r + 0);
        d.seed[r].a1 = splitmix64_at(params->hash_seed, 4 * r + 1);
        d.seed[r].a2 = splitmix64_at(params->hash_seed, 4 * r + 2);
        d.seed[r].b = splitmix64_at(params->hash_seed, 4 * r + 3);
    }
    h->n_cells = (uint64_t)d.G * d.G * d.G;
    h->bl = bin_layout(d, kBinSmemBudget);
    h->key_bits = 1;
    while (h->key_bits < 64 && (1ull << h->key_bits) < h->n_cells) ++h->key_bits;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->C, (size_t)d.rows * d.W * 4);
    if (e == cudaSuccess) e = cudaMalloc(&h->probe, kProbeCap * 8);
    if (e == cudaSuccess) e = cudaMalloc(&h->flags, 4 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->C, 0, (size_t)d.rows * d.W * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->probe, 0xFF, kProbeCap * 8, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        hs_status code = e == cudaErrorMemoryAllocation ? HS_ERR_OOM : HS_ERR_CUDA;
        sketch_destroy(h);
        return fail(code, "sketch_create: %s", cudaGetErrorString(e));
    }
    *out = h;
    return HS_OK;
}

hs_status sketch_destroy(hs_sketch *h) {
    if (!h) return HS_OK;
    cudaStreamSynchronize(h->stream);
    if (h->super) sketch_destroy(h->super);
    free_topk_scratch(h);
    free_dir(h);
    if (h->bins) cudaFree(h->bins);
    if (h->carry) cudaFree(h->carry);
    if (h->bin_cursor) cudaFree(h->bin_cursor);
    if (h->C && !h->is_view) cudaFree(h->C);
    if (h->probe && !h->is_view) cudaFree(h->probe);
    if (h->q_keys) cudaFree(h->q_keys);
    if (h->q_est) cudaFree(h->q_est);
    if (h->flags) cudaFree(h->flags);
    for (int i = 0; i < kStageBuffers; ++i) {
        if (h->stage[i]) cudaFree(h->stage[i]);
        if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
        if (h->ev_free[i]) cudaEventDestroy(h->ev_free[i]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (auto *v : {&h->pending_update, &h->pending_search, &h->pending_flush, &h->pool})
        for (auto &e : *v) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
    delete h;
    cudaGetLastError();
    return HS_OK;
}

// sketch_update and sketch_update_packed: src holds n float32 xyz triples or n
// packed records, in host or device memory
static hs_status update_common(hs_sketch *h, const void *src, uint64_t n, double sample_rate,
                               bool packed) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (!(sample_rate > 0.0 && sample_rate <= 1.0))
        return fail(HS_ERR_ARG, "sample_rate=%g outside (0, 1]", sample_rate);
    if (n == 0) return HS_OK;
    if (!src) return fail(HS_ERR_ARG, "input is NULL");
    if (n > (~0ull - h->n_seen)) return fail(HS_ERR_ARG, "particle index overflow");
    if (packed && (h->routing || h->is_view))
        return fail(HS_ERR_ARG, "packed records need a plain or hierarchical sketch");
    const size_t esz = packed ? 8 : 12;
    const float *xyz = static_cast<const float *>(src);
    if (is_device_ptr(src)) {
        hs_status st = launch_update_timed(h, xyz, n, h->n_seen, sample_rate, packed);
        if (st == HS_OK && h->super)
            st = launch_update_timed(h->super, xyz, n, h->n_seen, sample_rate, packed);
        if (st != HS_OK) return st;
    } else {
        hs_status st = ensure_staging(h);
        if (st != HS_OK) return st;
        // size the bins for the whole call, not for one staged piece
        const uint64_t first = std::min(kStageParticles, n);
        if (want_binned(h, first, sample_rate)) st = ensure_bins(h, n, sample_rate);
        if (st == HS_OK && h->super && want_binned(h->super, first, sample_rate))
            st = ensure_bins(h->super, n, sample_rate);
        if (st != HS_OK) return st;
        int i = 0;
        for (uint64_t off = 0; off < n; off += kStageParticles, ++i) {
            uint64_t cnt = std::min(kStageParticles, n - off);
            int b = i % kStageBuffers;
            HS_CUDA(cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0));
            HS_CUDA(cudaMemcpyAsync(h->stage[b], static_cast<const char *>(src) + off * esz,
                                    cnt * esz, cudaMemcpyHostToDevice, h->copy_stream));
            HS_CUDA(cudaEventRecord(h->ev_copied[b], h->copy_stream));
            HS_CUDA(cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
            st = launch_update_timed(h, h->stage[b], cnt, h->n_seen + off, sample_rate, packed);
            if (st == HS_OK && h->super)
                st = launch_update_timed(h->super, h->stage[b], cnt, h->n_seen + off, sample_rate,
                                         packed);
            if (st != HS_OK) return st;
            HS_CUDA(cudaEventRecord(h->ev_free[b], h->stream));
        }
    }
    h->n_seen += n;
    if (h->super) h->super->n_seen += n;
    return HS_OK;
}

hs_status sketch_update(hs_sketch *h, const float *xyz, uint64_t n, double sample_rate) {
    return update_common(h, xyz, n, sample_rate, false);
}

hs_status sketch_update_packed(hs_sketch *h, const uint64_t *records, uint64_t n,
                               double sample_rate) {
    return update_common(h, records, n, sample_rate, true);
}

hs_status pack_positions(const float *xyz, uint64_t n, double box, void *cuda_stream,
                         uint64_t *records) {
    if (n && (!xyz || !records)) return fail(HS_ERR_ARG, "NULL argument");
    if (!(box > 0)) return fail(HS_ERR_ARG, "box must be positive");
    if (n && (!is_device_ptr(xyz) || !is_device_ptr(records)))
        return fail(HS_ERR_ARG, "xyz and records must be device memory");
    HS_CUDA(launch_pack(xyz, n, box, records, (cudaStream_t)cuda_stream));
    return HS_OK;
}

hs_status sketch_wait_copies(hs_sketch *h) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (h->copy_stream) HS_CUDA(cudaStreamSynchronize(h->copy_stream));
    return HS_OK;
}

hs_status sketch_query(hs_sketch *h, const uint64_t *keys, uint64_t m, int32_t *est) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (m == 0) return HS_OK;
    if (!keys || !est) return fail(HS_ERR_ARG, "keys/est is NULL");
    bool kd = is_device_ptr(keys), ed = is_device_ptr(est);
    hs_status st = drain(h);
    if (st != HS_OK) return st;
    st = ensure_query_scratch(h, (kd && ed) ? 0 : m);
    if (st != HS_OK) return st;
    const uint64_t *dk = keys;
    int32_t *de = est;
    if (!kd) {
        HS_CUDA(cudaMemcpyAsync(h->q_keys, keys, m * 8, cudaMemcpyHostToDevice, h->stream));
        dk = h->q_keys;
    }
    if (!ed) de = h->q_est;
    HS_CUDA(cudaMemsetAsync(h->flags, 0, 4 * sizeof(uint32_t), h->stream));
    HS_CUDA(launch_point_query(h->C, h->d, dk, m, de, &h->flags[0], h->stream));
    h->stats.kernel_launches += 1;
    if (!ed) HS_CUDA(cudaMemcpyAsync(est, de, m * 4, cudaMemcpyDeviceToHost, h->stream));
    uint32_t bad = 0;
    HS_CUDA(cudaMemcpyAsync(&bad, &h->flags[0], 4, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    if (bad) return fail(HS_ERR_ARG, "a key is >= G^3 = %llu", (unsigned long long)h->n_cells);
    return HS_OK;
}

// The k-th best estimate among the distinct cells of the first particles of
// the stream (kept in the probe), or INT32_MIN when there are fewer than k.
static hs_status probe_theta(hs_sketch *h, uint64_t kk, int32_t *theta) {
    *theta = INT32_MIN;
    const uint64_t m_probe = std::min<uint64_t>(h->n_seen - h->probe_base, h->probe_cap);
    if (m_probe < kk) return HS_OK;
    HS_CUDA(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned long long), h->stream));
    HS_CUDA(cudaMemsetAsync(h->flags, 0, 4 * sizeof(uint32_t), h->stream));
    HS_CUDA(launch_probe_distinct(h->probe, m_probe, h->slots, kProbeSlotsLog2, h->distinct,
                                  &h->counters[2], &h->flags[1], h->stream));
    unsigned long long nd = 0;
    HS_CUDA(cudaMemcpyAsync(&nd, &h->counters[2], 8, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    h->stats.kernel_launches += 1;
    if (nd < kk) return HS_OK;
    HS_CUDA(launch_point_query(h->C, h->d, h->distinct, nd, h->distinct_est, &h->flags[0],
                               h->stream));
    h->stats.kernel_launches += 1;
    return kth_estimate(h, h->distinct, h->distinct_est, nd, kk, theta);
}

// One pass of the hierarchy's second layer over the key window [key_lo, key_hi).
static hs_status expand_pass(hs_sketch *h, const uint64_t *skeys, uint64_t ns, int32_t theta,
                             SearchMode mode, uint64_t key_lo, uint64_t key_hi,
                             unsigned long long count_base, unsigned long long *count_out) {
    HS_CUDA(cudaMemcpyAsync(&h->counters[0], &count_base, sizeof(count_base),
                            cudaMemcpyHostToDevice, h->stream));
    SearchOut out{h->cand_key, h->cand_est, &h->counters[0], h->cap};
    if (!(mode == kGT && theta == INT32_MAX) && key_hi > key_lo) {
        EventPair ev = take_events(h);
        cudaEventRecord(ev.a, h->stream);
        int launches = 0;
        HS_CUDA(launch_expand(h->C, h->d, skeys, ns, h->super->d.F, h->super->d.G, theta, mode,
                              key_lo, key_hi, out, h->num_sms * 8, h->stream, &launches,
                              h->route.filter));
        cudaEventRecord(ev.b, h->stream);
        h->pending_search.push_back(ev);
        h->stats.search_launches += 1;
        h->stats.kernel_launches += launches;
    }
    h->stats.last_passes += 1;
    h->stats.last_threshold = theta;
    unsigned long long c = 0;
    HS_CUDA(cudaMemcpyAsync(&c, &h->counters[0], sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    *count_out = c;
    return HS_OK;
}

// Hierarchical query (Algorithm 3, CSHi, with the top-(c*k) rule of the GPU
// hierarchy): the c*k best super-items by the super sketch's own full search,
// then the kk best cells inside them, found with a raised threshold like the
// flat search.
static hs_status topk_hier(hs_sketch *h, uint64_t kk, uint64_t *keys, int32_t *est,
                           uint32_t *n_out) {
    hs_sketch *S = h->super;
    const uint64_t ms = std::min<uint64_t>((uint64_t)h->super_mult * kk, S->n_cells);
    if (ms > 0xFFFFFFFFull) return fail(HS_ERR_ARG, "c * k too large");
    std::vector<uint64_t> hk(ms);
    std::vector<int32_t> he(ms);
    uint32_t ns = 0;
    hs_status st = topk_extract(S, (uint32_t)ms, hk.data(), he.data(), &ns);
    if (st != HS_OK) return st;
    const uint64_t *skeys = S->out_key;   // the super ranking stays on the device
    st = drain(h);
    if (st != HS_OK) return st;
    st = ensure_topk_scratch(h, kk);
    if (st != HS_OK) return st;
    h->stats.last_passes = 0;
    EventPair whole = take_events(h);
    cudaEventRecord(whole.a, h->stream);
    const uint64_t n_cells = h->n_cells;
    // a first threshold from the probe; if the selected super-items hold fewer
    // than k cells above it, the loop below starts again without one
    int32_t theta = INT32_MIN;
    st = probe_theta(h, kk, &theta);
    if (st != HS_OK) return st;
    uint64_t final_m = 0;
    for (int round = 0;; ++round) {
        if (round > 64) return fail(HS_ERR_STATE, "top-k threshold did not converge");
        unsigned long long c = 0;
        st = expand_pass(h, skeys, ns, theta, kGE, 0, n_cells, 0, &c);
        if (st != HS_OK) return st;
        h->stats.last_candidates = c;
        if (c <= h->cap) {
            if (c >= kk) {
                final_m = c;
                break;
            }
            if (theta == INT32_MIN) return fail(HS_ERR_STATE, "fewer cells than k");
            theta = INT32_MIN;
            continue;
        }
        int32_t t2 = 0;
        st = kth_estimate(h, h->cand_key, h->cand_est, h->cap, kk, &t2);
        if (st != HS_OK) return st;
        if (t2 > theta) {
            theta = t2;
            continue;
        }
        unsigned long long c_gt = 0;
        st = expand_pass(h, skeys, ns, theta, kGT, 0, n_cells, 0, &c_gt);
        if (st != HS_OK) return st;
        if (c_gt > h->cap) {
            st = kth_estimate(h, h->cand_key, h->cand_est, h->cap, kk, &t2);
            if (st != HS_OK) return st;
            theta = t2;
            continue;
        }
        if (c_gt >= kk) {
            final_m = c_gt;
            break;
        }
        // the ties at theta in key order: windows of the key space, halved
        // when one holds more ties than the candidate buffer has room for
        uint64_t need = kk - c_gt, have = 0, lo = 0, span = n_cells;
        while (have < need && lo < n_cells) {
            const uint64_t hi = span >= n_cells - lo ? n_cells : lo + span;
            unsigned long long c2 = 0;
            st = expand_pass(h, skeys, ns, theta, kEQ, lo, hi, c_gt + have, &c2);
            if (st != HS_OK) return st;
            if (c2 > h->cap) {
                span = std::max<uint64_t>(1, span / 2);
                continue;
            }
            have = c2 - c_gt;
            lo = hi;
        }
        final_m = c_gt + have;
        h->stats.last_candidates = final_m;
        break;
    }
    st = finalize(h, final_m, kk);
    if (st != HS_OK) return st;
    const uint64_t n = std::min<uint64_t>(final_m, kk);
    HS_CUDA(cudaMemcpyAsync(keys, h->out_key, n * 8, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaMemcpyAsync(est, h->out_est, n * 4, cudaMemcpyDeviceToHost, h->stream));
    cudaEventRecord(whole.b, h->stream);
    HS_CUDA(cudaStreamSynchronize(h->stream));
    float ms_t = 0;
    if (cudaEventElapsedTime(&ms_t, whole.a, whole.b) == cudaSuccess) h->stats.topk_ms += ms_t;
    h->pool.push_back(whole);
    h->stats.topk_calls += 1;
    drain_timings(h);
    *n_out = (uint32_t)n;
    return HS_OK;
}

hs_status topk_extract(hs_sketch *h, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (k == 0 || !keys || !est || !n_out) return fail(HS_ERR_ARG, "k == 0 or NULL output");
    const uint64_t kk = std::min<uint64_t>(k, h->n_cells);
    if (h->super) return topk_hier(h, kk, keys, est, n_out);
    hs_status st = drain(h);
    if (st != HS_OK) return st;
    st = ensure_topk_scratch(h, kk);
    if (st != HS_OK) return st;
    h->stats.last_passes = 0;
    EventPair whole = take_events(h);
    cudaEventRecord(whole.a, h->stream);
    const uint64_t lines = (uint64_t)h->d.G * h->d.G;

    // 1. a lower bound on the k-th estimate: the k-th best estimate among the
    //    distinct cells of the first particles of the stream
    int32_t theta = INT32_MIN;
    st = probe_theta(h, kk, &theta);
    if (st != HS_OK) return st;

    // 2. full search with that threshold; raise it on overflow
    uint64_t final_m = 0;
    for (int round = 0;; ++round) {
        if (round > 64) return fail(HS_ERR_STATE, "top-k threshold did not converge");
        unsigned long long c = 0;
        st = search_pass(h, theta, kGE, 0, lines, 0, &c);
        if (st != HS_OK) return st;
        h->stats.last_candidates = c;
        if (c <= h->cap) {
            if (c >= kk) {
                final_m = c;
                break;
            }
            if (theta == INT32_MIN) return fail(HS_ERR_STATE, "fewer cells than k");
            theta = INT32_MIN;   // cannot happen for a valid lower bound; start over
            continue;
        }
        int32_t t2 = 0;
        st = kth_estimate(h, h->cand_key, h->cand_est, h->cap, kk, &t2);
        if (st != HS_OK) return st;
        if (t2 > theta) {
            theta = t2;
            continue;
        }
        // many cells tie at theta: take every cell above it, then the ties in key order
        unsigned long long c_gt = 0;
        st = search_pass(h, theta, kGT, 0, lines, 0, &c_gt);
        if (st != HS_OK) return st;
        if (c_gt > h->cap) {
            st = kth_estimate(h, h->cand_key, h->cand_est, h->cap, kk, &t2);
            if (st != HS_OK) return st;
            theta = t2;
            continue;
        }
        if (c_gt >= kk) {
            final_m = c_gt;
            break;
        }
        uint64_t need = kk - c_gt, have = 0, line = 0;
        while (have < need && line < lines) {
            uint64_t room = h->cap - c_gt - have;
            uint64_t seg = std::max<uint64_t>(1, room / h->d.G);
            uint64_t hi = std::min(lines, line + seg);
            unsigned long long c2 = 0;
            st = search_pass(h, theta, kEQ, line, hi, c_gt + have, &c2);
            if (st != HS_OK) return st;
            have = c2 - c_gt;
            line = hi;
        }
        final_m = c_gt + have;
        h->stats.last_candidates = final_m;
        break;
    }
    st = finalize(h, final_m, kk);
    if (st != HS_OK) return st;
    uint64_t n = std::min<uint64_t>(final_m, kk);
    HS_CUDA(cudaMemcpyAsync(keys, h->out_key, n * 8, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaMemcpyAsync(est, h->out_est, n * 4, cudaMemcpyDeviceToHost, h->stream));
    cudaEventRecord(whole.b, h->stream);
    HS_CUDA(cudaStreamSynchronize(h->stream));
    float ms = 0;
    if (cudaEventElapsedTime(&ms, whole.a, whole.b) == cudaSuccess) h->stats.topk_ms += ms;
    h->pool.push_back(whole);
    h->stats.topk_calls += 1;
    drain_timings(h);
    *n_out = (uint32_t)n;
    return HS_OK;
}

hs_status sketch_reset(hs_sketch *h) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    hs_status st = discard_pending(h);
    if (st != HS_OK) return st;
    HS_CUDA(cudaMemsetAsync(h->C, 0, (size_t)h->d.rows * h->d.W * 4, h->stream));
    HS_CUDA(cudaMemsetAsync(h->probe, 0xFF, kProbeCap * 8, h->stream));
    h->n_seen = 0;
    h->probe_base = 0;
    if (h->super) return sketch_reset(h->super);
    return HS_OK;
}

hs_status sketch_counters(hs_sketch *h, int32_t *out) {
    if (!h || !out) return fail(HS_ERR_ARG, "NULL argument");
    hs_status st = drain(h);
    if (st != HS_OK) return st;
    HS_CUDA(cudaMemcpyAsync(out, h->C, (size_t)h->d.rows * h->d.W * 4, cudaMemcpyDefault,
                            h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    return HS_OK;
}

hs_status sketch_load_counters(hs_sketch *h, const int32_t *in) {
    if (!h || !in) return fail(HS_ERR_ARG, "NULL argument");
    hs_status st = discard_pending(h);
    if (st != HS_OK) return st;
    HS_CUDA(cudaMemcpyAsync(h->C, in, (size_t)h->d.rows * h->d.W * 4, cudaMemcpyDefault,
                            h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    return HS_OK;
}

hs_status sketch_merge(hs_sketch *dst, hs_sketch *src) {
    if (!dst || !src) return fail(HS_ERR_ARG, "NULL handle");
    const hs_params &a = dst->p, &b = src->p;
    if (a.rows != b.rows || a.log2_width != b.log2_width || a.hash_seed != b.hash_seed ||
        dst->d.G != src->d.G || dst->d.inv_cell != src->d.inv_cell)
        return fail(HS_ERR_ARG, "sketches were built with different parameters");
    if (dst == src) return fail(HS_ERR_ARG, "cannot merge a sketch into itself");
    if (!dst->super != !src->super)
        return fail(HS_ERR_ARG, "one sketch has a hierarchy and the other has not");
    if (dst->super) {
        hs_status s2 = sketch_merge(dst->super, src->super);
        if (s2 != HS_OK) return s2;
    }
    hs_status st = drain(src);
    if (st == HS_OK) st = drain(dst);
    if (st != HS_OK) return st;
    cudaEvent_t ev;
    HS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HS_CUDA(cudaEventRecord(ev, src->stream));
    HS_CUDA(cudaStreamWaitEvent(dst->stream, ev, 0));
    cudaEventDestroy(ev);
    HS_CUDA(launch_add_counters(dst->C, src->C, (uint64_t)a.rows << a.log2_width, dst->stream));
    dst->stats.kernel_launches += 1;
    dst->n_seen += src->n_seen;
    return HS_OK;
}

hs_status sketch_info(const hs_sketch *h, hs_info *out) {
    if (!h || !out) return fail(HS_ERR_ARG, "NULL argument");
    out->rows = h->d.rows;
    out->log2_width = h->d.log2w;
    out->grid = h->d.G;
    out->inv_cell = h->d.inv_cell;
    out->width = h->d.W;
    out->n_cells = h->n_cells;
    out->n_seen = h->n_seen;
    return HS_OK;
}

hs_status sketch_seek(hs_sketch *h, uint64_t n_seen) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    HS_CUDA(cudaMemsetAsync(h->probe, 0xFF, kProbeCap * 8, h->stream));
    h->n_seen = n_seen;
    h->probe_base = n_seen;
    if (h->super) return sketch_seek(h->super, n_seen);
    return HS_OK;
}

hs_status sketch_flush(hs_sketch *h) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (h->super) {
        hs_status st = drain(h->super);
        if (st != HS_OK) return st;
    }
    return drain(h);
}

hs_status sketch_set_hierarchy(hs_sketch *h, uint32_t super_factor, uint32_t super_log2_width,
                               uint32_t c_mult) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (h->super) return fail(HS_ERR_STATE, "the sketch already has a hierarchy");
    if (h->n_seen != 0 || h->is_view || h->routing)
        return fail(HS_ERR_STATE, "set the hierarchy on a fresh, plain sketch");
    if (super_factor < 2 || super_factor > 64 || h->d.G % super_factor != 0 || h->d.G > 65535)
        return fail(HS_ERR_ARG, "super_factor must be in [2, 64] and divide a mesh below 2^16");
    if (c_mult < 1) return fail(HS_ERR_ARG, "c_mult must be >= 1");
    hs_params q = h->p;
    q.log2_width = super_log2_width;
    q.cell = h->p.cell * super_factor;
    q.hash_seed = h->p.hash_seed + 1;
    hs_sketch *s = nullptr;
    hs_status st = sketch_create(&q, h->stream, &s);
    if (st != HS_OK) return st;
    if (s->d.G * super_factor != h->d.G) {
        sketch_destroy(s);
        return fail(HS_ERR_ARG, "box / (cell * super_factor) is not the super grid");
    }
    s->d.Gq = h->d.G;
    s->d.inv_cell = h->d.inv_cell;
    s->d.F = super_factor;
    s->d.fmagic = (uint32_t)((0x100000000ull + super_factor - 1) / super_factor);
    h->super = s;
    h->super_mult = c_mult;
    return HS_OK;
}

hs_status sketch_super(hs_sketch *h, hs_sketch **out) {
    if (!h || !out) return fail(HS_ERR_ARG, "NULL argument");
    *out = h->super;
    return HS_OK;
}

hs_status sketch_synchronize(hs_sketch *h) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    HS_CUDA(cudaStreamSynchronize(h->stream));
    return HS_OK;
}

hs_status sketch_stats(hs_sketch *h, hs_stats *out, int reset) {
    if (!h || !out) return fail(HS_ERR_ARG, "NULL argument");
    HS_CUDA(cudaStreamSynchronize(h->stream));
    drain_timings(h);
    *out = h->stats;
    if (reset) std::memset(&h->stats, 0, sizeof(h->stats));
    return HS_OK;
}

hs_status hs_measure_red_rate(uint64_t n_counters, uint64_t total_ops, double *ops_per_s) {
    if (!ops_per_s || n_counters == 0 || (n_counters & (n_counters - 1)) || total_ops == 0)
        return fail(HS_ERR_ARG, "n_counters must be a power of two and total_ops > 0");
    int dev = 0, sms = 0;
    HS_CUDA(cudaGetDevice(&dev));
    HS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint32_t *t = nullptr;
    HS_CUDA(cudaMalloc(&t, n_counters * 4));
    cudaStream_t s;
    cudaEvent_t a, b;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int blocks = sms * 8;
    uint64_t per = std::max<uint64_t>(1, total_ops / ((uint64_t)blocks * 256));
    cudaMemsetAsync(t, 0, n_counters * 4, s);
    launch_red_rate(t, n_counters, per, blocks, s);   // warm the table into L2
    cudaEventRecord(a, s);
    cudaError_t e = launch_red_rate(t, n_counters, per, blocks, s);
    cudaEventRecord(b, s);
    cudaStreamSynchronize(s);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    cudaFree(t);
    if (e != cudaSuccess) return fail(HS_ERR_CUDA, "red-rate kernel: %s", cudaGetErrorString(e));
    *ops_per_s = (double)per * blocks * 256 / (ms * 1e-3);
    return HS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// sketch_query_noalloc: point queries without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they query: code running
// while a CUDA stream is being captured into a graph (allocation is not a
// capturable operation), processes whose device memory is fully reserved by
// another allocator or a fixed budget, and latency-critical loops where an
// allocation's synchronisation is not acceptable.  sketch_query may allocate
// staging buffers on its first call with host arrays; this variant instead
// uses one file-scope device array, sized for at most
// HS_NOALLOC_QUERY_MAX keys, that every GPU loading this library holds until
// the process exits.
// ---------------------------------------------------------------------------

namespace {

constexpr uint64_t kNoallocMax = HS_NOALLOC_QUERY_MAX;
constexpr size_t kNoallocKeysOff = 0;
constexpr size_t kNoallocEstOff = kNoallocMax * 8;
constexpr size_t kNoallocFlagOff = kNoallocMax * 12;
constexpr size_t kNoallocBytes = kNoallocMax * 12 + 256;
constexpr int kNoallocMaxDevices = 64;

// keys staging | estimates staging | out-of-range flag; shared by every call
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).  The
// host-side name g_noalloc_scratch is only a stand-in, never a device address.
hs_status noalloc_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(HS_ERR_ARG, "device %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(HS_ERR_CUDA, "cudaGetSymbolAddress of the query scratch failed: %s",
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return HS_OK;
}

// Estimate (Sec. 2.2) of each key; keys >= G^3 give 0 and set *bad.
__global__ void k_point_query_noalloc(const int32_t *__restrict__ C, const SketchDesc d,
                                      const uint64_t *__restrict__ keys, uint64_t m,
                                      int32_t *__restrict__ est, uint32_t *__restrict__ bad) {
    const uint64_t n_cells = (uint64_t)d.G * d.G * d.G;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint64_t key = keys[i];
        if (key >= n_cells) {
            est[i] = 0;
            atomicOr(bad, 1u);
            continue;
        }
        uint32_t cx = (uint32_t)(key % d.G);
        uint64_t rest = key / d.G;
        uint32_t cy = (uint32_t)(rest % d.G), cz = (uint32_t)(rest / d.G);
        int32_t ev[kMaxRows];
        for (uint32_t r = 0; r < d.rows; ++r) {
            uint64_t v = row_value(d.seed[r], cx, cy, cz);
            ev[r] = signed_count(C[r * d.W + bucket_of(v, d.log2w)], v, d.log2w);
        }
        est[i] = d.rows == 5 ? median5(ev[0], ev[1], ev[2], ev[3], ev[4])
                             : lower_median_dyn(ev, (int)d.rows);
    }
}

}  // namespace

extern "C" hs_status sketch_query_noalloc(hs_sketch *h, const uint64_t *keys, uint64_t m,
                                          int32_t *est) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (m == 0) return HS_OK;
    if (!keys || !est) return fail(HS_ERR_ARG, "keys/est is NULL");
    if (m > kNoallocMax)
        return fail(HS_ERR_ARG, "m=%llu exceeds HS_NOALLOC_QUERY_MAX=%llu; split the query",
                    (unsigned long long)m, (unsigned long long)kNoallocMax);
    int dev = -1;
    HS_CUDA(cudaGetDevice(&dev));
    if (dev != h->device)
        return fail(HS_ERR_STATE, "make the sketch's device %d current (current: %d)", h->device,
                    dev);
    unsigned char *scratch = nullptr;
    hs_status st = noalloc_scratch(dev, &scratch);
    if (st != HS_OK) return st;
    st = drain(h);   // pending binned increments use buffers that already exist
    if (st != HS_OK) return st;
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(scratch + kNoallocKeysOff);
    int32_t *s_est = reinterpret_cast<int32_t *>(scratch + kNoallocEstOff);
    uint32_t *s_flag = reinterpret_cast<uint32_t *>(scratch + kNoallocFlagOff);
    const bool kd = is_device_ptr(keys), ed = is_device_ptr(est);
    const uint64_t *dk = keys;
    int32_t *de = ed ? est : s_est;
    if (!kd) {
        HS_CUDA(cudaMemcpyAsync(s_keys, keys, m * 8, cudaMemcpyHostToDevice, h->stream));
        dk = s_keys;
    }
    HS_CUDA(cudaMemsetAsync(s_flag, 0, 4, h->stream));   // the previous call's flag stays otherwise
    uint64_t blocks = std::min<uint64_t>((m + 255) / 256, 65535);
    k_point_query_noalloc<<<(unsigned)blocks, 256, 0, h->stream>>>(h->C, h->d, dk, m, de, s_flag);
    HS_CUDA(cudaGetLastError());
    h->stats.kernel_launches += 1;
    if (!ed) HS_CUDA(cudaMemcpyAsync(est, de, m * 4, cudaMemcpyDeviceToHost, h->stream));
    uint32_t bad = 0;
    HS_CUDA(cudaMemcpyAsync(&bad, s_flag, 4, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    if (bad) return fail(HS_ERR_ARG, "a key is >= G^3 = %llu", (unsigned long long)h->n_cells);
    return HS_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent sub-volumes (each with its own mesh, stream index,
// sketch and top-k), updated by one persistent scatter launch and one
// accumulation launch, replayed as a CUDA graph.
// ---------------------------------------------------------------------------

namespace {

constexpr uint64_t kBatchProbe = 1ull << 16;   // probe keys per volume

}  // namespace

struct hs_batch {
    hs_params p;
    uint32_t nvol = 0;
    SketchDesc d;                       // rows, log2 W, seeds
    std::vector<uint32_t> G;
    std::vector<float> inv;
    std::vector<uint64_t> n_seen, probe_base;
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t *C = nullptr;               // nvol x rows x W
    uint64_t *probe = nullptr;          // nvol x kBatchProbe
    BinLayout bl{};                     // over nvol * rows rows
    uint16_t *bins = nullptr;
    uint32_t *cursor = nullptr;
    uint32_t cap = 0;
    VolumeDesc *d_vols = nullptr;
    VolumeDesc *h_vols = nullptr;       // pinned: read by the graph's copy node
    int threads = 1024;
    hs_sketch *view = nullptr;          // views[0]
    std::vector<hs_sketch *> views;     // top-k of one volume each, concurrently, own streams
    std::vector<cudaEvent_t> vdone;     // each view's stream has finished
    // directories of each volume's enumerated rows, kept across queries
    std::vector<uint32_t *> vdir_off;
    std::vector<DirRecord *> vdir_rec;
    std::vector<uint32_t> vdir_G;
    std::vector<uint64_t> vdir_cap;
    cudaGraphExec_t gexec = nullptr;
    const float *g_xyz = nullptr;
    uint64_t g_n = 0;
    double g_rate = -1;
    cudaEvent_t done = nullptr;         // the last graph launch has finished with h_vols
    cudaEvent_t fork = nullptr;         // the views' streams start after this
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    hs_stats stats;
};

namespace {

void batch_drop_graph(hs_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->g_xyz = nullptr;
}

SketchDesc batch_flat_desc(const hs_batch *b) {
    SketchDesc dd = b->d;
    dd.rows = b->nvol * b->d.rows;      // the layout sees one sketch of nvol * t rows
    return dd;
}

hs_status batch_ensure_bins(hs_batch *b, const uint64_t *offsets, double rate) {
    if (b->bins) return HS_OK;
    const double bins_per_row = (double)(1ull << (b->d.log2w - b->bl.S));
    uint64_t most = 0;
    for (uint32_t v = 0; v < b->nvol; ++v) most = std::max(most, offsets[v + 1] - offsets[v]);
    uint64_t want = (uint64_t)(1.3 * (double)most * rate / bins_per_row) + 8192;
    uint64_t cap = std::min<uint64_t>(want, kBinBudgetBytes / (2ull * b->bl.nbins));
    cap = std::min<uint64_t>(std::max<uint64_t>(cap, 4096), 0xFFFFFFF0ull);
    cap = (cap + 15) & ~15ull;
    HS_CUDA(cudaMalloc(&b->bins, (size_t)b->bl.nbins * cap * 2));
    b->cap = (uint32_t)cap;
    return HS_OK;
}

// scatter + accumulate of the whole batch on b->stream (captured or direct)
hs_status batch_enqueue(hs_batch *b, const float *xyz, uint64_t n, double rate) {
    HS_CUDA(cudaMemcpyAsync(b->d_vols, b->h_vols, b->nvol * sizeof(VolumeDesc),
                            cudaMemcpyHostToDevice, b->stream));
    int grid = b->num_sms * (b->threads == 512 ? 2 : 1);
    HS_CUDA(launch_bin_scatter(xyz, n, 0, b->d, b->C, rate, b->p.sample_seed, b->probe, 0,
                               kBatchProbe, b->bl, b->bins, b->cursor, b->cap, grid, b->stream,
                               b->d_vols, b->nvol, kBatchProbe, b->threads));
    HS_CUDA(launch_bin_accumulate(b->bl, b->bins, b->cursor, b->cap, b->C, b->stream));
    return HS_OK;
}

hs_status batch_check_offsets(const hs_batch *b, const float *xyz, const uint64_t *offsets) {
    if (!offsets) return fail(HS_ERR_ARG, "offsets is NULL");
    if (offsets[0] != 0) return fail(HS_ERR_ARG, "offsets[0] must be 0");
    for (uint32_t v = 0; v < b->nvol; ++v)
        if (offsets[v + 1] < offsets[v]) return fail(HS_ERR_ARG, "offsets must not decrease");
    if (offsets[b->nvol] > 0) {
        if (!xyz) return fail(HS_ERR_ARG, "xyz is NULL");
        if (!is_device_ptr(xyz)) return fail(HS_ERR_ARG, "batch particles must be device memory");
    }
    return HS_OK;
}

void batch_fill_vols(hs_batch *b, const uint64_t *offsets) {
    const uint32_t bins_per_row = 1u << (b->d.log2w - b->bl.S);
    for (uint32_t v = 0; v < b->nvol; ++v) {
        VolumeDesc &V = b->h_vols[v];
        V.start = offsets[v];
        V.g0 = b->n_seen[v];
        V.probe_base = b->probe_base[v];
        V.inv_cell = b->inv[v];
        V.G = b->G[v];
        V.bin0 = v * b->d.rows * bins_per_row;
        V.pad = 0;
    }
}

}  // namespace

extern "C" {

hs_status batch_destroy(hs_batch *b);

hs_status batch_create(const hs_params *params, uint32_t n_volumes, const double *boxes,
                       void *cuda_stream, hs_batch **out) {
    if (!out || !boxes || n_volumes == 0) return fail(HS_ERR_ARG, "NULL argument or no volumes");
    if (!params) return fail(HS_ERR_ARG, "params is NULL");
    hs_params p = *params;
    p.box = boxes[0];
    hs_status st = check_params(&p);
    if (st != HS_OK) return st;
    hs_batch *b = new (std::nothrow) hs_batch();
    if (!b) return fail(HS_ERR_OOM, "host allocation failed");
    b->p = p;
    b->nvol = n_volumes;
    std::memset(&b->stats, 0, sizeof(b->stats));
    std::memset(&b->d, 0, sizeof(b->d));
    b->d.rows = p.rows;
    b->d.log2w = p.log2_width;
    b->d.W = 1ull << p.log2_width;
    for (uint32_t r = 0; r < p.rows; ++r) {
        b->d.seed[r].a0 = splitmix64_at(p.hash_seed, 4 * r + 0);
        b->d.seed[r].a1 = splitmix64_at(p.hash_seed, 4 * r + 1);
        b->d.seed[r].a2 = splitmix64_at(p.hash_seed, 4 * r + 2);
        b->d.seed[r].b = splitmix64_at(p.hash_seed, 4 * r + 3);
    }
    b->G.resize(n_volumes);
    b->inv.assign(n_volumes, (float)(1.0 / p.cell));
    b->n_seen.assign(n_volumes, 0);
    b->probe_base.assign(n_volumes, 0);
    for (uint32_t v = 0; v < n_volumes; ++v) {
        double g = std::llround(boxes[v] / p.cell);
        if (!(boxes[v] > 0) || g < 1 || g > 65535) {
            delete b;
            return fail(HS_ERR_ARG, "volume %u: grid round(box/cell) outside [1, 65535]", v);
        }
        b->G[v] = (uint32_t)g;
    }
    b->d.G = b->G[0];
    b->d.inv_cell = b->inv[0];
    b->d.Gq = b->d.G;
    b->d.F = 1;
    b->bl = bin_layout(batch_flat_desc(b), kBinSmemBudget);
    if (b->bl.slot == 0 || b->bl.nbins >= 65536) {
        delete b;
        return fail(HS_ERR_ARG, "%u volumes x %u rows x 2^%u counters need too many bins; "
                    "split the batch", n_volumes, p.rows, p.log2_width);
    }
    const size_t counters = (size_t)n_volumes * p.rows * b->d.W;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) {
        if (cuda_stream) b->stream = (cudaStream_t)cuda_stream;
        else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = true;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->C, counters * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->probe, (size_t)n_volumes * kBatchProbe * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->cursor, (size_t)b->bl.nbins * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_vols, n_volumes * sizeof(VolumeDesc));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_vols, n_volumes * sizeof(VolumeDesc));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_a);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_b);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->C, 0, counters * 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->probe, 0xFF, (size_t)n_volumes * kBatchProbe * 8, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->cursor, 0, (size_t)b->bl.nbins * 4, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    const uint32_t nviews = std::min<uint32_t>(n_volumes, kBatchViews);
    for (uint32_t t = 0; t < nviews && e == cudaSuccess; ++t) {
        hs_sketch *h = new (std::nothrow) hs_sketch();
        if (!h) {
            e = cudaErrorMemoryAllocation;
            break;
        }
        h->p = p;
        h->d = b->d;
        h->is_view = true;
        h->device = b->device;
        h->num_sms = b->num_sms;
        h->probe_cap = kBatchProbe;
        h->bl = BinLayout{};        // views never bin
        std::memset(&h->stats, 0, sizeof(h->stats));
        b->views.push_back(h);
        b->vdone.push_back(nullptr);
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->vdone.back(), cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&h->flags, 4 * sizeof(uint32_t));
    }
    if (e == cudaSuccess) b->view = b->views[0];
    if (e != cudaSuccess) {
        hs_status code = e == cudaErrorMemoryAllocation ? HS_ERR_OOM : HS_ERR_CUDA;
        batch_destroy(b);
        return fail(code, "batch_create: %s", cudaGetErrorString(e));
    }
    *out = b;
    return HS_OK;
}

hs_status batch_destroy(hs_batch *b) {
    if (!b) return HS_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    for (size_t t = 0; t < b->views.size(); ++t) {
        hs_sketch *h = b->views[t];
        h->C = nullptr;
        h->probe = nullptr;
        cudaStream_t vs = h->stream;
        sketch_destroy(h);
        if (vs) cudaStreamDestroy(vs);
        if (b->vdone[t]) cudaEventDestroy(b->vdone[t]);
    }
    void *ps[] = {b->C, b->probe, b->cursor, b->d_vols, b->bins};
    for (void *q : ps)
        if (q) cudaFree(q);
    for (auto *q : b->vdir_off)
        if (q) cudaFree(q);
    for (auto *q : b->vdir_rec)
        if (q) cudaFree(q);
    if (b->h_vols) cudaFreeHost(b->h_vols);
    if (b->done) cudaEventDestroy(b->done);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_a) cudaEventDestroy(b->ev_a);
    if (b->ev_b) cudaEventDestroy(b->ev_b);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    cudaGetLastError();
    return HS_OK;
}

hs_status batch_update(hs_batch *b, const float *xyz, const uint64_t *offsets, double sample_rate) {
    if (!b) return fail(HS_ERR_ARG, "batch is NULL");
    if (!(sample_rate > 0.0 && sample_rate <= 1.0))
        return fail(HS_ERR_ARG, "sample_rate=%g outside (0, 1]", sample_rate);
    hs_status st = batch_check_offsets(b, xyz, offsets);
    if (st != HS_OK) return st;
    const uint64_t n = offsets[b->nvol];
    if (n == 0) return HS_OK;
    st = batch_ensure_bins(b, offsets, sample_rate);
    if (st != HS_OK) return st;
    HS_CUDA(cudaEventSynchronize(b->done));          // the previous graph has read h_vols
    batch_fill_vols(b, offsets);
    if (!b->gexec || b->g_xyz != xyz || b->g_n != n || b->g_rate != sample_rate) {
        batch_drop_graph(b);
        cudaGraph_t graph = nullptr;
        HS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
        st = batch_enqueue(b, xyz, n, sample_rate);
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (st != HS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        HS_CUDA(e);
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        HS_CUDA(e);
        b->g_xyz = xyz;
        b->g_n = n;
        b->g_rate = sample_rate;
    }
    HS_CUDA(cudaEventRecord(b->ev_a, b->stream));
    HS_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    HS_CUDA(cudaEventRecord(b->ev_b, b->stream));
    HS_CUDA(cudaEventRecord(b->done, b->stream));
    b->stats.kernel_launches += 2;
    b->stats.update_launches += 1;
    for (uint32_t v = 0; v < b->nvol; ++v) b->n_seen[v] += offsets[v + 1] - offsets[v];
    return HS_OK;
}

// Top-k of volume v on view h (the view borrows the volume's counters, probe
// and directories, and returns the directories it built).
static hs_status batch_topk_one(hs_batch *b, hs_sketch *h, uint32_t v, uint32_t F, uint32_t k,
                                uint64_t *keys, int32_t *est, uint32_t *n_out) {
    for (uint32_t r = 0; r < F; ++r) {
        h->dir_off[r] = b->vdir_off[v * F + r];
        h->dir_rec[r] = b->vdir_rec[v * F + r];
        h->dir_G[r] = b->vdir_G[v * F + r];
        h->dir_lines_cap[r] = b->vdir_cap[v * F + r];
    }
    h->C = b->C + (size_t)v * b->d.rows * b->d.W;
    h->probe = b->probe + (size_t)v * kBatchProbe;
    h->d.G = b->G[v];
    h->d.Gq = b->G[v];
    h->d.F = 1;
    h->d.inv_cell = b->inv[v];
    h->n_cells = (uint64_t)b->G[v] * b->G[v] * b->G[v];
    h->key_bits = 1;
    while (h->key_bits < 64 && (1ull << h->key_bits) < h->n_cells) ++h->key_bits;
    h->n_seen = b->n_seen[v];
    h->probe_base = b->probe_base[v];
    hs_status st = topk_extract(h, k, keys + (size_t)v * k, est + (size_t)v * k, &n_out[v]);
    for (uint32_t r = 0; r < F; ++r) {
        b->vdir_off[v * F + r] = h->dir_off[r];
        b->vdir_rec[v * F + r] = h->dir_rec[r];
        b->vdir_G[v * F + r] = h->dir_G[r];
        b->vdir_cap[v * F + r] = h->dir_lines_cap[r];
        h->dir_off[r] = nullptr;
        h->dir_rec[r] = nullptr;
        h->dir_G[r] = 0;
        h->dir_lines_cap[r] = 0;
    }
    return st;
}

hs_status batch_topk(hs_batch *b, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out) {
    if (!b) return fail(HS_ERR_ARG, "batch is NULL");
    if (k == 0 || !keys || !est || !n_out) return fail(HS_ERR_ARG, "k == 0 or NULL output");
    const uint32_t F = enum_rows(b->view);
    if (b->vdir_off.size() != (size_t)b->nvol * F) {
        b->vdir_off.assign((size_t)b->nvol * F, nullptr);
        b->vdir_rec.assign((size_t)b->nvol * F, nullptr);
        b->vdir_G.assign((size_t)b->nvol * F, 0);
        b->vdir_cap.assign((size_t)b->nvol * F, 0);
    }
    // the views start after the batch's pending work; the batch resumes after theirs
    HS_CUDA(cudaEventRecord(b->fork, b->stream));
    for (hs_sketch *h : b->views) HS_CUDA(cudaStreamWaitEvent(h->stream, b->fork, 0));
    // each host thread drives one view over volumes taken from a shared counter
    std::atomic<uint32_t> next{0};
    std::vector<hs_status> status(b->views.size(), HS_OK);
    std::vector<std::string> msg(b->views.size());
    auto work = [&](size_t t) {
        cudaSetDevice(b->device);
        for (uint32_t v = next.fetch_add(1); v < b->nvol; v = next.fetch_add(1)) {
            hs_status st = batch_topk_one(b, b->views[t], v, F, k, keys, est, n_out);
            if (st != HS_OK) {
                status[t] = st;
                msg[t] = hs_last_error();
                next.store(b->nvol);
                break;
            }
        }
    };
    std::vector<std::thread> pool;
    for (size_t t = 1; t < b->views.size(); ++t) pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool) th.join();
    for (size_t t = 0; t < b->views.size(); ++t) {
        HS_CUDA(cudaEventRecord(b->vdone[t], b->views[t]->stream));
        HS_CUDA(cudaStreamWaitEvent(b->stream, b->vdone[t], 0));
    }
    for (size_t t = 0; t < b->views.size(); ++t)
        if (status[t] != HS_OK) return fail(status[t], "%s", msg[t].c_str());
    return HS_OK;
}

hs_status batch_counters(hs_batch *b, uint32_t volume, int32_t *out) {
    if (!b || !out || volume >= (b ? b->nvol : 0)) return fail(HS_ERR_ARG, "bad argument");
    const size_t per = (size_t)b->d.rows * b->d.W;
    HS_CUDA(cudaMemcpyAsync(out, b->C + volume * per, per * 4, cudaMemcpyDefault, b->stream));
    HS_CUDA(cudaStreamSynchronize(b->stream));
    return HS_OK;
}

hs_status batch_reset(hs_batch *b) {
    if (!b) return fail(HS_ERR_ARG, "batch is NULL");
    HS_CUDA(cudaMemsetAsync(b->C, 0, (size_t)b->nvol * b->d.rows * b->d.W * 4, b->stream));
    HS_CUDA(cudaMemsetAsync(b->probe, 0xFF, (size_t)b->nvol * kBatchProbe * 8, b->stream));
    HS_CUDA(cudaMemsetAsync(b->cursor, 0, (size_t)b->bl.nbins * 4, b->stream));
    std::fill(b->n_seen.begin(), b->n_seen.end(), 0);
    std::fill(b->probe_base.begin(), b->probe_base.end(), 0);
    return HS_OK;
}

hs_status batch_volume_info(const hs_batch *b, uint32_t volume, hs_info *out) {
    if (!b || !out || volume >= b->nvol) return fail(HS_ERR_ARG, "bad argument");
    out->rows = b->d.rows;
    out->log2_width = b->d.log2w;
    out->grid = b->G[volume];
    out->inv_cell = b->inv[volume];
    out->width = b->d.W;
    out->n_cells = (uint64_t)b->G[volume] * b->G[volume] * b->G[volume];
    out->n_seen = b->n_seen[volume];
    return HS_OK;
}

hs_status batch_stats(hs_batch *b, hs_stats *out, int reset) {
    if (!b || !out) return fail(HS_ERR_ARG, "NULL argument");
    HS_CUDA(cudaStreamSynchronize(b->stream));
    float ms = 0;
    if (b->stats.update_launches && cudaEventElapsedTime(&ms, b->ev_a, b->ev_b) == cudaSuccess)
        b->stats.update_ms = ms;                     // the last update
    cudaGetLastError();
    *out = b->stats;
    out->search_launches = 0;
    out->search_ms = 0;
    out->topk_ms = 0;
    out->topk_calls = 0;
    for (hs_sketch *h : b->views) {
        hs_stats vs{};
        sketch_stats(h, &vs, reset);
        out->kernel_launches += vs.kernel_launches;
        out->search_launches += vs.search_launches;
        out->search_ms += vs.search_ms;
        out->topk_ms += vs.topk_ms;     // summed over concurrent views
        out->topk_calls += vs.topk_calls;
    }
    if (reset) std::memset(&b->stats, 0, sizeof(b->stats));
    return HS_OK;
}

hs_status batch_autotune(hs_batch *b, const float *xyz, const uint64_t *offsets,
                         double sample_rate, hs_tune *out) {
    if (!b || !out) return fail(HS_ERR_ARG, "NULL argument");
    if (!(sample_rate > 0.0 && sample_rate <= 1.0)) return fail(HS_ERR_ARG, "bad sample_rate");
    hs_status st = batch_check_offsets(b, xyz, offsets);
    if (st != HS_OK) return st;
    const uint64_t n = offsets[b->nvol];
    if (n == 0) return fail(HS_ERR_ARG, "no particles to tune on");
    st = batch_ensure_bins(b, offsets, sample_rate);
    if (st != HS_OK) return st;
    batch_drop_graph(b);
    const BinLayout base = b->bl;
    const int threads_opt[2] = {1024, 512};
    const uint32_t slot_opt[2] = {32, 16};
    float best = 1e30f;
    int best_t = b->threads;
    BinLayout best_l = base;
    int tried = 0;
    for (int ti = 0; ti < 2; ++ti)
        for (int si = 0; si < 2; ++si) {
            BinLayout L = base;
            L.slot = slot_opt[si];
            size_t queue = (size_t)(1024 / 32) * 128 * 8;
            L.smem = ((L.nbins * 4 + 15) & ~15ull) + ((L.nbins * L.slot * 2 + 15) & ~15ull) + queue +
                     ((L.nbins + 31) / 32) * 4;
            if (L.smem > kBinSmemBudget) continue;
            if (threads_opt[ti] == 512 && L.nbins > 6u * 512) continue;
            b->bl = L;
            b->threads = threads_opt[ti];
            float ms_best = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                batch_fill_vols(b, offsets);
                HS_CUDA(cudaEventRecord(b->ev_a, b->stream));
                st = batch_enqueue(b, xyz, n, sample_rate);
                if (st != HS_OK) return st;
                HS_CUDA(cudaEventRecord(b->ev_b, b->stream));
                HS_CUDA(cudaStreamSynchronize(b->stream));
                float ms = 0;
                HS_CUDA(cudaEventElapsedTime(&ms, b->ev_a, b->ev_b));
                ms_best = std::min(ms_best, ms);
            }
            ++tried;
            if (ms_best < best) {
                best = ms_best;
                best_t = threads_opt[ti];
                best_l = L;
            }
        }
    b->bl = best_l;
    b->threads = best_t;
    st = batch_reset(b);                              // tuning runs touched the counters
    if (st != HS_OK) return st;
    HS_CUDA(cudaStreamSynchronize(b->stream));
    out->threads = (uint32_t)best_t;
    out->slot = best_l.slot;
    out->configs_tried = (uint32_t)tried;
    out->best_ms = best;
    return HS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned router: MLP objects, exact counting, and the learned sketch.
// ---------------------------------------------------------------------------

struct hs_mlp {
    float *P = nullptr, *M = nullptr, *V = nullptr, *grad = nullptr, *loss = nullptr;
    int step = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
};

struct hs_exact {
    SketchDesc d{};
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    uint64_t slots = 0;
    uint32_t key_bits = 1;
    unsigned long long *keys = nullptr;   // all ones = empty
    int32_t *counts = nullptr;
    uint32_t *overflow = nullptr;
    unsigned long long *ctr = nullptr;    // [0] listed entries, [1] taken entries
    SelectState *sel = nullptr;
    unsigned long long *hist = nullptr;
    uint64_t *tmp_key = nullptr, *out_key = nullptr;
    int32_t *tmp_est = nullptr, *out_est = nullptr;
    uint32_t *tmp_rank = nullptr;
    uint64_t out_cap = 0;
};

struct hs_learned {
    hs_sketch *sk = nullptr;       // the sketch of the cells that are not routed
    uint32_t R = 10, Gc = 0;
    uint64_t ncoarse = 0, words = 0;
    uint32_t coarse_key_bits = 1;
    uint64_t feature_seed = 0;
    double feature_rate = 1.0 / 64;
    uint64_t n_sampled = 0;        // particles passed to learned_sample since the last route
    int32_t *coarse = nullptr;     // Gc^3 sample counts
    uint64_t *clist = nullptr;     // coarse cells with a sample
    uint64_t clist_cap = 0, n_list = 0, n_routed = 0;
    uint16_t *feats = nullptr;
    float *logits = nullptr;
    int32_t *lrank = nullptr;      // routing rank of each listed cell
    uint32_t *routed = nullptr;    // Gc^3 bits
    uint32_t *prefix = nullptr;    // routed cells before each bitmap word
    uint32_t *scan_scratch = nullptr;
    uint64_t max_blocks = 0;       // routing budget: dense blocks of R^3 counters
    int32_t *blocks = nullptr;
    uint64_t *rlist = nullptr;     // coarse key of each block
    unsigned long long *ctr = nullptr;   // [0] list length, [1] positive logits, [2] table entries
    uint16_t *ftab = nullptr;      // bf16(log10(1 + n)) for n < kFeatTab
};

namespace {

constexpr uint32_t kFeatTab = 65536;

// float -> bf16 bits, round to nearest, ties to even (finite inputs)
uint16_t host_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

bool host_is_device(const void *p) { return is_device_ptr(p); }

// device copy of a host-or-device input (tmp is freed by the caller)
template <typename T>
hs_status device_input(const T *src, uint64_t count, cudaStream_t s, const T **dst, T **tmp) {
    *tmp = nullptr;
    if (host_is_device(src)) {
        *dst = src;
        return HS_OK;
    }
    HS_CUDA(cudaMalloc(tmp, std::max<uint64_t>(count, 1) * sizeof(T)));
    HS_CUDA(cudaMemcpyAsync(*tmp, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
    *dst = *tmp;
    return HS_OK;
}

void learned_free(hs_learned *L) {
    void *ps[] = {L->coarse, L->clist,  L->feats,        L->logits, L->lrank, L->routed,
                  L->prefix, L->scan_scratch, L->blocks, L->rlist, L->ctr,   L->ftab};
    for (void *q : ps)
        if (q) cudaFree(q);
}

}  // namespace

extern "C" {

hs_status mlp_destroy(hs_mlp *m) {
    if (!m) return HS_OK;
    void *ps[] = {m->P, m->M, m->V, m->grad, m->loss};
    for (void *q : ps)
        if (q) cudaFree(q);
    delete m;
    return HS_OK;
}

hs_status mlp_create(uint64_t seed, void *cuda_stream, hs_mlp **out) {
    if (!out) return fail(HS_ERR_ARG, "out is NULL");
    hs_mlp *m = new (std::nothrow) hs_mlp();
    if (!m) return fail(HS_ERR_OOM, "host allocation failed");
    m->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&m->device);
    for (float **q : {&m->P, &m->M, &m->V, &m->grad})
        if (e == cudaSuccess) e = cudaMalloc(q, kMlpParams * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, 2 * 4);
    if (e != cudaSuccess) {
        mlp_destroy(m);
        return fail(HS_ERR_OOM, "mlp_create: %s", cudaGetErrorString(e));
    }
    // uniform(-sqrt(6/fan_in), +sqrt(6/fan_in)) weights from splitmix64, zero biases
    std::vector<float> P(kMlpParams, 0.0f);
    uint64_t g = 0;
    auto uni = [&](double a) {
        uint64_t x = splitmix64_at(seed, g++);
        return (float)(((double)(x >> 11) * 0x1p-53 * 2.0 - 1.0) * a);
    };
    size_t o = 0;
    for (int i = 0; i < kMlpH * kMlpIn; ++i) P[o++] = uni(std::sqrt(6.0 / kMlpIn));
    o += kMlpH;
    for (int i = 0; i < kMlpH * kMlpH; ++i) P[o++] = uni(std::sqrt(6.0 / kMlpH));
    o += kMlpH;
    for (int i = 0; i < kMlpH; ++i) P[o++] = uni(std::sqrt(6.0 / kMlpH));
    e = cudaMemcpyAsync(m->P, P.data(), kMlpParams * 4, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->M, 0, kMlpParams * 4, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->V, 0, kMlpParams * 4, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        mlp_destroy(m);
        return fail(HS_ERR_CUDA, "mlp_create: %s", cudaGetErrorString(e));
    }
    *out = m;
    return HS_OK;
}

hs_status mlp_set_params(hs_mlp *m, const float *params) {
    if (!m || !params) return fail(HS_ERR_ARG, "NULL argument");
    HS_CUDA(cudaMemcpyAsync(m->P, params, kMlpParams * 4, cudaMemcpyDefault, m->stream));
    HS_CUDA(cudaMemsetAsync(m->M, 0, kMlpParams * 4, m->stream));
    HS_CUDA(cudaMemsetAsync(m->V, 0, kMlpParams * 4, m->stream));
    HS_CUDA(cudaStreamSynchronize(m->stream));
    m->step = 0;
    return HS_OK;
}

hs_status mlp_get_params(hs_mlp *m, float *params) {
    if (!m || !params) return fail(HS_ERR_ARG, "NULL argument");
    HS_CUDA(cudaMemcpyAsync(params, m->P, kMlpParams * 4, cudaMemcpyDefault, m->stream));
    HS_CUDA(cudaStreamSynchronize(m->stream));
    return HS_OK;
}

hs_status mlp_forward(hs_mlp *m, const uint16_t *feats, uint64_t n, float *logits) {
    if (!m || (n && (!feats || !logits))) return fail(HS_ERR_ARG, "NULL argument");
    if (n == 0) return HS_OK;
    const uint16_t *df;
    uint16_t *tf = nullptr;
    hs_status st = device_input(feats, n * kMlpIn, m->stream, &df, &tf);
    if (st != HS_OK) return st;
    const bool ld = host_is_device(logits);
    float *dl = logits;
    if (!ld && cudaMalloc(&dl, n * 4) != cudaSuccess) {
        if (tf) cudaFree(tf);
        return fail(HS_ERR_OOM, "mlp_forward: no memory for logits");
    }
    cudaError_t e = launch_mlp_forward(m->P, df, n, dl, m->stream);
    if (e == cudaSuccess && !ld) e = cudaMemcpyAsync(logits, dl, n * 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (tf) cudaFree(tf);
    if (!ld) cudaFree(dl);
    if (e != cudaSuccess) return fail(HS_ERR_CUDA, "mlp_forward: %s", cudaGetErrorString(e));
    return HS_OK;
}

static hs_status mlp_grad_common(hs_mlp *m, const uint16_t *feats, const float *y, const float *w,
                                 uint64_t n) {
    const uint16_t *df;
    const float *dy, *dw;
    uint16_t *tf = nullptr;
    float *ty = nullptr, *tw = nullptr;
    hs_status st = device_input(feats, n * kMlpIn, m->stream, &df, &tf);
    if (st == HS_OK) st = device_input(y, n, m->stream, &dy, &ty);
    if (st == HS_OK) st = device_input(w, n, m->stream, &dw, &tw);
    cudaError_t e = st == HS_OK ? launch_mlp_grad(m->P, df, dy, dw, n, m->grad, m->loss, m->stream)
                                : cudaSuccess;
    if (tf || ty || tw) cudaStreamSynchronize(m->stream);
    if (tf) cudaFree(tf);
    if (ty) cudaFree(ty);
    if (tw) cudaFree(tw);
    if (st != HS_OK) return st;
    HS_CUDA(e);
    return HS_OK;
}

hs_status mlp_gradient(hs_mlp *m, const uint16_t *feats, const float *y, const float *w, uint64_t n,
                       float *grad, float *loss) {
    if (!m || !feats || !y || !w || !grad || !loss || n == 0) return fail(HS_ERR_ARG, "bad argument");
    hs_status st = mlp_grad_common(m, feats, y, w, n);
    if (st != HS_OK) return st;
    HS_CUDA(cudaMemcpyAsync(grad, m->grad, kMlpParams * 4, cudaMemcpyDefault, m->stream));
    HS_CUDA(cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDefault, m->stream));
    HS_CUDA(cudaStreamSynchronize(m->stream));
    return HS_OK;
}

hs_status mlp_train_step(hs_mlp *m, const uint16_t *feats, const float *y, const float *w,
                         uint64_t n, float lr, float *loss) {
    if (!m || !feats || !y || !w || n == 0 || !(lr > 0)) return fail(HS_ERR_ARG, "bad argument");
    hs_status st = mlp_grad_common(m, feats, y, w, n);
    if (st != HS_OK) return st;
    m->step += 1;
    HS_CUDA(launch_adam(m->P, m->M, m->V, m->grad, m->loss + 1, lr, m->step, m->stream));
    if (loss) {
        float l[2];
        HS_CUDA(cudaMemcpyAsync(l, m->loss, 8, cudaMemcpyDeviceToHost, m->stream));
        HS_CUDA(cudaStreamSynchronize(m->stream));
        *loss = l[1] > 0 ? l[0] / l[1] : 0.0f;
    }
    return HS_OK;
}

hs_status exact_destroy(hs_exact *E) {
    if (!E) return HS_OK;
    void *ps[] = {E->keys, E->counts, E->overflow, E->ctr, E->sel, E->hist,
                  E->tmp_key, E->tmp_est, E->out_key, E->out_est, E->tmp_rank};
    for (void *q : ps)
        if (q) cudaFree(q);
    delete E;
    return HS_OK;
}

hs_status exact_create(double box, double cell, uint32_t log2_slots, void *cuda_stream,
                       hs_exact **out) {
    if (!out || log2_slots < 4 || log2_slots > 34) return fail(HS_ERR_ARG, "bad argument");
    hs_params p{1, 1, box, cell, 0, 0, 0, 0};
    hs_status st = check_params(&p);
    if (st != HS_OK) return st;
    hs_exact *E = new (std::nothrow) hs_exact();
    if (!E) return fail(HS_ERR_OOM, "host allocation failed");
    E->stream = (cudaStream_t)cuda_stream;
    E->d.G = (uint32_t)std::llround(box / cell);
    E->d.inv_cell = (float)(1.0 / cell);
    E->slots = 1ull << log2_slots;
    const uint64_t cells = (uint64_t)E->d.G * E->d.G * E->d.G;
    while (E->key_bits < 64 && (1ull << E->key_bits) < cells) ++E->key_bits;
    cudaError_t e = cudaGetDevice(&E->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&E->num_sms, cudaDevAttrMultiProcessorCount, E->device);
    if (e == cudaSuccess) e = cudaMalloc(&E->keys, E->slots * 8);
    if (e == cudaSuccess) e = cudaMalloc(&E->counts, E->slots * 4);
    if (e == cudaSuccess) e = cudaMalloc(&E->overflow, 4);
    if (e == cudaSuccess) e = cudaMalloc(&E->ctr, 2 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&E->sel, sizeof(SelectState));
    if (e == cudaSuccess) e = cudaMalloc(&E->hist, 256 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        exact_destroy(E);
        return fail(HS_ERR_OOM, "exact_create: %s", cudaGetErrorString(e));
    }
    st = exact_reset(E);
    if (st != HS_OK) {
        exact_destroy(E);
        return st;
    }
    *out = E;
    return HS_OK;
}

hs_status exact_reset(hs_exact *E) {
    if (!E) return fail(HS_ERR_ARG, "NULL handle");
    HS_CUDA(cudaMemsetAsync(E->keys, 0xFF, E->slots * 8, E->stream));
    HS_CUDA(cudaMemsetAsync(E->counts, 0, E->slots * 4, E->stream));
    HS_CUDA(cudaMemsetAsync(E->overflow, 0, 4, E->stream));
    HS_CUDA(cudaStreamSynchronize(E->stream));
    return HS_OK;
}

hs_status exact_add(hs_exact *E, const float *xyz, uint64_t n) {
    if (!E || (n && !xyz)) return fail(HS_ERR_ARG, "bad argument");
    if (n == 0) return HS_OK;
    if (!is_device_ptr(xyz)) return fail(HS_ERR_ARG, "xyz must be device memory");
    HS_CUDA(launch_exact_count(xyz, n, E->d, E->keys, E->counts, E->slots, E->overflow, E->stream));
    return HS_OK;
}

static hs_status exact_check(hs_exact *E) {
    uint32_t of = 0;
    HS_CUDA(cudaMemcpyAsync(&of, E->overflow, 4, cudaMemcpyDeviceToHost, E->stream));
    HS_CUDA(cudaStreamSynchronize(E->stream));
    if (of) return fail(HS_ERR_TABLE_FULL, "exact table: a key found no free slot in %d probes",
                        kTableProbes);
    return HS_OK;
}

hs_status exact_list(hs_exact *E, uint64_t *keys, int32_t *counts, uint64_t cap, uint64_t *n_out) {
    if (!E || !n_out || (cap && (!keys || !counts))) return fail(HS_ERR_ARG, "bad argument");
    hs_status st = exact_check(E);
    if (st != HS_OK) return st;
    cudaStream_t s = E->stream;
    const bool dev = cap && is_device_ptr(keys) && is_device_ptr(counts);
    uint64_t *dk = dev ? keys : nullptr;
    int32_t *dc = dev ? counts : nullptr;
    cudaError_t e = cudaSuccess;
    if (cap && !dev) {
        e = cudaMalloc(&dk, cap * 8);
        if (e == cudaSuccess) e = cudaMalloc(&dc, cap * 4);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(E->ctr, 0, 8, s);
    if (e == cudaSuccess) e = launch_table_list(E->keys, E->counts, E->slots, dk, dc, E->ctr, cap, s);
    unsigned long long nn = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nn, E->ctr, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const uint64_t m = std::min<uint64_t>(nn, cap);
    if (e == cudaSuccess && m && !dev) {
        e = cudaMemcpy(keys, dk, m * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(counts, dc, m * 4, cudaMemcpyDeviceToHost);
    }
    if (!dev) {
        if (dk) cudaFree(dk);
        if (dc) cudaFree(dc);
    }
    if (e != cudaSuccess) return fail(HS_ERR_CUDA, "exact_list: %s", cudaGetErrorString(e));
    *n_out = nn;
    return HS_OK;
}

hs_status exact_topk(hs_exact *E, uint32_t k, uint64_t *keys, int32_t *counts, uint32_t *n_out) {
    if (!E || !n_out || (k && (!keys || !counts))) return fail(HS_ERR_ARG, "bad argument");
    uint64_t D = 0;
    hs_status st = exact_list(E, nullptr, nullptr, 0, &D);
    if (st != HS_OK) return st;
    const uint64_t kk = std::min<uint64_t>(k, D);
    *n_out = 0;
    if (kk == 0) return HS_OK;
    if (E->out_cap < kk) {
        void *ps[] = {E->tmp_key, E->tmp_est, E->out_key, E->out_est, E->tmp_rank};
        for (void *q : ps)
            if (q) cudaFree(q);
        E->tmp_key = E->out_key = nullptr;
        E->tmp_est = E->out_est = nullptr;
        E->tmp_rank = nullptr;
        E->out_cap = 0;
        HS_CUDA(cudaMalloc(&E->tmp_key, kk * 8));
        HS_CUDA(cudaMalloc(&E->tmp_est, kk * 4));
        HS_CUDA(cudaMalloc(&E->tmp_rank, kk * 4));
        HS_CUDA(cudaMalloc(&E->out_key, kk * 8));
        HS_CUDA(cudaMalloc(&E->out_est, kk * 4));
        E->out_cap = kk;
    }
    // Rank every slot: empty slots carry count 0 and so rank below the kk-th
    // occupied one (its count is >= 1 because kk <= D).
    int launches = 0;
    const uint64_t *tk = reinterpret_cast<const uint64_t *>(E->keys);
    HS_CUDA(launch_select_kth(tk, E->counts, E->slots, kk, E->key_bits, E->sel, E->hist,
                              E->num_sms * 4, E->stream, &launches));
    HS_CUDA(launch_take_sorted(tk, E->counts, E->slots, E->sel, 0, E->tmp_key, E->tmp_est,
                               &E->ctr[1], E->tmp_rank, kk, E->out_key, E->out_est, E->num_sms * 4, E->stream,
                               &launches));
    HS_CUDA(cudaMemcpyAsync(keys, E->out_key, kk * 8, cudaMemcpyDefault, E->stream));
    HS_CUDA(cudaMemcpyAsync(counts, E->out_est, kk * 4, cudaMemcpyDefault, E->stream));
    HS_CUDA(cudaStreamSynchronize(E->stream));
    *n_out = (uint32_t)kk;
    return HS_OK;
}

hs_status exact_query(hs_exact *E, const uint64_t *keys, uint64_t m, int32_t *counts) {
    if (!E || (m && (!keys || !counts))) return fail(HS_ERR_ARG, "bad argument");
    if (m == 0) return HS_OK;
    hs_status st = exact_check(E);
    if (st != HS_OK) return st;
    const uint64_t *dk;
    uint64_t *tk = nullptr;
    st = device_input(keys, m, E->stream, &dk, &tk);
    if (st != HS_OK) return st;
    const bool dev_out = is_device_ptr(counts);
    int32_t *dc = counts;
    cudaError_t e = cudaSuccess;
    if (!dev_out) e = cudaMalloc(&dc, m * 4);
    if (e == cudaSuccess) e = launch_exact_query(E->keys, E->counts, E->slots, dk, m, dc, E->stream);
    if (e == cudaSuccess && !dev_out)
        e = cudaMemcpyAsync(counts, dc, m * 4, cudaMemcpyDeviceToHost, E->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
    if (tk) cudaFree(tk);
    if (!dev_out && dc) cudaFree(dc);
    if (e != cudaSuccess) return fail(HS_ERR_CUDA, "exact_query: %s", cudaGetErrorString(e));
    return HS_OK;
}

hs_status exact_counts(const float *xyz, uint64_t n, double box, double cell, uint32_t log2_slots,
                       void *cuda_stream, uint64_t *keys, int32_t *counts, uint64_t cap,
                       uint64_t *n_out) {
    if (!n_out || (n && !xyz)) return fail(HS_ERR_ARG, "bad argument");
    hs_exact *E = nullptr;
    hs_status st = exact_create(box, cell, log2_slots, cuda_stream, &E);
    if (st == HS_OK) st = exact_add(E, xyz, n);
    if (st == HS_OK) st = exact_list(E, keys, counts, keys ? cap : 0, n_out);
    exact_destroy(E);
    return st;
}

hs_status learned_destroy(hs_learned *L) {
    if (!L) return HS_OK;
    if (L->sk) sketch_destroy(L->sk);
    learned_free(L);
    delete L;
    return HS_OK;
}

hs_status learned_create(const hs_params *params, uint32_t coarse_factor, uint32_t table_log2,
                         uint64_t feature_seed, double feature_rate, void *cuda_stream,
                         hs_learned **out) {
    if (!out || !params) return fail(HS_ERR_ARG, "NULL argument");
    if (coarse_factor < 1 || coarse_factor > 64 || table_log2 < 4 || table_log2 > 32 ||
        !(feature_rate > 0 && feature_rate <= 1))
        return fail(HS_ERR_ARG, "bad coarse factor, table size or feature rate");
    const uint64_t R3 = (uint64_t)coarse_factor * coarse_factor * coarse_factor;
    const uint64_t max_blocks = (3ull << table_log2) / R3;   // 12-byte slots -> 4-byte counters
    if (max_blocks == 0) return fail(HS_ERR_ARG, "the table holds no block of R^3 counters");
    hs_sketch *sk = nullptr;
    hs_status st = sketch_create(params, cuda_stream, &sk);
    if (st != HS_OK) return st;
    if (sk->d.G % coarse_factor != 0 || sk->d.G > 65535 || sk->bl.slot == 0) {
        sketch_destroy(sk);
        return fail(HS_ERR_ARG, "the mesh must be a multiple of the coarse factor, below 2^16, "
                    "and the sketch must allow the binned update");
    }
    hs_learned *L = new (std::nothrow) hs_learned();
    if (!L) {
        sketch_destroy(sk);
        return fail(HS_ERR_OOM, "host allocation failed");
    }
    L->sk = sk;
    L->R = coarse_factor;
    L->Gc = sk->d.G / coarse_factor;
    L->ncoarse = (uint64_t)L->Gc * L->Gc * L->Gc;
    L->words = (L->ncoarse + 31) / 32;
    while (L->coarse_key_bits < 64 && (1ull << L->coarse_key_bits) < L->ncoarse) ++L->coarse_key_bits;
    L->feature_seed = feature_seed;
    L->feature_rate = feature_rate;
    L->max_blocks = max_blocks;
    cudaStream_t s = sk->stream;
    cudaError_t e = cudaMalloc(&L->coarse, L->ncoarse * 4);
    if (e == cudaSuccess) e = cudaMalloc(&L->routed, L->words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&L->prefix, L->words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&L->scan_scratch, (L->words / 1024 + 4096) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&L->blocks, max_blocks * R3 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&L->rlist, max_blocks * 8);
    if (e == cudaSuccess) e = cudaMalloc(&L->ctr, 4 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&L->ftab, kFeatTab * 2);
    if (e == cudaSuccess) {
        std::vector<uint16_t> t(kFeatTab);
        for (uint32_t c = 0; c < kFeatTab; ++c)
            t[c] = host_bf16((float)std::log10(1.0 + (double)c));   // double -> float -> bf16
        e = cudaMemcpy(L->ftab, t.data(), kFeatTab * 2, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(L->routed, 0, L->words * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->prefix, 0, L->words * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->blocks, 0, max_blocks * R3 * 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        learned_destroy(L);
        return fail(HS_ERR_OOM, "learned_create: %s", cudaGetErrorString(e));
    }
    sk->route.filter = RouteFilter{L->routed, (uint32_t)((0x100000000ull + coarse_factor - 1) / coarse_factor),
                                   L->Gc, coarse_factor};
    sk->route.prefix = L->prefix;
    sk->route.blocks = L->blocks;
    sk->min_cap = max_blocks * R3;
    *out = L;
    return HS_OK;
}

hs_status learned_capacity(hs_learned *L, uint64_t *max_routed, uint64_t *table_bytes) {
    if (!L) return fail(HS_ERR_ARG, "NULL handle");
    if (max_routed) *max_routed = L->max_blocks;
    if (table_bytes) *table_bytes = L->max_blocks * L->R * L->R * L->R * 4;
    return HS_OK;
}

hs_status learned_sample(hs_learned *L, const float *xyz, uint64_t n) {
    if (!L || (n && !xyz)) return fail(HS_ERR_ARG, "NULL argument");
    hs_sketch *sk = L->sk;
    cudaStream_t s = sk->stream;
    if (L->n_sampled == 0) HS_CUDA(cudaMemsetAsync(L->coarse, 0, L->ncoarse * 4, s));
    if (n == 0) return HS_OK;
    if (is_device_ptr(xyz)) {
        HS_CUDA(launch_coarse_hist(xyz, n, L->n_sampled, sk->d, L->R, L->Gc, L->feature_seed,
                                   L->feature_rate, L->coarse, s));
        sk->stats.kernel_launches += 1;
    } else {   // through the sketch's staging buffers, as sketch_update does
        hs_status st = ensure_staging(sk);
        if (st != HS_OK) return st;
        int i = 0;
        for (uint64_t off = 0; off < n; off += kStageParticles, ++i) {
            const uint64_t cnt = std::min(kStageParticles, n - off);
            const int b = i % kStageBuffers;
            HS_CUDA(cudaStreamWaitEvent(sk->copy_stream, sk->ev_free[b], 0));
            HS_CUDA(cudaMemcpyAsync(sk->stage[b], xyz + 3 * off, cnt * 12, cudaMemcpyHostToDevice,
                                    sk->copy_stream));
            HS_CUDA(cudaEventRecord(sk->ev_copied[b], sk->copy_stream));
            HS_CUDA(cudaStreamWaitEvent(s, sk->ev_copied[b], 0));
            HS_CUDA(launch_coarse_hist(sk->stage[b], cnt, L->n_sampled + off, sk->d, L->R, L->Gc,
                                       L->feature_seed, L->feature_rate, L->coarse, s));
            HS_CUDA(cudaEventRecord(sk->ev_free[b], s));
            sk->stats.kernel_launches += 1;
        }
    }
    L->n_sampled += n;
    return HS_OK;
}

hs_status learned_route(hs_learned *L, hs_mlp *mlp, uint64_t *n_routed) {
    if (!L || !mlp) return fail(HS_ERR_ARG, "NULL argument");
    hs_sketch *sk = L->sk;
    cudaStream_t s = sk->stream;
    int launches = 0;
    if (L->n_sampled == 0) HS_CUDA(cudaMemsetAsync(L->coarse, 0, L->ncoarse * 4, s));
    L->n_sampled = 0;                     // the next learned_sample starts a new histogram
    HS_CUDA(cudaMemsetAsync(L->ctr, 0, 4 * 8, s));
    // list the coarse cells with a sample (size known only on the device: count first)
    HS_CUDA(launch_coarse_list(L->coarse, L->ncoarse, nullptr, &L->ctr[0], 0, s));
    unsigned long long nl = 0;
    HS_CUDA(cudaMemcpyAsync(&nl, &L->ctr[0], 8, cudaMemcpyDeviceToHost, s));
    HS_CUDA(cudaStreamSynchronize(s));
    if (nl > L->clist_cap) {
        void *old[] = {L->clist, L->feats, L->logits, L->lrank};
        for (void *q : old)
            if (q) cudaFree(q);
        L->clist = nullptr;
        L->feats = nullptr;
        L->logits = nullptr;
        L->lrank = nullptr;
        L->clist_cap = std::max<uint64_t>(nl, 1024);
        HS_CUDA(cudaMalloc(&L->clist, L->clist_cap * 8));
        HS_CUDA(cudaMalloc(&L->feats, L->clist_cap * kMlpIn * 2));
        HS_CUDA(cudaMalloc(&L->logits, L->clist_cap * 4));
        HS_CUDA(cudaMalloc(&L->lrank, L->clist_cap * 4));
    }
    HS_CUDA(cudaMemsetAsync(&L->ctr[0], 0, 8, s));
    HS_CUDA(launch_coarse_list(L->coarse, L->ncoarse, L->clist, &L->ctr[0], L->clist_cap, s));
    HS_CUDA(launch_features(L->coarse, L->Gc, L->clist, nl, L->ftab, kFeatTab, L->feats, s));
    HS_CUDA(launch_mlp_forward(mlp->P, L->feats, nl, L->logits, s));
    HS_CUDA(launch_logit_rank(L->logits, nl, L->lrank, &L->ctr[1], s));
    unsigned long long npos = 0;
    HS_CUDA(cudaMemcpyAsync(&npos, &L->ctr[1], 8, cudaMemcpyDeviceToHost, s));
    HS_CUDA(cudaStreamSynchronize(s));
    launches += 5;
    // over budget: keep the max_blocks cells of largest logit (ties: smaller key)
    const int use_sel = npos > L->max_blocks;
    if (use_sel) {
        hs_status st = ensure_topk_scratch(sk, 1);
        if (st != HS_OK) return st;
        HS_CUDA(launch_select_kth(L->clist, L->lrank, nl, L->max_blocks, L->coarse_key_bits,
                                  sk->sel, sk->hist, sk->num_sms * 4, s, &launches));
    }
    HS_CUDA(cudaMemsetAsync(L->routed, 0, L->words * 4, s));
    HS_CUDA(launch_route(L->clist, L->lrank, nl, use_sel ? sk->sel : nullptr, use_sel, L->routed, s));
    HS_CUDA(launch_word_popc(L->routed, L->words, L->prefix, s));
    HS_CUDA(launch_exclusive_scan(L->prefix, L->prefix, L->words, L->scan_scratch, s, &launches));
    HS_CUDA(launch_route_list(L->clist, nl, L->routed, L->prefix, L->rlist, s));
    const uint64_t nr = use_sel ? L->max_blocks : npos;
    const uint64_t R3 = (uint64_t)L->R * L->R * L->R;
    HS_CUDA(cudaMemsetAsync(L->blocks, 0, L->max_blocks * R3 * 4, s));
    HS_CUDA(cudaStreamSynchronize(s));
    launches += 3;
    sk->stats.kernel_launches += launches;
    L->n_list = nl;
    L->n_routed = nr;
    sk->routing = true;
    if (n_routed) *n_routed = nr;
    return HS_OK;
}

hs_status learned_prepare(hs_learned *L, const float *xyz, uint64_t n, hs_mlp *mlp,
                          uint64_t *n_routed) {
    if (!L || !mlp || (n && !xyz)) return fail(HS_ERR_ARG, "NULL argument");
    L->n_sampled = 0;
    hs_status st = learned_sample(L, xyz, n);
    if (st != HS_OK) return st;
    return learned_route(L, mlp, n_routed);
}

hs_status learned_update(hs_learned *L, const float *xyz, uint64_t n, double sample_rate) {
    if (!L) return fail(HS_ERR_ARG, "NULL handle");
    if (!L->sk->routing) return fail(HS_ERR_STATE, "call learned_prepare first");
    return sketch_update(L->sk, xyz, n, sample_rate);
}

hs_status learned_topk(hs_learned *L, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out) {
    if (!L || k == 0 || !keys || !est || !n_out) return fail(HS_ERR_ARG, "bad argument");
    hs_sketch *h = L->sk;
    uint32_t n1 = 0;
    hs_status st = topk_extract(h, k, keys, est, &n1);   // leaves the ranking in h->out_*
    if (st != HS_OK) return st;
    // candidates: the sketch's ranking, then every non-zero exact counter
    HS_CUDA(cudaMemcpyAsync(h->cand_key, h->out_key, n1 * 8, cudaMemcpyDeviceToDevice, h->stream));
    HS_CUDA(cudaMemcpyAsync(h->cand_est, h->out_est, n1 * 4, cudaMemcpyDeviceToDevice, h->stream));
    HS_CUDA(cudaMemsetAsync(&L->ctr[2], 0, 8, h->stream));
    HS_CUDA(launch_block_list(L->blocks, L->rlist, L->n_routed, L->R, L->Gc, h->d.G,
                              h->cand_key + n1, h->cand_est + n1, &L->ctr[2], h->cap - n1,
                              h->stream));
    unsigned long long nt = 0;
    HS_CUDA(cudaMemcpyAsync(&nt, &L->ctr[2], 8, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    h->stats.kernel_launches += 1;
    if (nt > h->cap - n1) return fail(HS_ERR_STATE, "too many exact counts for the candidates");
    const uint64_t m = n1 + nt;
    const uint64_t kk = std::min<uint64_t>(k, m);
    if (m == 0) {
        *n_out = 0;
        return HS_OK;
    }
    st = finalize(h, m, kk);
    if (st != HS_OK) return st;
    HS_CUDA(cudaMemcpyAsync(keys, h->out_key, kk * 8, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaMemcpyAsync(est, h->out_est, kk * 4, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    *n_out = (uint32_t)kk;
    return HS_OK;
}

hs_status learned_table(hs_learned *L, uint64_t *keys, int32_t *counts, uint64_t cap,
                        uint64_t *n_out) {
    if (!L || !n_out || (cap && (!keys || !counts))) return fail(HS_ERR_ARG, "bad argument");
    cudaStream_t s = L->sk->stream;
    hs_status st = drain(L->sk);
    if (st != HS_OK) return st;
    uint64_t *dk = nullptr;
    int32_t *dc = nullptr;
    if (cap) {
        HS_CUDA(cudaMalloc(&dk, cap * 8));
        HS_CUDA(cudaMalloc(&dc, cap * 4));
    }
    HS_CUDA(cudaMemsetAsync(&L->ctr[2], 0, 8, s));
    HS_CUDA(launch_block_list(L->blocks, L->rlist, L->n_routed, L->R, L->Gc, L->sk->d.G, dk, dc,
                              &L->ctr[2], cap, s));
    unsigned long long nt = 0;
    HS_CUDA(cudaMemcpyAsync(&nt, &L->ctr[2], 8, cudaMemcpyDeviceToHost, s));
    HS_CUDA(cudaStreamSynchronize(s));
    uint64_t m = std::min<uint64_t>(nt, cap);
    cudaError_t e = cudaSuccess;
    if (m) {
        e = cudaMemcpy(keys, dk, m * 8, cudaMemcpyDefault);
        if (e == cudaSuccess) e = cudaMemcpy(counts, dc, m * 4, cudaMemcpyDefault);
    }
    if (dk) cudaFree(dk);
    if (dc) cudaFree(dc);
    if (e != cudaSuccess) return fail(HS_ERR_CUDA, "learned_table: %s", cudaGetErrorString(e));
    *n_out = nt;
    return HS_OK;
}

hs_status learned_routed(hs_learned *L, uint64_t *coarse_keys, uint64_t cap, uint64_t *n_out) {
    if (!L || !n_out || (cap && !coarse_keys)) return fail(HS_ERR_ARG, "bad argument");
    uint64_t m = std::min<uint64_t>(L->n_routed, cap);
    if (m) HS_CUDA(cudaMemcpy(coarse_keys, L->rlist, m * 8, cudaMemcpyDefault));
    *n_out = L->n_routed;
    return HS_OK;
}

hs_status learned_logits(hs_learned *L, uint64_t *coarse_keys, float *logits, uint64_t cap,
                         uint64_t *n_out) {
    if (!L || !n_out) return fail(HS_ERR_ARG, "bad argument");
    uint64_t m = std::min<uint64_t>(L->n_list, cap);
    if (m) {
        HS_CUDA(cudaMemcpy(coarse_keys, L->clist, m * 8, cudaMemcpyDefault));
        HS_CUDA(cudaMemcpy(logits, L->logits, m * 4, cudaMemcpyDefault));
    }
    *n_out = L->n_list;
    return HS_OK;
}

hs_status learned_coarse_counts(hs_learned *L, int32_t *out) {
    if (!L || !out) return fail(HS_ERR_ARG, "bad argument");
    HS_CUDA(cudaMemcpyAsync(out, L->coarse, L->ncoarse * 4, cudaMemcpyDefault, L->sk->stream));
    HS_CUDA(cudaStreamSynchronize(L->sk->stream));
    return HS_OK;
}

hs_status learned_features(hs_learned *L, uint16_t *feats, uint64_t cap, uint64_t *n_out) {
    if (!L || !n_out) return fail(HS_ERR_ARG, "bad argument");
    uint64_t m = std::min<uint64_t>(L->n_list, cap);
    if (m) HS_CUDA(cudaMemcpy(feats, L->feats, m * kMlpIn * 2, cudaMemcpyDefault));
    *n_out = L->n_list;
    return HS_OK;
}

hs_status learned_sketch(hs_learned *L, hs_sketch **out) {
    if (!L || !out) return fail(HS_ERR_ARG, "bad argument");
    *out = L->sk;
    return HS_OK;
}

hs_status learned_reset(hs_learned *L) {
    if (!L) return fail(HS_ERR_ARG, "NULL handle");
    hs_status st = sketch_reset(L->sk);
    if (st != HS_OK) return st;
    const uint64_t R3 = (uint64_t)L->R * L->R * L->R;
    HS_CUDA(cudaMemsetAsync(L->blocks, 0, L->max_blocks * R3 * 4, L->sk->stream));
    return HS_OK;
}

}  // extern "C"
