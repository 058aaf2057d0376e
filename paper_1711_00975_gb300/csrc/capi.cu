// capi.cu - the library's C ABI (include/halosketch.h): handle lifetime, the
// update path (device buffers directly, host buffers through double-buffered
// staging), point queries and the exact full-search top-k.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
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
constexpr uint64_t kStageParticles = 1ull << 23;  // 96 MiB per staging buffer
constexpr size_t kSearchSmemBudget = 192 * 1024;
constexpr size_t kBinSmemBudget = 224 * 1024;
constexpr uint64_t kBinBudgetBytes = 4ull << 30;   // global bins, at most
constexpr double kBinnedMinUpdates = 1 << 20;      // smaller calls add directly

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
    float *stage[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_free[2] = {nullptr, nullptr};

    // top-k scratch
    uint64_t cap = 0;               // candidate capacity
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

    // binned update: codes waiting in global bins until the next drain
    BinLayout bl{};
    uint16_t *bins = nullptr;
    uint32_t *bin_cursor = nullptr;
    uint32_t bin_cap = 0;
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
                  h->out_key, h->out_est};
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
    h->out_key = nullptr;
    h->out_est = nullptr;
    h->cap = 0;
    h->out_cap = 0;
}

hs_status ensure_topk_scratch(hs_sketch *h, uint64_t k) {
    uint64_t want_cap = std::max<uint64_t>(1ull << 22, 8 * k);
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
    for (int i = 0; i < 2; ++i) {
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
                               double rate);

// add every binned code to the counters (before anything reads them)
hs_status drain(hs_sketch *h) {
    if (h->pending <= 0) return HS_OK;
    EventPair ev = take_events(h);
    cudaEventRecord(ev.a, h->stream);
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
    return HS_OK;
}

bool want_binned(hs_sketch *h, uint64_t n, double rate) {
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

hs_status launch_update_timed(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                              double rate) {
    if (want_binned(h, n, rate)) {
        hs_status st = ensure_bins(h, n, rate);
        if (st != HS_OK) return st;
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
                HS_CUDA(launch_bin_scatter(xyz + 3 * off, cnt, g0 + off, h->d, h->C, rate,
                                           h->p.sample_seed, h->probe, h->probe_base, kProbeCap,
                                           h->bl, h->bins,
                                           h->bin_cursor, h->bin_cap, h->num_sms, h->stream));
                cudaEventRecord(ev.b, h->stream);
                h->pending_update.push_back(ev);
                h->pending += (double)cnt * rate;
                h->stats.update_launches += 1;
                h->stats.kernel_launches += 1;
            }
            return HS_OK;
        }
    }
    return launch_update_direct(h, xyz, n, g0, rate);
}

hs_status launch_update_direct(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                               double rate) {
    EventPair ev = take_events(h);
    cudaEventRecord(ev.a, h->stream);
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
    // relative costs: one scanned cell ~ 1; one (cx, hot bucket) query ~ 20
    // units per directory line it reads; building a directory ~ 60 units/line
    const double per_slot = (double)lines / (double)(1ull << h->dir_D);
    double cost_dir = 0, cost_scan = (double)G * G * G;
    for (uint32_t r = 0; r < F; ++r) {
        if (cnt[r] > h->hot_cap) return HS_OK;
        cost_dir += 20.0 * (double)G * (double)cnt[r] * (2.0 + 2.0 * per_slot);
        if (!h->dir_off[r] || h->dir_G[r] != h->d.G) cost_dir += 60.0 * (double)lines;
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
                                 line_lo, line_hi, out, h->num_sms * 16, h->stream));
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
        EventPair ev = take_events(h);
        cudaEventRecord(ev.a, h->stream);
        HS_CUDA(launch_full_search(h->C, h->d, theta, mode, h->bitmap, h->nb, prune, line_lo,
                                   line_hi, out, h->num_sms, h->stream));
        cudaEventRecord(ev.b, h->stream);
        h->pending_search.push_back(ev);
        h->stats.search_launches += 1;
        h->stats.kernel_launches += 1;
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
                               &h->counters[1], n_take, h->out_key, h->out_est, h->num_sms * 4,
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
    free_topk_scratch(h);
    free_dir(h);
    if (h->bins) cudaFree(h->bins);
    if (h->bin_cursor) cudaFree(h->bin_cursor);
    if (h->C && !h->is_view) cudaFree(h->C);
    if (h->probe && !h->is_view) cudaFree(h->probe);
    if (h->q_keys) cudaFree(h->q_keys);
    if (h->q_est) cudaFree(h->q_est);
    if (h->flags) cudaFree(h->flags);
    for (int i = 0; i < 2; ++i) {
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

hs_status sketch_update(hs_sketch *h, const float *xyz, uint64_t n, double sample_rate) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (!(sample_rate > 0.0 && sample_rate <= 1.0))
        return fail(HS_ERR_ARG, "sample_rate=%g outside (0, 1]", sample_rate);
    if (n == 0) return HS_OK;
    if (!xyz) return fail(HS_ERR_ARG, "xyz is NULL");
    if (n > (~0ull - h->n_seen)) return fail(HS_ERR_ARG, "particle index overflow");
    if (is_device_ptr(xyz)) {
        hs_status st = launch_update_timed(h, xyz, n, h->n_seen, sample_rate);
        if (st != HS_OK) return st;
    } else {
        hs_status st = ensure_staging(h);
        if (st != HS_OK) return st;
        int i = 0;
        for (uint64_t off = 0; off < n; off += kStageParticles, ++i) {
            uint64_t cnt = std::min(kStageParticles, n - off);
            int b = i & 1;
            HS_CUDA(cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0));
            HS_CUDA(cudaMemcpyAsync(h->stage[b], xyz + 3 * off, cnt * 12, cudaMemcpyHostToDevice,
                                    h->copy_stream));
            HS_CUDA(cudaEventRecord(h->ev_copied[b], h->copy_stream));
            HS_CUDA(cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
            st = launch_update_timed(h, h->stage[b], cnt, h->n_seen + off, sample_rate);
            if (st != HS_OK) return st;
            HS_CUDA(cudaEventRecord(h->ev_free[b], h->stream));
        }
    }
    h->n_seen += n;
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

hs_status topk_extract(hs_sketch *h, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (k == 0 || !keys || !est || !n_out) return fail(HS_ERR_ARG, "k == 0 or NULL output");
    const uint64_t kk = std::min<uint64_t>(k, h->n_cells);
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
    uint64_t m_probe = std::min<uint64_t>(h->n_seen - h->probe_base, h->probe_cap);
    if (m_probe >= kk) {
        HS_CUDA(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned long long), h->stream));
        HS_CUDA(cudaMemsetAsync(h->flags, 0, 4 * sizeof(uint32_t), h->stream));
        HS_CUDA(launch_probe_distinct(h->probe, m_probe, h->slots, kProbeSlotsLog2, h->distinct,
                                      &h->counters[2], &h->flags[1], h->stream));
        unsigned long long nd = 0;
        HS_CUDA(cudaMemcpyAsync(&nd, &h->counters[2], 8, cudaMemcpyDeviceToHost, h->stream));
        HS_CUDA(cudaStreamSynchronize(h->stream));
        h->stats.kernel_launches += 1;
        if (nd >= kk) {
            HS_CUDA(launch_point_query(h->C, h->d, h->distinct, nd, h->distinct_est, &h->flags[0],
                                       h->stream));
            h->stats.kernel_launches += 1;
            st = kth_estimate(h, h->distinct, h->distinct_est, nd, kk, &theta);
            if (st != HS_OK) return st;
        }
    }

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
    return HS_OK;
}

hs_status sketch_flush(hs_sketch *h) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    return drain(h);
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
    hs_sketch *view = nullptr;          // top-k of one volume at a time
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
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_a);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_b);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->C, 0, counters * 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->probe, 0xFF, (size_t)n_volumes * kBatchProbe * 8, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->cursor, 0, (size_t)b->bl.nbins * 4, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) {
        hs_sketch *h = new (std::nothrow) hs_sketch();
        if (!h) e = cudaErrorMemoryAllocation;
        else {
            h->p = p;
            h->d = b->d;
            h->is_view = true;
            h->stream = b->stream;
            h->device = b->device;
            h->num_sms = b->num_sms;
            h->probe_cap = kBatchProbe;
            h->bl = BinLayout{};        // views never bin
            std::memset(&h->stats, 0, sizeof(h->stats));
            e = cudaMalloc(&h->flags, 4 * sizeof(uint32_t));
            b->view = h;
        }
    }
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
    if (b->view) {
        b->view->C = nullptr;
        b->view->probe = nullptr;
        sketch_destroy(b->view);
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

hs_status batch_topk(hs_batch *b, uint32_t k, uint64_t *keys, int32_t *est, uint32_t *n_out) {
    if (!b) return fail(HS_ERR_ARG, "batch is NULL");
    if (k == 0 || !keys || !est || !n_out) return fail(HS_ERR_ARG, "k == 0 or NULL output");
    hs_sketch *h = b->view;
    const uint32_t F = enum_rows(h);
    if (b->vdir_off.size() != (size_t)b->nvol * F) {
        b->vdir_off.assign((size_t)b->nvol * F, nullptr);
        b->vdir_rec.assign((size_t)b->nvol * F, nullptr);
        b->vdir_G.assign((size_t)b->nvol * F, 0);
        b->vdir_cap.assign((size_t)b->nvol * F, 0);
    }
    for (uint32_t v = 0; v < b->nvol; ++v) {
        for (uint32_t r = 0; r < F; ++r) {     // lend volume v's directories to the view
            h->dir_off[r] = b->vdir_off[v * F + r];
            h->dir_rec[r] = b->vdir_rec[v * F + r];
            h->dir_G[r] = b->vdir_G[v * F + r];
            h->dir_lines_cap[r] = b->vdir_cap[v * F + r];
        }
        h->C = b->C + (size_t)v * b->d.rows * b->d.W;
        h->probe = b->probe + (size_t)v * kBatchProbe;
        h->d.G = b->G[v];
        h->d.inv_cell = b->inv[v];
        h->n_cells = (uint64_t)b->G[v] * b->G[v] * b->G[v];
        h->key_bits = 1;
        while (h->key_bits < 64 && (1ull << h->key_bits) < h->n_cells) ++h->key_bits;
        h->n_seen = b->n_seen[v];
        h->probe_base = b->probe_base[v];
        hs_status st = topk_extract(h, k, keys + (size_t)v * k, est + (size_t)v * k, &n_out[v]);
        for (uint32_t r = 0; r < F; ++r) {     // keep what the view built
            b->vdir_off[v * F + r] = h->dir_off[r];
            b->vdir_rec[v * F + r] = h->dir_rec[r];
            b->vdir_G[v * F + r] = h->dir_G[r];
            b->vdir_cap[v * F + r] = h->dir_lines_cap[r];
            h->dir_off[r] = nullptr;
            h->dir_rec[r] = nullptr;
            h->dir_G[r] = 0;
            h->dir_lines_cap[r] = 0;
        }
        if (st != HS_OK) return st;
    }
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
    hs_stats vs{};
    sketch_stats(b->view, &vs, reset);
    *out = b->stats;
    out->kernel_launches += vs.kernel_launches;
    out->search_launches = vs.search_launches;
    out->search_ms = vs.search_ms;
    out->topk_ms = vs.topk_ms;
    out->topk_calls = vs.topk_calls;
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
