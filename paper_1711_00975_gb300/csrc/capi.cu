// capi.cu - the library's C ABI (include/halosketch.h), single sketches:
// handle lifetime, the update path (device buffers directly, host buffers
// through staged copies), point queries, the exact full-search top-k and the
// hierarchical query.  Batches, the no-allocation query and the learned
// router live in capi_batch.cu, capi_noalloc.cu and capi_learned.cu.
#include <atomic>
#include <mutex>
#include <thread>

#include "capi_internal.h"

namespace hs {
namespace capi {

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


// The device address of page-locked host memory (nullptr for anything else).
const void *pinned_device_view(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

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
                           HS_FLAG_UPDATE_BINNED | HS_FLAG_DIR_INLINE;
    if ((p->flags & ~known) != 0 || p->reserved != 0)
        return fail(HS_ERR_ARG, "unknown flags or reserved != 0");
    if ((p->flags & HS_FLAG_SEARCH_SCAN) && (p->flags & HS_FLAG_SEARCH_DIRECTORY))
        return fail(HS_ERR_ARG, "at most one search method may be forced");
    if ((p->flags & HS_FLAG_UPDATE_DIRECT) && (p->flags & HS_FLAG_UPDATE_BINNED))
        return fail(HS_ERR_ARG, "at most one update method may be forced");
    return HS_OK;
}

// An event pair for timing one launch: from the pool, else newly created.
// Lists of pairs still waiting to be folded into the stats are bounded: past
// kMaxPendingEvents entries the older half is waited for and folded, so a long
// loop of updates and point queries neither grows them nor creates events
// without end.
hs_status take_events(hs_sketch *h, EventPair *out) {
    for (auto *v : {&h->pending_update, &h->pending_search, &h->pending_flush, &h->pending_copy}) {
        if (v->size() < kMaxPendingEvents) continue;
        const size_t half = v->size() / 2;
        HS_CUDA(cudaEventSynchronize((*v)[half - 1].b));
        for (size_t i = 0; i < half; ++i) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, (*v)[i].a, (*v)[i].b) == cudaSuccess) {
                if (v == &h->pending_search) h->stats.search_ms += ms;
                else if (v == &h->pending_copy) h->stats.h2d_ms += ms;
                else h->stats.update_ms += ms;
                if (v == &h->pending_flush) h->stats.flush_ms += ms;
            }
            h->pool.push_back((*v)[i]);
        }
        v->erase(v->begin(), v->begin() + (ptrdiff_t)half);
        cudaGetLastError();
    }
    if (!h->pool.empty()) {
        *out = h->pool.back();
        h->pool.pop_back();
        return HS_OK;
    }
    EventPair e{nullptr, nullptr};
    cudaError_t err = cudaEventCreate(&e.a);
    if (err == cudaSuccess) {
        err = cudaEventCreate(&e.b);
        if (err != cudaSuccess) cudaEventDestroy(e.a);
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(HS_ERR_CUDA, "cudaEventCreate failed: %s", cudaGetErrorString(err));
    }
    *out = e;
    return HS_OK;
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
    for (auto &e : h->pending_copy) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) h->stats.h2d_ms += ms;
        h->pool.push_back(e);
    }
    h->pending_copy.clear();
    cudaGetLastError();
}

// A top-k list must be strictly ranked (estimate desc, key asc): each
// candidate is placed at the count of candidates ranked before it, so two
// equal candidates would share a slot and leave another one stale.  Checked on
// the host copy of every list before it is returned.
hs_status check_ranked(const uint64_t *keys, const int32_t *est, uint64_t n) {
    for (uint64_t i = 1; i < n; ++i) {
        const bool before = est[i - 1] > est[i] || (est[i - 1] == est[i] && keys[i - 1] < keys[i]);
        if (!before)
            return fail(HS_ERR_STATE, "top-k entries %llu and %llu are not strictly ranked",
                        (unsigned long long)(i - 1), (unsigned long long)i);
    }
    return HS_OK;
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
    HS_CUDA(cudaMalloc(&h->xbits, (size_t)h->d.rows * wpr * 4 * 2));   // signed maps
    HS_CUDA(cudaMalloc(&h->hot_list, (size_t)enum_rows(h) * h->hot_cap * 4));
    HS_CUDA(cudaMalloc(&h->hot_cnt, kMaxRows * sizeof(unsigned long long)));
    HS_CUDA(cudaMalloc(&h->dir_cursor, (nslots + 1) * 4));
    HS_CUDA(cudaMalloc(&h->scan_scratch, (nslots / 1024 + 4096) * 4));
    return HS_OK;
}

// build the directory of row r (once per mesh; the buffers are reused when a
// batch view moves to a mesh whose directory fits them); false when memory is
// short
bool ensure_dir(hs_sketch *h, int r) {
    uint64_t lines = (uint64_t)h->d.G * h->d.G;
    const bool force = (h->p.flags & HS_FLAG_DIR_INLINE) != 0;
    if (h->dir_off[r] && h->dir_G[r] == h->d.G) return true;
    if (h->dir_off[r] && (h->dir_lines_cap[r] < lines || dir_bytes(h->dir_G[r], h->dir_D, force) <
                                                             dir_bytes(h->d.G, h->dir_D, force))) {
        cudaFree(h->dir_off[r]);
        cudaFree(h->dir_rec[r]);
        h->dir_off[r] = nullptr;
        h->dir_rec[r] = nullptr;
    }
    if (!h->dir_off[r]) {
        if (cudaMalloc(&h->dir_off[r], dir_bytes(h->d.G, h->dir_D, force)) != cudaSuccess ||
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
    cudaError_t e = launch_dir_build(h->d, r, h->dir_D, dir_has_inline(h->d.G, h->dir_D, force),
                                     h->dir_off[r], h->dir_cursor, h->dir_rec[r], h->scan_scratch,
                                     h->num_sms * 8, h->stream, &launches);
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


uint32_t region_capacity(double mean, uint32_t half, double pad_halves) {
    const double c = 1.08 * mean + 8.0 * std::sqrt(mean) + 64.0 + (pad_halves + 1.0) * half;
    const double most = 4294967040.0;
    return (uint32_t)((std::min(c, most) + 15.0) / 16.0) * 16u;
}

hs_status alloc_bins(BinBuffers &bb, const std::vector<uint32_t> &caps, uint32_t bpg,
                     uint32_t nblocks, cudaStream_t s) {
    free_bins(bb);
    const size_t ng = caps.size();
    if (ng == 0 || ng > kMaxBinGroups) return fail(HS_ERR_ARG, "%zu region groups (at most %u)", ng, kMaxBinGroups);
    std::vector<uint64_t> base(ng);
    uint64_t total = 0;
    uint32_t lo = 0xFFFFFFFFu;
    for (size_t g = 0; g < ng; ++g) {
        base[g] = total;
        total += (uint64_t)caps[g] * bpg * nblocks;
        lo = std::min(lo, caps[g]);
    }
    HS_CUDA(cudaMalloc(&bb.codes, std::max<uint64_t>(total, 8) * 2));
    HS_CUDA(cudaMalloc(&bb.gbase, ng * 8));
    HS_CUDA(cudaMalloc(&bb.gcap, ng * 4));
    HS_CUDA(cudaMalloc(&bb.fill, ng * bpg * nblocks * 4));
    HS_CUDA(cudaMemcpyAsync(bb.gbase, base.data(), ng * 8, cudaMemcpyHostToDevice, s));
    HS_CUDA(cudaMemcpyAsync(bb.gcap, caps.data(), ng * 4, cudaMemcpyHostToDevice, s));
    HS_CUDA(cudaMemsetAsync(bb.fill, 0, ng * bpg * nblocks * 4, s));
    HS_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
    bb.nblocks = nblocks;
    bb.bpg = bpg;
    bb.ngroups = (uint32_t)ng;
    bb.min_cap = lo;
    return HS_OK;
}

void free_bins(BinBuffers &bb) {
    void *ps[] = {bb.codes, bb.fill, bb.gbase, bb.gcap};
    for (void *p : ps)
        if (p) cudaFree(p);
    bb = BinBuffers{};
}

// add every binned code to the counters (before anything reads them)
hs_status drain(hs_sketch *h) {
    if (h->pending <= 0) return HS_OK;
    EventPair ev;
    HS_TRY(take_events(h, &ev));
    cudaEventRecord(ev.a, h->stream);
    HS_CUDA(launch_bin_accumulate(h->bl, h->bb.store(), h->C, h->stream));
    cudaEventRecord(ev.b, h->stream);
    h->pending_flush.push_back(ev);
    h->stats.kernel_launches += 1;
    h->stats.flush_launches += 1;
    h->pending = 0;
    return HS_OK;
}

// drop binned codes that were never drained (reset / load)
hs_status discard_pending(hs_sketch *h) {
    if (h->pending > 0 && h->bb.fill)
        HS_CUDA(cudaMemsetAsync(h->bb.fill, 0, (size_t)h->bl.nbins * h->bb.nblocks * 4, h->stream));
    h->pending = 0;
    return HS_OK;
}

bool want_binned(hs_sketch *h, uint64_t n, double rate) {
    if (h->routing) return true;          // only the binned scatter routes
    if (h->p.flags & HS_FLAG_UPDATE_DIRECT) return false;
    if (h->bl.slot == 0) return false;
    if (h->p.flags & HS_FLAG_UPDATE_BINNED) return true;
    return (double)n * rate * h->d.rows >= kBinnedMinUpdates;
}

// Regions sized for a call of n particles in `launches` scatter launches (a
// host buffer is staged in pieces, each its own launch).  Every bin of a plain
// sketch receives the same expected share.
hs_status ensure_bins(hs_sketch *h, uint64_t n, double rate, uint64_t launches) {
    if (h->bb.codes) return HS_OK;
    const uint32_t nblocks = (uint32_t)h->num_sms;
    const double per_region = (double)n * rate * h->d.rows / ((double)h->bl.nbins * nblocks);
    uint32_t cap = region_capacity(per_region, h->bl.half, (double)launches);
    const uint64_t most = kBinBudgetBytes / (2ull * h->bl.nbins * nblocks);
    cap = (uint32_t)std::min<uint64_t>(cap, most & ~15ull);
    cap = std::max<uint32_t>(cap, std::max<uint32_t>(4 * h->bl.slot, 1024));
    HS_TRY(alloc_bins(h->bb, std::vector<uint32_t>(1, cap), h->bl.nbins, nblocks, h->stream));
    // drain before the expected fill of a region comes within 8 standard
    // deviations and 64 codes of its capacity
    const double c = (double)cap;
    h->pending_limit = std::max(0.0, c - 8.0 * std::sqrt(c) - 64.0);
    return HS_OK;
}

// Regions for a call of n particles at `rate`: regions sized for a smaller
// call are drained and grown for this one.
static hs_status size_regions(hs_sketch *h, uint64_t n, double rate) {
    if (h->bb.codes) {
        const double mean = (double)n * rate * h->d.rows / ((double)h->bl.nbins * h->bb.nblocks);
        if (region_capacity(mean, h->bl.half, 1.0) > h->bb.min_cap && !h->routing) {
            HS_TRY(drain(h));
            HS_CUDA(cudaStreamSynchronize(h->stream));
            free_bins(h->bb);
        }
    }
    return ensure_bins(h, n, rate);
}

// xyz: float32 positions, or packed 64-bit records when packed is set
hs_status launch_update_timed(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                              double rate, bool packed) {
    const size_t esz = packed ? 8 : 12;
    if (want_binned(h, n, rate)) {
        HS_TRY(size_regions(h, n, rate));
        // expected codes per region of one particle; each launch adds at most
        // one partial half (padded) per region
        const double per = rate * h->d.rows / ((double)h->bl.nbins * h->bb.nblocks);
        const double room = h->pending_limit - h->bl.half;
        if (room < 1.0) {
            if (h->routing) return fail(HS_ERR_STATE, "routing needs regions of useful capacity");
            return launch_update_direct(h, xyz, n, g0, rate, packed);
        }
        const uint64_t piece = std::max<uint64_t>(4, (uint64_t)std::floor(room / per) & ~3ull);
        for (uint64_t off = 0; off < n; off += piece) {
            const uint64_t cnt = std::min(piece, n - off);
            const double add = (double)cnt * per + h->bl.half;
            if (h->pending + add > h->pending_limit) HS_TRY(drain(h));
            EventPair ev;
            HS_TRY(take_events(h, &ev));
            cudaEventRecord(ev.a, h->stream);
            const float *src = reinterpret_cast<const float *>(
                reinterpret_cast<const char *>(xyz) + off * esz);
            HS_CUDA(launch_bin_scatter(src, cnt, g0 + off, h->d, h->C, rate, h->p.sample_seed,
                                       h->probe, h->probe_base, kProbeCap, h->bl, h->bb.store(),
                                       h->stream, nullptr, 0, 0,
                                       h->routing ? &h->route : nullptr, packed ? 1 : 0));
            cudaEventRecord(ev.b, h->stream);
            h->pending_update.push_back(ev);
            h->pending += add;
            h->stats.update_launches += 1;
            h->stats.kernel_launches += (h->d.rows + h->bl.rows_per_pass - 1) / h->bl.rows_per_pass;
        }
        return HS_OK;
    }
    return launch_update_direct(h, xyz, n, g0, rate, packed);
}

hs_status launch_update_direct(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0,
                               double rate, bool packed) {
    EventPair ev;
    HS_TRY(take_events(h, &ev));
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

// Scatter passes one update of h takes over its input (row passes of a
// sketch whose rings do not fit one block).
static uint32_t scatter_passes(const hs_sketch *h) {
    const uint32_t rpp = h->bl.rows_per_pass ? h->bl.rows_per_pass : h->d.rows;
    return (h->d.rows + rpp - 1) / rpp;
}

// The compaction pass pays when the binned updates of h (and of its
// super-item sketch) would read the input in several passes: it reads the
// input once (12 bytes a float32 particle, 8 a packed record) and writes 8 a
// kept one, which every pass then reads instead of the input.
bool want_compact(hs_sketch *h, uint64_t n, double rate, bool packed) {
    if (h->routing || h->is_view || h->d.F != 1 || h->d.Gq >= (1u << kPackBits)) return false;
    if (!want_binned(h, n, rate)) return false;
    uint32_t passes = scatter_passes(h);
    if (h->super) {
        if (!want_binned(h->super, n, rate)) return false;
        passes += scatter_passes(h->super);
    }
    const double in = packed ? 8.0 : 12.0;
    return in + 8.0 * rate * (1.0 + passes) < in * passes;
}

// Binned update of h from the cell records of a compaction pass: `bound`
// records at most, *cells_cnt of them written; about bound * rate expected.
static hs_status launch_cells_timed(hs_sketch *h, uint64_t bound, double rate) {
    HS_TRY(size_regions(h, bound, rate));
    const double per = (double)h->d.rows / ((double)h->bl.nbins * h->bb.nblocks);   // a record
    const double room = h->pending_limit - h->bl.half;
    if (room < 1.0) return fail(HS_ERR_STATE, "binned regions too small for an update");
    // launches of room / per records up to a generous bound on the count;
    // one more takes whatever lies beyond (in practice nothing)
    const double expect = (double)bound * rate;
    const uint64_t likely = std::min<uint64_t>(
        bound, ((uint64_t)(1.05 * expect + 8.0 * std::sqrt(expect) + 4096.0) + 3) & ~3ull);
    const uint64_t piece = std::max<uint64_t>(4, (uint64_t)std::floor(room / per) & ~3ull);
    for (uint64_t off = 0; off < bound;) {
        const uint64_t cnt = off < likely ? std::min(piece, likely - off) : bound - off;
        const double add = (off < likely ? (double)cnt * per : 0.0) + h->bl.half;
        if (h->pending + add > h->pending_limit) HS_TRY(drain(h));
        EventPair ev;
        HS_TRY(take_events(h, &ev));
        cudaEventRecord(ev.a, h->stream);
        HS_CUDA(launch_bin_scatter(reinterpret_cast<const float *>(h->cells + off), cnt, 0, h->d,
                                   h->C, 1.0, h->p.sample_seed, nullptr, 0, 0, h->bl,
                                   h->bb.store(), h->stream, nullptr, 0, 0, nullptr, 2, 0, 0,
                                   nullptr, h->cells_cnt, off));
        cudaEventRecord(ev.b, h->stream);
        h->pending_update.push_back(ev);
        h->pending += add;
        h->stats.update_launches += 1;
        h->stats.kernel_launches += scatter_passes(h);
        off += cnt;
    }
    return HS_OK;
}

// The cells of a call's kept particles accumulate in h->cells (at most
// h->cells_bound records: every particle appended so far) and go through the
// binned passes of h and of its super-item sketch once per call, or when the
// buffer would overflow.  The super-item sketch reads the same records (it
// runs on h's stream).
static hs_status cells_flush(hs_sketch *h, double rate) {
    if (h->cells_bound == 0) return HS_OK;
    HS_TRY(launch_cells_timed(h, h->cells_bound, rate));
    if (hs_sketch *s = h->super) {
        s->cells = h->cells;
        s->cells_cnt = h->cells_cnt;
        hs_status st = launch_cells_timed(s, h->cells_bound, rate);
        s->cells = nullptr;
        s->cells_cnt = nullptr;
        HS_TRY(st);
    }
    HS_CUDA(cudaMemsetAsync(h->cells_cnt, 0, sizeof(unsigned long long), h->stream));
    h->cells_bound = 0;
    return HS_OK;
}

// The compaction pass over float32 particles or packed records (device or
// page-locked host memory) of a call of call_n particles: the cells of the
// kept ones are appended; it writes both sketches' probes.
static hs_status cells_append(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0, double rate,
                              uint64_t call_n, bool packed) {
    const size_t esz = packed ? 8 : 12;
    const uint64_t want = std::max<uint64_t>(std::min(call_n, kCellsMax), 1u << 20);
    if (h->cells_bound == 0 && h->cells_cap < want) {
        if (h->cells) cudaFree(h->cells);
        h->cells = nullptr;
        h->cells_cap = 0;
        HS_CUDA(cudaMalloc(&h->cells, want * 8));
        h->cells_cap = want;
    }
    if (!h->cells_cnt) {
        HS_CUDA(cudaMalloc(&h->cells_cnt, sizeof(unsigned long long)));
        HS_CUDA(cudaMemsetAsync(h->cells_cnt, 0, sizeof(unsigned long long), h->stream));
    }
    hs_sketch *s = h->super;
    const CompactProbe p0{h->probe, h->probe_base, h->probe_base + kProbeCap, 1, 0, h->d.G};
    const CompactProbe p1 = s ? CompactProbe{s->probe, s->probe_base, s->probe_base + kProbeCap,
                                             s->d.F, s->d.fmagic, s->d.G}
                              : CompactProbe{nullptr, 0, 0, 1, 0, 1};
    for (uint64_t off = 0; off < n;) {
        const uint64_t cnt = std::min(n - off, h->cells_cap);
        if (h->cells_bound + cnt > h->cells_cap) HS_TRY(cells_flush(h, rate));
        EventPair ev;
        HS_TRY(take_events(h, &ev));
        cudaEventRecord(ev.a, h->stream);
        const float *src = reinterpret_cast<const float *>(reinterpret_cast<const char *>(xyz) + off * esz);
        HS_CUDA(launch_compact_cells(src, cnt, g0 + off, h->d, rate, h->p.sample_seed, p0, p1,
                                     h->cells, h->cells_cnt, h->num_sms * 8, h->stream,
                                     packed ? 1 : 0));
        cudaEventRecord(ev.b, h->stream);
        h->pending_update.push_back(ev);
        h->stats.kernel_launches += 1;
        h->cells_bound += cnt;
        off += cnt;
    }
    return HS_OK;
}

// One piece of an update call: appended to the call's compacted cells (when
// the call compacts), else the sketch's (and its super-item sketch's) own
// scatter.  update_finish ends the call.
hs_status update_piece(hs_sketch *h, const float *xyz, uint64_t n, uint64_t g0, double rate,
                       bool packed, bool compact, uint64_t call_n) {
    if (compact) return cells_append(h, xyz, n, g0, rate, call_n, packed);
    HS_TRY(launch_update_timed(h, xyz, n, g0, rate, packed));
    if (h->super) HS_TRY(launch_update_timed(h->super, xyz, n, g0, rate, packed));
    return HS_OK;
}

hs_status update_finish(hs_sketch *h, double rate) { return cells_flush(h, rate); }

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
    if (h->d.W < 32 || hot < 1) return HS_OK;          // the scan instead
    HS_CUDA(launch_signed_bits(h->C, h->d, (int32_t)std::min<int64_t>(hot, INT32_MAX), h->xbits,
                               h->num_sms * 8, h->stream));
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
    // cells/s); one (cx, hot bucket and sign) query ~ 0.25 per directory slot it reads
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
    EventPair ev;
    HS_TRY(take_events(h, &ev));
    cudaEventRecord(ev.a, h->stream);
    for (uint32_t r = 0; r < F; ++r) {
        HS_CUDA(launch_dir_query(h->C, h->d, (int)r, h->dir_D,
                                 dir_has_inline(h->d.G, h->dir_D,
                                                (h->p.flags & HS_FLAG_DIR_INLINE) != 0),
                                 h->dir_off[r], h->dir_rec[r],
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
        EventPair ev;
        HS_TRY(take_events(h, &ev));
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

}  // namespace capi
}  // namespace hs

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
    free_bins(h->bb);
    if (h->C && !h->is_view) cudaFree(h->C);
    if (h->probe && !h->is_view) cudaFree(h->probe);
    if (h->cells) cudaFree(h->cells);
    if (h->cells_cnt) cudaFree(h->cells_cnt);
    if (h->q_keys) cudaFree(h->q_keys);
    if (h->q_est) cudaFree(h->q_est);
    if (h->flags) cudaFree(h->flags);
    for (int i = 0; i < kStageBuffers; ++i) {
        if (h->stage[i]) cudaFree(h->stage[i]);
        if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
        if (h->ev_free[i]) cudaEventDestroy(h->ev_free[i]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (auto *v : {&h->pending_update, &h->pending_search, &h->pending_flush, &h->pending_copy, &h->pool})
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
    const void *view = nullptr;
    const bool compact = want_compact(h, n, sample_rate, packed);
    if (is_device_ptr(src)) {
        HS_TRY(update_piece(h, xyz, n, h->n_seen, sample_rate, packed, compact, n));
    } else if (!h->super && (view = pinned_device_view(src)) != nullptr) {
        // page-locked host memory: the kernels read it over the host link
        // once (a hierarchy stages it: its compaction pass, reading the link
        // directly, measured slower than staged copies overlapping the work)
        HS_TRY(update_piece(h, static_cast<const float *>(view), n, h->n_seen, sample_rate, packed,
                            compact, n));
        h->stats.h2d_bytes += n * esz;
    } else {
        hs_status st = ensure_staging(h);
        if (st != HS_OK) return st;
        // size the bins for the whole call, not for one staged piece
        const uint64_t first = std::min(kStageParticles, n);
        const uint64_t pieces = (n + kStageParticles - 1) / kStageParticles;
        if (want_binned(h, first, sample_rate)) st = ensure_bins(h, n, sample_rate, pieces);
        if (st == HS_OK && h->super && want_binned(h->super, first, sample_rate))
            st = ensure_bins(h->super, n, sample_rate, pieces);
        if (st != HS_OK) return st;
        int i = 0;
        for (uint64_t off = 0; off < n; off += kStageParticles, ++i) {
            uint64_t cnt = std::min(kStageParticles, n - off);
            int b = i % kStageBuffers;
            HS_CUDA(cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0));
            EventPair ce;
            HS_TRY(take_events(h, &ce));
            HS_CUDA(cudaEventRecord(ce.a, h->copy_stream));
            HS_CUDA(cudaMemcpyAsync(h->stage[b], static_cast<const char *>(src) + off * esz,
                                    cnt * esz, cudaMemcpyHostToDevice, h->copy_stream));
            HS_CUDA(cudaEventRecord(ce.b, h->copy_stream));
            h->pending_copy.push_back(ce);
            h->stats.h2d_bytes += cnt * esz;
            HS_CUDA(cudaEventRecord(h->ev_copied[b], h->copy_stream));
            HS_CUDA(cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
            HS_TRY(update_piece(h, h->stage[b], cnt, h->n_seen + off, sample_rate, packed, compact, n));
            HS_CUDA(cudaEventRecord(h->ev_free[b], h->stream));
        }
    }
    HS_TRY(update_finish(h, sample_rate));
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
    drain_timings(h);
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
        EventPair ev;
        HS_TRY(take_events(h, &ev));
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
    EventPair whole;
    HS_TRY(take_events(h, &whole));
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
    HS_TRY(check_ranked(keys, est, n));
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
    EventPair whole;
    HS_TRY(take_events(h, &whole));
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
    HS_TRY(check_ranked(keys, est, n));
    *n_out = (uint32_t)n;
    return HS_OK;
}

hs_status sketch_reset(hs_sketch *h) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    hs_status st = discard_pending(h);
    if (st != HS_OK) return st;
    HS_CUDA(cudaMemsetAsync(h->C, 0, (size_t)h->d.rows * h->d.W * 4, h->stream));
    HS_CUDA(cudaMemsetAsync(h->probe, 0xFF, kProbeCap * 8, h->stream));
    if (h->cells_cnt) HS_CUDA(cudaMemsetAsync(h->cells_cnt, 0, sizeof(unsigned long long), h->stream));
    h->cells_bound = 0;
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
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    int blocks = sms * 8;
    uint64_t per = std::max<uint64_t>(1, total_ops / ((uint64_t)blocks * 256));
    if (e == cudaSuccess) e = cudaMemsetAsync(t, 0, n_counters * 4, s);
    if (e == cudaSuccess) e = launch_red_rate(t, n_counters, per, blocks, s);   // warm the table into L2
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = launch_red_rate(t, n_counters, per, blocks, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    cudaFree(t);
    if (e != cudaSuccess) return fail(HS_ERR_CUDA, "red-rate measurement: %s", cudaGetErrorString(e));
    *ops_per_s = (double)per * blocks * 256 / (ms * 1e-3);
    return HS_OK;
}

}  // extern "C"
