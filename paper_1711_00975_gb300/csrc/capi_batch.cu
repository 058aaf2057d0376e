// capi_batch.cu - batches of independent sub-volumes (batch_* of the C ABI).
#include <atomic>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>

#include "capi_internal.h"

// ---------------------------------------------------------------------------
// Batches of independent sub-volumes (each with its own mesh, stream index,
// sketch and top-k), updated by one persistent scatter launch and one
// accumulation launch, replayed as a CUDA graph.
// ---------------------------------------------------------------------------

namespace {

constexpr uint64_t kBatchProbe = 1ull << 16;   // probe keys per volume

// Ring depths chosen by batch_autotune, per (device, log2 W, rows, sample
// rate), kept for the process so later batches of the same shape skip tuning.
struct TuneChoice {
    uint32_t wvols, slot;
    float ms;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, uint32_t, uint32_t, double>, TuneChoice> g_tune_cache;

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
    BinBuffers bb;                      // code regions, sized per volume
    uint32_t rounds = 0;                // scatter tiles between flushes (0: default)
    uint32_t slot = 0;                  // scatter ring depth (0: largest that fits)
    uint32_t wvols = 0;                 // ring window of volumes at most (0: up to 4)
    VolumeDesc *d_vols = nullptr;
    VolumeDesc *h_vols = nullptr;       // pinned: read by the graph's copy node
    uint32_t *tvols = nullptr;          // per scatter tile: its first and last volume
    uint64_t tvols_cap = 0;
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
    // top-k of every volume on the device, one graph per k (k_batch_topk.cu)
    struct {
        uint32_t k = 0;
        bool dirs = false;              // every volume's directories are built
        bool failed = false;            // memory short: the general path only
        BatchTopkBufs bufs{};
        std::vector<void *> dev;        // device buffers of bufs
        BatchTopkVol *h_vol = nullptr;  // pinned, read by the graph's copy node
        uint64_t *h_key = nullptr;      // pinned results, written by the graph
        int32_t *h_est = nullptr;
        uint32_t *h_n = nullptr, *h_status = nullptr;
        cudaGraphExec_t gexec = nullptr;
        cudaEvent_t ev_a = nullptr, ev_b = nullptr;
        uint32_t launches = 0;          // kernels a replay runs
        // each volume's directories of rows 0..F-1 at its own resolution D
        std::vector<uint32_t *> doff;
        std::vector<DirRecord *> drec;
        std::vector<uint32_t> D;
    } tk;
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

// Regions sized per volume: a volume of N particles spans about N / tile + 2
// scatter tiles, dealt round-robin to the blocks, and each tile adds tile *
// rate / (bins per row) codes to each of the volume's bins on average; a
// block's bin leaves its ring window once a launch (one padded half).
hs_status batch_ensure_bins(hs_batch *b, const uint64_t *offsets, double rate) {
    const uint64_t ntiles = (offsets[b->nvol] + kScatterTile - 1) / kScatterTile;
    if (ntiles > b->tvols_cap) {
        if (b->tvols) cudaFree(b->tvols);
        b->tvols = nullptr;
        b->tvols_cap = 0;
        HS_CUDA(cudaMalloc(&b->tvols, std::max<uint64_t>(ntiles, 1024) * 4));
        b->tvols_cap = std::max<uint64_t>(ntiles, 1024);
    }
    if (b->bb.codes) return HS_OK;
    // padding of the deepest ring any window may use (a window of one volume)
    const uint32_t half = batch_ring(b->bl, b->d, b->nvol, rate, 0, 1).slot / 2;
    const uint32_t nblocks = (uint32_t)b->num_sms;
    const uint32_t bpr = 1u << (b->d.log2w - b->bl.S);
    const uint32_t bpv = b->d.rows * bpr;
    std::vector<uint32_t> caps(b->nvol);
    for (uint32_t v = 0; v < b->nvol; ++v) {
        const uint64_t N = offsets[v + 1] - offsets[v];
        const uint64_t tiles = N / kScatterTile + 2;
        const uint64_t per_block = (tiles + nblocks - 1) / nblocks;
        const double mean = (double)per_block * kScatterTile * rate / bpr;
        caps[v] = std::max<uint32_t>(region_capacity(mean, half, 1.0), 4 * half);
    }
    return alloc_bins(b->bb, caps, bpv, nblocks, b->stream);
}

// scatter + accumulate of the whole batch on b->stream (captured or direct)
hs_status batch_enqueue(hs_batch *b, const float *xyz, uint64_t n, double rate) {
    HS_CUDA(cudaMemcpyAsync(b->d_vols, b->h_vols, b->nvol * sizeof(VolumeDesc),
                            cudaMemcpyHostToDevice, b->stream));
    HS_CUDA(launch_bin_scatter(xyz, n, 0, b->d, b->C, rate, b->p.sample_seed, b->probe, 0,
                               kBatchProbe, b->bl, b->bb.store(), b->stream, b->d_vols, b->nvol,
                               kBatchProbe, nullptr, 0, b->rounds, b->slot, b->tvols, nullptr, 0,
                               b->wvols));
    HS_CUDA(launch_bin_accumulate(b->bl, b->bb.store(), b->C, b->stream));
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
static void tk_free(hs_batch *b);
static void tk_free_dirs(hs_batch *b);

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
    // every bin is numbered (16 bits); rings are kept for a window of volumes
    b->bl = bin_layout(batch_flat_desc(b), kBinSmemBudget, false);
    const BatchRing ring = batch_ring(b->bl, b->d, n_volumes, 1.0, 0);
    b->bl.slot = ring.slot;
    b->bl.half = ring.slot / 2;
    b->bl.rows_per_pass = p.rows;
    if (b->bl.nbins == 0 || b->bl.nbins >= 65536 || ring.wvols == 0 || n_volumes > kMaxBinGroups) {
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
    if (e == cudaSuccess) e = cudaMalloc(&b->d_vols, n_volumes * sizeof(VolumeDesc));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_vols, n_volumes * sizeof(VolumeDesc));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_a);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_b);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->C, 0, counters * 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->probe, 0xFF, (size_t)n_volumes * kBatchProbe * 8, b->stream);
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
    tk_free(b);
    tk_free_dirs(b);
    if (b->tk.ev_a) cudaEventDestroy(b->tk.ev_a);
    if (b->tk.ev_b) cudaEventDestroy(b->tk.ev_b);
    for (size_t t = 0; t < b->views.size(); ++t) {
        hs_sketch *h = b->views[t];
        h->C = nullptr;
        h->probe = nullptr;
        cudaStream_t vs = h->stream;
        sketch_destroy(h);
        if (vs) cudaStreamDestroy(vs);
        if (b->vdone[t]) cudaEventDestroy(b->vdone[t]);
    }
    free_bins(b->bb);
    void *ps[] = {b->C, b->probe, b->d_vols, b->tvols};
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

// A view borrows volume v's directories of rows 0..F-1 and its mesh ...
static void view_borrow(hs_batch *b, hs_sketch *h, uint32_t v, uint32_t F) {
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
}

// ... and gives back the directories it built or kept
static void view_return(hs_batch *b, hs_sketch *h, uint32_t v, uint32_t F) {
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
}

// Top-k of volume v on view h by the general path (sketch's topk_extract)
static hs_status batch_topk_one(hs_batch *b, hs_sketch *h, uint32_t v, uint32_t F, uint32_t k,
                                uint64_t *keys, int32_t *est, uint32_t *n_out) {
    view_borrow(b, h, v, F);
    hs_status st = topk_extract(h, k, keys + (size_t)v * k, est + (size_t)v * k, &n_out[v]);
    view_return(b, h, v, F);
    return st;
}

// The general path for the volumes in `vols`: host threads drive one view
// each (own stream) over volumes taken from a shared counter.
static hs_status batch_topk_host(hs_batch *b, uint32_t k, uint64_t *keys, int32_t *est,
                                 uint32_t *n_out, const std::vector<uint32_t> &vols, uint32_t F) {
    if (vols.empty()) return HS_OK;
    // the views start after the batch's pending work; the batch resumes after theirs
    HS_CUDA(cudaEventRecord(b->fork, b->stream));
    for (hs_sketch *h : b->views) HS_CUDA(cudaStreamWaitEvent(h->stream, b->fork, 0));
    std::atomic<uint32_t> next{0};
    const uint32_t nv = (uint32_t)vols.size();
    std::vector<hs_status> status(b->views.size(), HS_OK);
    std::vector<std::string> msg(b->views.size());
    auto work = [&](size_t t) {
        cudaSetDevice(b->device);
        for (uint32_t i = next.fetch_add(1); i < nv; i = next.fetch_add(1)) {
            hs_status st = batch_topk_one(b, b->views[t], vols[i], F, k, keys, est, n_out);
            if (st != HS_OK) {
                status[t] = st;
                msg[t] = hs_last_error();
                next.store(nv);
                break;
            }
        }
    };
    const size_t nthreads = std::min<size_t>(b->views.size(), nv);
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nthreads; ++t) pool.emplace_back(work, t);
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

static void tk_free(hs_batch *b) {
    if (b->tk.gexec) cudaGraphExecDestroy(b->tk.gexec);
    b->tk.gexec = nullptr;
    for (void *q : b->tk.dev)
        if (q) cudaFree(q);
    b->tk.dev.clear();
    void *ph[] = {b->tk.h_vol, b->tk.h_key, b->tk.h_est, b->tk.h_n, b->tk.h_status};
    for (void *q : ph)
        if (q) cudaFreeHost(q);
    b->tk.h_vol = nullptr;
    b->tk.h_key = nullptr;
    b->tk.h_est = nullptr;
    b->tk.h_n = nullptr;
    b->tk.h_status = nullptr;
    b->tk.k = 0;
    cudaGetLastError();
}

static void tk_free_dirs(hs_batch *b) {
    for (auto *q : b->tk.doff)
        if (q) cudaFree(q);
    for (auto *q : b->tk.drec)
        if (q) cudaFree(q);
    b->tk.doff.clear();
    b->tk.drec.clear();
    b->tk.D.clear();
    b->tk.dirs = false;
    cudaGetLastError();
}

// Every volume's directories of rows 0..F-1, built once (they depend on the
// mesh and the hash seeds only), each with 2^D slots, D the smallest in
// [log2 W, 26] with 2^D >= G^2: a bucket's lines are then the records of a
// run of slots holding about one line each.  false: memory is short.
static hs_status tk_dirs(hs_batch *b, uint32_t F, bool *ok) {
    *ok = false;
    tk_free_dirs(b);
    const uint32_t nv = b->nvol;
    b->tk.D.assign(nv, 0);
    uint32_t Dmax = 0;
    for (uint32_t v = 0; v < nv; ++v) {
        const uint64_t lines = (uint64_t)b->G[v] * b->G[v];
        uint32_t D = b->d.log2w;
        while (D < 26 && (1ull << D) < lines) ++D;
        b->tk.D[v] = D;
        Dmax = std::max(Dmax, D);
    }
    const uint64_t nslots = 1ull << Dmax;
    uint32_t *cursor = nullptr, *scratch = nullptr;
    bool good = cudaMalloc(&cursor, (nslots + 1) * 4) == cudaSuccess &&
                cudaMalloc(&scratch, ((nslots + 1) / 1024 + 4096) * 4) == cudaSuccess;
    b->tk.doff.assign((size_t)nv * F, nullptr);
    b->tk.drec.assign((size_t)nv * F, nullptr);
    int launches = 0;
    for (uint32_t v = 0; v < nv && good; ++v) {
        SketchDesc dv = b->d;
        dv.G = dv.Gq = b->G[v];
        dv.F = 1;
        const uint64_t lines = (uint64_t)b->G[v] * b->G[v];
        for (uint32_t r = 0; r < F && good; ++r) {
            uint32_t *&off = b->tk.doff[v * F + r];
            DirRecord *&rec = b->tk.drec[v * F + r];
            good = cudaMalloc(&off, dir_bytes(b->G[v], b->tk.D[v], false)) == cudaSuccess &&
                   cudaMalloc(&rec, std::max<uint64_t>(lines, 1) * sizeof(DirRecord)) == cudaSuccess &&
                   launch_dir_build(dv, (int)r, b->tk.D[v], false, off, cursor, rec, scratch,
                                    b->num_sms * 8, b->stream, &launches) == cudaSuccess;
        }
    }
    if (good) good = cudaStreamSynchronize(b->stream) == cudaSuccess;   // before the scratch goes
    if (cursor) cudaFree(cursor);
    if (scratch) cudaFree(scratch);
    b->stats.kernel_launches += launches;
    if (!good) {
        tk_free_dirs(b);
        return HS_OK;
    }
    b->tk.dirs = true;
    *ok = true;
    return HS_OK;
}

// Buffers, directory tables and the graph of the device top-k for k; false
// (nothing kept) when k is too large for its fixed capacities or memory is short.
static hs_status tk_prepare(hs_batch *b, uint32_t k, uint32_t F, bool *ok) {
    *ok = false;
    tk_free(b);
    // the final step sorts kk <= k entries in shared memory; candidates (cells
    // at or above the probe's threshold) are kept up to 2^16 a volume
    if (k > 4096) return HS_OK;
    const uint32_t cand_cap = std::max<uint32_t>(1u << 16, 16 * k);
    BatchTopkBufs &B = b->tk.bufs;
    B = BatchTopkBufs{};
    const uint32_t nv = b->nvol;
    B.nvol = nv;
    B.F = F;
    B.k = k;
    B.hot_cap = (uint32_t)std::min<uint64_t>(b->d.W, 1u << 16);
    B.cand_cap = cand_cap;
    B.set_log2 = 1;
    while ((1ull << B.set_log2) < 2 * kBatchProbe) ++B.set_log2;
    B.probe_per_vol = kBatchProbe;
    B.probe = b->probe;
    bool good = true;
    auto dev = [&](auto **ptr, size_t bytes) {
        void *q = nullptr;
        if (good && cudaMalloc(&q, std::max<size_t>(bytes, 16)) == cudaSuccess) b->tk.dev.push_back(q);
        else good = false;
        *ptr = reinterpret_cast<std::remove_pointer_t<decltype(ptr)>>(q);
    };
    BatchTopkVol *d_vol = nullptr;
    const uint32_t **d_off = nullptr;
    const DirRecord **d_rec = nullptr;
    dev(&d_vol, nv * sizeof(BatchTopkVol));
    dev(&B.set, ((size_t)nv << B.set_log2) * 8);
    dev(&B.dkey, (size_t)nv * kBatchProbe * 8);
    dev(&B.dest, (size_t)nv * kBatchProbe * 4);
    dev(&B.dcnt, nv * 4);
    dev(&B.theta, nv * 4);
    dev(&B.status, nv * 4);
    dev(&B.scan, nv * 4);
    dev(&B.bits, (size_t)nv * b->d.rows * (b->d.W >> 5) * 4 * 2);   // positive and negative maps
    dev(&B.hot, (size_t)nv * F * B.hot_cap * 4);
    dev(&B.hot_cnt, (size_t)nv * F * 4);
    dev(&B.pre, ((size_t)nv * F + 1) * 8);
    dev(&d_off, (size_t)nv * F * sizeof(void *));
    dev(&d_rec, (size_t)nv * F * sizeof(void *));
    dev(&B.ckey, (size_t)nv * cand_cap * 8);
    dev(&B.cest, (size_t)nv * cand_cap * 4);
    dev(&B.ccnt, nv * 4);
    dev(&B.okey, (size_t)nv * k * 8);
    dev(&B.oest, (size_t)nv * k * 4);
    dev(&B.on, nv * 4);
    if (!good) {
        tk_free(b);
        return HS_OK;
    }
    B.vol = d_vol;
    B.dir_off = d_off;
    B.dir_rec = d_rec;
    std::vector<const uint32_t *> off(b->tk.doff.begin(), b->tk.doff.end());
    std::vector<const DirRecord *> rec(b->tk.drec.begin(), b->tk.drec.end());
    HS_CUDA(cudaMemcpy(d_off, off.data(), off.size() * sizeof(void *), cudaMemcpyHostToDevice));
    HS_CUDA(cudaMemcpy(d_rec, rec.data(), rec.size() * sizeof(void *), cudaMemcpyHostToDevice));
    HS_CUDA(cudaMallocHost(&b->tk.h_vol, nv * sizeof(BatchTopkVol)));
    HS_CUDA(cudaMallocHost(&b->tk.h_key, (size_t)nv * k * 8));
    HS_CUDA(cudaMallocHost(&b->tk.h_est, (size_t)nv * k * 4));
    HS_CUDA(cudaMallocHost(&b->tk.h_n, nv * 4));
    HS_CUDA(cudaMallocHost(&b->tk.h_status, nv * 4));
    if (!b->tk.ev_a) HS_CUDA(cudaEventCreate(&b->tk.ev_a));
    if (!b->tk.ev_b) HS_CUDA(cudaEventCreate(&b->tk.ev_b));
    // the graph: table in, every launch, results out
    cudaGraph_t graph = nullptr;
    int launches = 0;
    HS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaMemcpyAsync(d_vol, b->tk.h_vol, nv * sizeof(BatchTopkVol),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_batch_topk(b->C, b->d, B, b->num_sms, b->stream, &launches);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tk.h_key, B.okey, (size_t)nv * k * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tk.h_est, B.oest, (size_t)nv * k * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->tk.h_n, B.on, nv * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tk.h_status, B.status, nv * 4, cudaMemcpyDeviceToHost, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->tk.gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        tk_free(b);
        HS_CUDA(e);
    }
    b->tk.k = k;
    b->tk.launches = (uint32_t)launches;
    *ok = true;
    return HS_OK;
}

// The device top-k of every volume it can answer; the others go to `rest`.
static hs_status batch_topk_device(hs_batch *b, uint32_t k, uint32_t F, uint64_t *keys,
                                   int32_t *est, uint32_t *n_out, std::vector<uint32_t> &rest) {
    bool ok = true;
    if (!b->tk.dirs) {
        tk_free(b);                      // the graph reads the directory tables
        HS_TRY(tk_dirs(b, F, &ok));
        if (!ok) {
            b->tk.failed = true;
            return HS_OK;
        }
    }
    if (b->tk.k != k) {
        HS_CUDA(cudaStreamSynchronize(b->stream));
        HS_TRY(tk_prepare(b, k, F, &ok));
        if (!ok) return HS_OK;
    }
    for (uint32_t v = 0; v < b->nvol; ++v) {
        BatchTopkVol &V = b->tk.h_vol[v];
        const uint64_t cells = (uint64_t)b->G[v] * b->G[v] * b->G[v];
        V.m_probe = std::min<uint64_t>(b->n_seen[v] - b->probe_base[v], kBatchProbe);
        V.G = b->G[v];
        V.kk = (uint32_t)std::min<uint64_t>(k, cells);
        V.use = 1;
        V.D = b->tk.D[v];
        V.gmagic = div_magic(b->G[v]);   // items below 2^16 G and cells below 2^34: x < 2^48 / G
    }
    HS_CUDA(cudaEventRecord(b->tk.ev_a, b->stream));
    HS_CUDA(cudaGraphLaunch(b->tk.gexec, b->stream));
    HS_CUDA(cudaEventRecord(b->tk.ev_b, b->stream));
    HS_CUDA(cudaEventSynchronize(b->tk.ev_b));
    float ms = 0;
    if (cudaEventElapsedTime(&ms, b->tk.ev_a, b->tk.ev_b) == cudaSuccess) b->stats.topk_ms += ms;
    b->stats.kernel_launches += b->tk.launches;
    b->stats.search_launches += 1;
    for (uint32_t v = 0; v < b->nvol; ++v) {
        const uint32_t kk = b->tk.h_vol[v].kk;
        if (b->tk.h_status[v] != 0 || b->tk.h_n[v] != kk) {
            rest.push_back(v);
            continue;
        }
        std::memcpy(keys + (size_t)v * k, b->tk.h_key + (size_t)v * k, (size_t)kk * 8);
        std::memcpy(est + (size_t)v * k, b->tk.h_est + (size_t)v * k, (size_t)kk * 4);
        HS_TRY(check_ranked(keys + (size_t)v * k, est + (size_t)v * k, kk));
        n_out[v] = kk;
    }
    return HS_OK;
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
    std::vector<uint32_t> rest;
    // the device path: directory search in one graph (not when a scan is asked for)
    const bool scan = (b->p.flags & (HS_FLAG_SEARCH_SCAN | HS_FLAG_SEARCH_DIRECTORY)) == HS_FLAG_SEARCH_SCAN;
    if (!scan && !b->tk.failed && b->d.W >= 32) {
        HS_TRY(batch_topk_device(b, k, F, keys, est, n_out, rest));
        if (b->tk.k != k) {   // not prepared: every volume by the general path
            rest.clear();
            for (uint32_t v = 0; v < b->nvol; ++v) rest.push_back(v);
        }
    } else {
        for (uint32_t v = 0; v < b->nvol; ++v) rest.push_back(v);
    }
    b->stats.topk_calls += 1;
    b->stats.host_path_volumes = rest.size();
    return batch_topk_host(b, k, keys, est, n_out, rest, F);
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
    if (b->bb.fill)
        HS_CUDA(cudaMemsetAsync(b->bb.fill, 0, (size_t)b->bl.nbins * b->bb.nblocks * 4, b->stream));
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
    *out = b->stats;                   // topk_calls: batch queries
    for (hs_sketch *h : b->views) {    // plus the per-volume path's work
        hs_stats vs{};
        sketch_stats(h, &vs, reset);
        out->kernel_launches += vs.kernel_launches;
        out->search_launches += vs.search_launches;
        out->search_ms += vs.search_ms;
        out->topk_ms += vs.topk_ms;     // summed over concurrent views
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
    const auto key = std::make_tuple(b->device, b->d.log2w, b->d.rows, sample_rate);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {          // tuned before for this shape: no runs
            b->wvols = it->second.wvols;
            b->slot = it->second.slot;
            b->rounds = 1;
            const BatchRing r = batch_ring(b->bl, b->d, b->nvol, sample_rate, b->slot, b->wvols);
            out->rounds = 1;
            out->slot = r.slot;
            out->window_volumes = r.wvols;
            out->configs_tried = 0;
            out->best_ms = it->second.ms;
            return HS_OK;
        }
    }
    // candidates: the deepest ring of the widest window that holds a tile's
    // codes (up to 4 volumes), then windows of one volume with the deepest
    // ring, a half and a quarter of it; one tile is staged between flushes
    const uint32_t deep1 = batch_ring(b->bl, b->d, b->nvol, sample_rate, 0, 1).slot;
    const uint32_t wv_opt[4] = {0, 1, 1, 1};
    const uint32_t slot_opt[4] = {0, 0, deep1 / 2, deep1 / 4};
    float best = 1e30f;
    uint32_t best_slot = 0, best_wv = 0, best_rounds = 1;
    int tried = 0;
    for (int si = 0; si < 4; ++si) {
        if (slot_opt[si] != 0 && slot_opt[si] < 16) continue;
        b->wvols = wv_opt[si];
        b->slot = slot_opt[si];
        b->rounds = 1;
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
            best_slot = slot_opt[si];
            best_wv = wv_opt[si];
        }
    }
    b->wvols = best_wv;
    b->slot = best_slot;
    b->rounds = best_rounds;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = TuneChoice{best_wv, best_slot, best};
    }
    st = batch_reset(b);                              // tuning runs touched the counters
    if (st != HS_OK) return st;
    HS_CUDA(cudaStreamSynchronize(b->stream));
    const BatchRing chosen = batch_ring(b->bl, b->d, b->nvol, sample_rate, best_slot, best_wv);
    out->rounds = best_rounds;
    out->slot = chosen.slot;
    out->window_volumes = chosen.wvols;
    out->configs_tried = (uint32_t)tried;
    out->best_ms = best;
    return HS_OK;
}

}  // extern "C"
