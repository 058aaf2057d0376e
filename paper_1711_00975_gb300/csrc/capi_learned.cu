// capi_learned.cu - the router MLP, exact counts and the learned sketch
// (mlp_*, exact_*, learned_* of the C ABI).
#include "capi_internal.h"

// ---------------------------------------------------------------------------
// Learned router: MLP objects, exact counting, and the learned sketch.
// ---------------------------------------------------------------------------

struct hs_mlp {
    float *P = nullptr, *M = nullptr, *V = nullptr, *grad = nullptr, *loss = nullptr;
    float *part = nullptr;      // per-block gradient sums of one mini-batch
    size_t part_cap = 0;        // floats
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
    void *ps[] = {m->P, m->M, m->V, m->grad, m->loss, m->part};
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
    const size_t need = mlp_grad_scratch_floats(n);
    if (st == HS_OK && need > m->part_cap) {
        if (m->part) cudaFree(m->part);
        m->part = nullptr;
        m->part_cap = 0;
        cudaError_t ea = cudaMalloc(&m->part, need * 4);
        if (ea != cudaSuccess) st = fail(HS_ERR_OOM, "gradient scratch: %s", cudaGetErrorString(ea));
        else m->part_cap = need;
    }
    cudaError_t e = st == HS_OK ? launch_mlp_grad(m->P, df, dy, dw, n, m->grad, m->loss, m->part,
                                                  m->stream)
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
