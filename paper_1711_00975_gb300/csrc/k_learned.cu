// k_learned.cu - the learned router: coarse density features, a small MLP that
// predicts which coarse cells hold heavy fine cells, an exact hash table for
// the cells it routes, and its training kernels.
//
// This is an addition to the paper's method (arXiv:1711.00975 finds heavy
// cells with a Count Sketch alone, Sec. 2.2).  Fine cells inside coarse cells
// predicted heavy are counted exactly (the exact algorithm of Sec. 4.2,
// restricted to those cells); every other particle goes to the sketch.
//
// Bit-exactness with the CPU oracle: features come from a table of
// bf16(log10(1 + n)) built in double precision; every neuron is an explicit
// float32 fused multiply-add chain over its inputs in index order; hidden
// activations are rounded to bf16 after ReLU; a coarse cell is routed iff its
// final float32 logit is > 0 (sigmoid > 1/2), so no transcendental decides it.
#include <cuda_bf16.h>

#include <algorithm>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

__device__ __forceinline__ float bf16_round(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

// ---- coarse histogram of a hashed sample of the stream ----
__global__ void k_coarse_hist(const float *__restrict__ xyz, uint64_t n, uint64_t g0,
                              const SketchDesc d, uint32_t R, uint32_t Gc, uint64_t seed,
                              uint64_t thr, uint32_t keep_all, int32_t *__restrict__ counts) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t g = g0 + i;
        if (!keep_all && splitmix64_at(seed, g) >= thr) continue;
        uint32_t cx, cy, cz;
        bool ok = axis_cell(xyz[3 * i], d.inv_cell, d.G, cx);
        ok &= axis_cell(xyz[3 * i + 1], d.inv_cell, d.G, cy);
        ok &= axis_cell(xyz[3 * i + 2], d.inv_cell, d.G, cz);
        if (!ok) continue;
        const uint64_t ck = (uint64_t)(cx / R) + (uint64_t)Gc * ((cy / R) + (uint64_t)Gc * (cz / R));
        atomicAdd(&counts[ck], 1);
    }
}

// ---- coarse keys with a non-zero count ----
__global__ void k_coarse_list(const int32_t *__restrict__ counts, uint64_t ncoarse,
                              uint64_t *__restrict__ list, unsigned long long *__restrict__ n_list,
                              uint64_t cap) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < ncoarse; base += stride) {
        const uint64_t i = base + threadIdx.x;
        const bool on = i < ncoarse && counts[i] != 0;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, on);
        if (!m) continue;
        unsigned long long b0 = 0;
        if (lane == __ffs(m) - 1) b0 = atomicAdd(n_list, (unsigned long long)__popc(m));
        b0 = __shfl_sync(0xFFFFFFFFu, b0, __ffs(m) - 1);
        if (on) {
            unsigned long long j = b0 + __popc(m & ((1u << lane) - 1u));
            if (j < cap) list[j] = i;
        }
    }
}

// ---- 27 features per listed coarse cell: neighbour (dx,dy,dz) in -1..1 at
// index (dz+1)*9 + (dy+1)*3 + (dx+1), periodic, bf16(log10(1 + count)) ----
__global__ void k_features(const int32_t *__restrict__ counts, uint32_t Gc,
                           const uint64_t *__restrict__ list, uint64_t m,
                           const uint16_t *__restrict__ ftab, uint32_t ftab_n,
                           uint16_t *__restrict__ feats) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        const uint64_t ck = list[s];
        const uint32_t x = (uint32_t)(ck % Gc), y = (uint32_t)((ck / Gc) % Gc),
                       z = (uint32_t)(ck / ((uint64_t)Gc * Gc));
        int f = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++f) {
                    const uint32_t xx = (x + Gc + dx) % Gc, yy = (y + Gc + dy) % Gc,
                                   zz = (z + Gc + dz) % Gc;
                    const int32_t c =
                        counts[(uint64_t)xx + (uint64_t)Gc * (yy + (uint64_t)Gc * zz)];
                    uint16_t v;
                    if ((uint32_t)c < ftab_n) {
                        v = ftab[c];
                    } else {
                        __nv_bfloat16 b = __float2bfloat16_rn((float)log10(1.0 + (double)c));
                        v = *reinterpret_cast<uint16_t *>(&b);
                    }
                    feats[s * kMlpIn + f] = v;
                }
    }
}

// ---- MLP forward: one thread per sample, parameters in shared memory ----
struct MlpSmem {
    float w1[kMlpH * kMlpIn], b1[kMlpH], w2[kMlpH * kMlpH], b2[kMlpH], w3[kMlpH], b3;
};

__device__ __forceinline__ void load_params_bf16(MlpSmem &s, const float *__restrict__ P) {
    // the forward uses bf16-rounded weights and biases
    float *dst = reinterpret_cast<float *>(&s);
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) dst[i] = bf16_round(P[i]);
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t v) {
    return __uint_as_float((uint32_t)v << 16);
}

// h1 = bf16(relu(W1 x + b1)), h2 = bf16(relu(W2 h1 + b2)), z = w3 . h2 + b3, each
// a float32 fma chain in index order starting from the bias.
__device__ __forceinline__ float mlp_forward_one(const MlpSmem &s, const float *x, float *h1,
                                                 float *h2) {
    for (int j = 0; j < kMlpH; ++j) {
        float a = s.b1[j];
        for (int i = 0; i < kMlpIn; ++i) a = __fmaf_rn(s.w1[j * kMlpIn + i], x[i], a);
        h1[j] = bf16_round(fmaxf(a, 0.0f));
    }
    for (int j = 0; j < kMlpH; ++j) {
        float a = s.b2[j];
        for (int i = 0; i < kMlpH; ++i) a = __fmaf_rn(s.w2[j * kMlpH + i], h1[i], a);
        h2[j] = bf16_round(fmaxf(a, 0.0f));
    }
    float z = s.b3;
    for (int i = 0; i < kMlpH; ++i) z = __fmaf_rn(s.w3[i], h2[i], z);
    return z;
}

__global__ void __launch_bounds__(128)
    k_mlp_forward(const float *__restrict__ P, const uint16_t *__restrict__ feats, uint64_t m,
                  float *__restrict__ logits) {
    __shared__ MlpSmem s;
    load_params_bf16(s, P);
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += stride) {
        float x[kMlpIn], h1[kMlpH], h2[kMlpH];
        for (int i = 0; i < kMlpIn; ++i) x[i] = bf16_bits_to_float(feats[t * kMlpIn + i]);
        logits[t] = mlp_forward_one(s, x, h1, h2);
    }
}

// ---- training: forward + backward of a mini-batch, gradients summed ----
// Loss per sample: w * (softplus(z) - y z); the caller divides by sum(w).
// The gradient treats the bf16 roundings as identities (straight-through).
// Each block leaves its sums (every parameter's gradient, then the loss and
// the weight sum) in its own row of `part`; k_grad_sum adds the rows in block
// order, so a training run is reproducible bit for bit.
constexpr int kTrainBlock = 128;
constexpr int kPartWidth = kMlpParams + 2;

struct TrainSmem {
    MlpSmem s;
    float x[kTrainBlock][kMlpIn + 1];
    float h1[kTrainBlock][kMlpH + 1];
    float d1[kTrainBlock][kMlpH + 1];
    float h2[kTrainBlock][kMlpH + 1];
    float d2[kTrainBlock][kMlpH + 1];
    float dz[kTrainBlock];
};

__global__ void __launch_bounds__(kTrainBlock)
    k_mlp_grad(const float *__restrict__ P, const uint16_t *__restrict__ feats,
               const float *__restrict__ y, const float *__restrict__ w, uint64_t m,
               float *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    MlpSmem &s = S.s;
    auto &sx = S.x;
    auto &sh1 = S.h1;
    auto &sd1 = S.d1;
    auto &sh2 = S.h2;
    auto &sd2 = S.d2;
    auto &sdz = S.dz;
    load_params_bf16(s, P);
    __syncthreads();
    const int t = threadIdx.x;
    const uint64_t base = (uint64_t)blockIdx.x * kTrainBlock;
    const uint64_t smp = base + t;
    float lsum = 0.0f;
    if (smp < m) {
        float x[kMlpIn], h1[kMlpH], h2[kMlpH];
        for (int i = 0; i < kMlpIn; ++i) x[i] = bf16_bits_to_float(feats[smp * kMlpIn + i]);
        const float z = mlp_forward_one(s, x, h1, h2);
        const float yy = y[smp], ww = w[smp];
        const float sp = z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z));   // softplus
        lsum = ww * (sp - yy * z);
        const float sig = 1.0f / (1.0f + expf(-z));
        const float dz = ww * (sig - yy);
        sdz[t] = dz;
        for (int i = 0; i < kMlpIn; ++i) sx[t][i] = x[i];
        for (int j = 0; j < kMlpH; ++j) {
            sh2[t][j] = h2[j];
            sd2[t][j] = h2[j] > 0.0f ? dz * s.w3[j] : 0.0f;
            sh1[t][j] = h1[j];
        }
        for (int i = 0; i < kMlpH; ++i) {
            float a = 0.0f;
            for (int j = 0; j < kMlpH; ++j) a = __fmaf_rn(sd2[t][j], s.w2[j * kMlpH + i], a);
            sd1[t][i] = h1[i] > 0.0f ? a : 0.0f;
        }
    } else {
        sdz[t] = 0.0f;
        for (int i = 0; i < kMlpIn; ++i) sx[t][i] = 0.0f;
        for (int j = 0; j < kMlpH; ++j) sh2[t][j] = sd2[t][j] = sh1[t][j] = sd1[t][j] = 0.0f;
    }
    __syncthreads();
    // block sums of the per-sample outer products, one parameter per thread step
    const uint64_t left = m > base ? m - base : 0;
    const int nb = left < (uint64_t)kTrainBlock ? (int)left : kTrainBlock;
    for (int p = t; p < kMlpParams; p += kTrainBlock) {
        float acc = 0.0f;
        if (p < kMlpH * kMlpIn) {                          // w1[j][i]
            const int j = p / kMlpIn, i = p % kMlpIn;
            for (int q = 0; q < nb; ++q) acc = __fmaf_rn(sd1[q][j], sx[q][i], acc);
        } else if (p < kMlpH * kMlpIn + kMlpH) {           // b1[j]
            const int j = p - kMlpH * kMlpIn;
            for (int q = 0; q < nb; ++q) acc += sd1[q][j];
        } else if (p < kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH) {   // w2[j][i]
            const int o = p - kMlpH * kMlpIn - kMlpH, j = o / kMlpH, i = o % kMlpH;
            for (int q = 0; q < nb; ++q) acc = __fmaf_rn(sd2[q][j], sh1[q][i], acc);
        } else if (p < kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH) {  // b2[j]
            const int j = p - kMlpH * kMlpIn - kMlpH - kMlpH * kMlpH;
            for (int q = 0; q < nb; ++q) acc += sd2[q][j];
        } else if (p < kMlpParams - 1) {                   // w3[i]
            const int i = p - (kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH);
            for (int q = 0; q < nb; ++q) acc = __fmaf_rn(sdz[q], sh2[q][i], acc);
        } else {                                           // b3
            for (int q = 0; q < nb; ++q) acc += sdz[q];
        }
        part[(uint64_t)blockIdx.x * kPartWidth + p] = acc;
    }
    // loss and weight sums of the block, added in sample order
    __syncthreads();
    sdz[t] = lsum;
    sx[t][0] = smp < m ? w[smp] : 0.0f;
    __syncthreads();
    if (t == 0) {
        float ls = 0.0f, ws = 0.0f;
        for (int q = 0; q < kTrainBlock; ++q) {
            ls += sdz[q];
            ws += sx[q][0];
        }
        part[(uint64_t)blockIdx.x * kPartWidth + kMlpParams] = ls;
        part[(uint64_t)blockIdx.x * kPartWidth + kMlpParams + 1] = ws;
    }
}

// grad[p] = sum over blocks b (in order) of part[b][p]; loss[0..1] likewise
__global__ void k_grad_sum(const float *__restrict__ part, uint32_t nblocks,
                           float *__restrict__ grad, float *__restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kPartWidth) return;
    float acc = 0.0f;
    for (uint32_t b = 0; b < nblocks; ++b) acc += part[(uint64_t)b * kPartWidth + p];
    if (p < kMlpParams) grad[p] = acc;
    else loss[p - kMlpParams] = acc;
}

// Adam on the float32 master parameters; gradients are divided by *gscale
// (the mini-batch's weight sum) first.
__global__ void k_adam(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                       const float *__restrict__ grad, const float *__restrict__ gscale, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMlpParams) return;
    const float sc = *gscale;
    const float g = sc > 0.0f ? grad[p] / sc : 0.0f;
    const float m = b1 * M[p] + (1.0f - b1) * g;
    const float v = b2 * V[p] + (1.0f - b2) * g * g;
    M[p] = m;
    V[p] = v;
    P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// Routing rank of a listed coarse cell: the bit pattern of a positive logit
// (positive floats order like their bit patterns), INT32_MIN for logit <= 0
// (never routed).  Counts the positive ones.
__global__ void k_logit_rank(const float *__restrict__ logits, uint64_t m,
                             int32_t *__restrict__ rank, unsigned long long *__restrict__ n_pos) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t c = 0;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        const float z = logits[s];
        const bool pos = z > 0.0f;
        rank[s] = pos ? (int32_t)__float_as_uint(z) : INT32_MIN;
        c += pos;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_pos, (unsigned long long)c);
}

// Route listed coarse cell s iff its logit > 0 and, when a budget applies, its
// (rank desc, key asc) position is within the budget: its 96-bit rank value
// ((rank ^ 2^31) << 64 | ~key) is at or above the selected threshold.
__global__ void k_route(const uint64_t *__restrict__ list, const int32_t *__restrict__ rank,
                        uint64_t m, const SelectState *__restrict__ sel, int use_sel,
                        uint32_t *__restrict__ bits) {
    const uint32_t th = use_sel ? sel->hi : 0u;
    const uint64_t tl = use_sel ? sel->lo : 0ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        const int32_t r = rank[s];
        if (r == INT32_MIN) continue;
        const uint64_t ck = list[s];
        if (use_sel) {
            const uint32_t hi = (uint32_t)r ^ 0x80000000u;
            const uint64_t lo = ~ck;
            if (!(hi > th || (hi == th && lo >= tl))) continue;
        }
        atomicOr(&bits[ck >> 5], 1u << (ck & 31));
    }
}

__global__ void k_word_popc(const uint32_t *__restrict__ bits, uint64_t words,
                            uint32_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride)
        out[w] = __popc(bits[w]);
}

// rlist[block of ck] = ck for every routed listed cell
__global__ void k_route_list(const uint64_t *__restrict__ list, uint64_t m,
                             const uint32_t *__restrict__ bits, const uint32_t *__restrict__ prefix,
                             uint64_t *__restrict__ rlist) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        const uint64_t ck = list[s];
        const uint32_t w = (uint32_t)(ck >> 5), b = (uint32_t)(ck & 31), word = bits[w];
        if ((word >> b) & 1u) rlist[prefix[w] + __popc(word & ((1u << b) - 1u))] = ck;
    }
}

// non-zero counters of the dense blocks -> (fine key, count)
__global__ void k_block_list(const int32_t *__restrict__ blocks, const uint64_t *__restrict__ rlist,
                             uint64_t nblocks, uint32_t R, uint32_t Gc, uint32_t G,
                             uint64_t *__restrict__ out_keys, int32_t *__restrict__ out_counts,
                             unsigned long long *__restrict__ n_out, uint64_t cap) {
    const uint32_t R3 = R * R * R;
    const uint64_t total = nblocks * R3;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
        const uint64_t i = base + threadIdx.x;
        const int32_t c = i < total ? blocks[i] : 0;
        const bool on = c != 0;
        const unsigned msk = __ballot_sync(0xFFFFFFFFu, on);
        if (!msk) continue;
        unsigned long long b0 = 0;
        if (lane == __ffs(msk) - 1) b0 = atomicAdd(n_out, (unsigned long long)__popc(msk));
        b0 = __shfl_sync(0xFFFFFFFFu, b0, __ffs(msk) - 1);
        if (on) {
            const unsigned long long j = b0 + __popc(msk & ((1u << lane) - 1u));
            if (j < cap && out_keys) {
                const uint64_t ck = rlist[i / R3];
                const uint32_t l = (uint32_t)(i % R3);
                const uint32_t cx = (uint32_t)(ck % Gc) * R + l % R,
                               cy = (uint32_t)((ck / Gc) % Gc) * R + (l / R) % R,
                               cz = (uint32_t)(ck / ((uint64_t)Gc * Gc)) * R + l / (R * R);
                out_keys[j] = key_of(cx, cy, cz, G);
                out_counts[j] = c;
            }
        }
    }
}

}  // namespace


cudaError_t launch_coarse_hist(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                               uint32_t R, uint32_t Gc, uint64_t seed, double rate,
                               int32_t *counts, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 8192);
    k_coarse_hist<<<(unsigned)blocks, 256, 0, s>>>(xyz, n, g0, d, R, Gc, seed,
                                                   rate >= 1.0 ? 0 : (uint64_t)ldexp(rate, 64),
                                                   rate >= 1.0 ? 1u : 0u, counts);
    return cudaGetLastError();
}

cudaError_t launch_coarse_list(const int32_t *counts, uint64_t ncoarse, uint64_t *list,
                               unsigned long long *n_list, uint64_t cap, cudaStream_t s) {
    uint64_t blocks = std::min<uint64_t>((ncoarse + 255) / 256, 8192);
    k_coarse_list<<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, s>>>(counts, ncoarse, list,
                                                                          n_list, cap);
    return cudaGetLastError();
}

cudaError_t launch_features(const int32_t *counts, uint32_t Gc, const uint64_t *list, uint64_t m,
                            const uint16_t *ftab, uint32_t ftab_n, uint16_t *feats,
                            cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((m + 127) / 128, 8192);
    k_features<<<(unsigned)blocks, 128, 0, s>>>(counts, Gc, list, m, ftab, ftab_n, feats);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *P, const uint16_t *feats, uint64_t m, float *logits,
                               cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((m + 127) / 128, 4096);
    k_mlp_forward<<<(unsigned)blocks, 128, 0, s>>>(P, feats, m, logits);
    return cudaGetLastError();
}

size_t mlp_grad_scratch_floats(uint64_t m) {
    return (size_t)((m + kTrainBlock - 1) / kTrainBlock) * kPartWidth;
}

cudaError_t launch_mlp_grad(const float *P, const uint16_t *feats, const float *y, const float *w,
                            uint64_t m, float *grad, float *loss, float *part, cudaStream_t s) {
    if (m == 0) {
        cudaError_t e = cudaMemsetAsync(grad, 0, kMlpParams * 4, s);
        return e == cudaSuccess ? cudaMemsetAsync(loss, 0, 8, s) : e;
    }
    const uint64_t blocks = (m + kTrainBlock - 1) / kTrainBlock;
    cudaError_t e = ensure_smem_limit(k_mlp_grad, sizeof(TrainSmem));
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<(unsigned)blocks, kTrainBlock, sizeof(TrainSmem), s>>>(P, feats, y, w, m, part);
    k_grad_sum<<<(kPartWidth + 255) / 256, 256, 0, s>>>(part, (uint32_t)blocks, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *P, float *M, float *V, const float *grad, const float *gscale,
                        float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(P, M, V, grad, gscale, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_logit_rank(const float *logits, uint64_t m, int32_t *rank,
                              unsigned long long *n_pos, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((m + 255) / 256, 8192);
    k_logit_rank<<<(unsigned)blocks, 256, 0, s>>>(logits, m, rank, n_pos);
    return cudaGetLastError();
}

cudaError_t launch_route(const uint64_t *list, const int32_t *rank, uint64_t m,
                         const SelectState *sel, int use_sel, uint32_t *bits, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((m + 255) / 256, 8192);
    k_route<<<(unsigned)blocks, 256, 0, s>>>(list, rank, m, sel, use_sel, bits);
    return cudaGetLastError();
}

cudaError_t launch_word_popc(const uint32_t *bits, uint64_t words, uint32_t *out, cudaStream_t s) {
    uint64_t blocks = std::min<uint64_t>((words + 255) / 256, 8192);
    k_word_popc<<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, s>>>(bits, words, out);
    return cudaGetLastError();
}

cudaError_t launch_route_list(const uint64_t *list, uint64_t m, const uint32_t *bits,
                              const uint32_t *prefix, uint64_t *rlist, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((m + 255) / 256, 8192);
    k_route_list<<<(unsigned)blocks, 256, 0, s>>>(list, m, bits, prefix, rlist);
    return cudaGetLastError();
}

cudaError_t launch_block_list(const int32_t *blocks_, const uint64_t *rlist, uint64_t nblocks,
                              uint32_t R, uint32_t Gc, uint32_t G, uint64_t *out_keys,
                              int32_t *out_counts, unsigned long long *n_out, uint64_t cap,
                              cudaStream_t s) {
    const uint64_t total = nblocks * R * R * R;
    if (total == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((total + 255) / 256, 8192);
    k_block_list<<<(unsigned)blocks, 256, 0, s>>>(blocks_, rlist, nblocks, R, Gc, G, out_keys,
                                                  out_counts, n_out, cap);
    return cudaGetLastError();
}

}  // namespace hs
