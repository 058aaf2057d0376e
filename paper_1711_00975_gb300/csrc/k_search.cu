// k_search.cu - estimate mode of Count Sketch with Full Search
// (arXiv:1711.00975 Algorithm 1, "Querying the data structure"; Sec. 3.1
// "GPU without heap": estimate every cell of the mesh and keep the items above
// a threshold; Algorithm 4, Estimate: median of the t row estimates).
//
// The paper gives one block per cell and one thread per row, and finds the
// median by rank counting in shared memory.  Here one warp walks a whole mesh
// line (fixed cy, cz; cx = lane, lane + 32, ...), so each row's hash value
// advances by a constant a0 * 32 per step (one 64-bit add), and the median of
// five is a six-comparison register network.
//
// Pruning, exact by construction: a cell whose median is >= theta > 0 has at
// least need = t - floor((t-1)/2) rows with sign * C >= theta, hence with
// |C| >= theta.  A per-row bitmap of "hot" super-buckets (some counter with
// |C| >= theta) in shared memory rejects a cell as soon as more than t - need
// of its rows are cold, before any counter is read.  Survivors are estimated
// exactly from the counters and compared with theta.
#include <algorithm>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t hot_bit(const uint32_t *s_bits, uint32_t words_per_row, int r,
                                            uint64_t v, uint32_t nb) {
    uint32_t sb = (uint32_t)(v >> (64 - nb));
    return (s_bits[(uint32_t)r * words_per_row + (sb >> 5)] >> (sb & 31)) & 1u;
}

__device__ __forceinline__ bool passes(int32_t e, int32_t theta, uint32_t mode) {
    return mode == kGE ? e >= theta : (mode == kGT ? e > theta : e == theta);
}

// Append the lanes with `pass` set: one atomic per warp, slots in lane order.
__device__ __forceinline__ void warp_append(bool pass, uint64_t key, int32_t est,
                                            const SearchOut &out, int lane) {
    unsigned m = __ballot_sync(kFull, pass);
    if (!m) return;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(out.count, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (pass) {
        unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
        if (idx < out.cap) {
            out.key[idx] = key;
            out.est[idx] = est;
        }
    }
}

template <int T>
__global__ void __launch_bounds__(1024, 1)
    k_full_search(const int32_t *__restrict__ C, const SketchDesc d, int32_t theta, uint32_t mode,
                  const uint32_t *__restrict__ bitmap, uint32_t nb, int prune, uint64_t line_lo,
                  uint64_t line_hi, SearchOut out, RouteFilter skip) {
    extern __shared__ uint32_t s_bits[];
    const uint32_t rows = T > 0 ? (uint32_t)T : d.rows;
    const uint32_t words_per_row = (1u << nb) >> 5 ? (1u << nb) >> 5 : 1u;
    if (prune) {
        const uint32_t nwords = rows * words_per_row;
        for (uint32_t i = threadIdx.x; i < nwords; i += blockDim.x) s_bits[i] = bitmap[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t G = d.G;
    const uint32_t need = rows - (rows - 1) / 2;     // rows that must reach theta
    const uint32_t max_cold = rows - need;
    const uint32_t iters = (G + 31) / 32;
    constexpr int kR = T > 0 ? T : kMaxRows;

    for (uint64_t line = line_lo + warp; line < line_hi; line += nwarps) {
        const uint32_t cy = (uint32_t)(line % G);
        const uint32_t cz = (uint32_t)(line / G);
        uint64_t v[kR], step[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            if (T == 0 && r >= (int)rows) break;
            v[r] = row_value(d.seed[r], (uint32_t)lane, cy, cz);
            step[r] = d.seed[r].a0 * 32ull;
        }
        for (uint32_t it = 0; it < iters; ++it) {
            const uint32_t cx = it * 32 + lane;
            bool cand = cx < G;
            if (cand && prune) {
                if (T == 5) {
                    uint32_t hot = hot_bit(s_bits, words_per_row, 0, v[0], nb) +
                                   hot_bit(s_bits, words_per_row, 1, v[1], nb) +
                                   hot_bit(s_bits, words_per_row, 2, v[2], nb);
                    cand = false;
                    if (hot >= 1) {
                        hot += hot_bit(s_bits, words_per_row, 3, v[3], nb);
                        if (hot >= 2) cand = hot + hot_bit(s_bits, words_per_row, 4, v[4], nb) >= 3;
                    }
                } else {
                    uint32_t cold = 0;
#pragma unroll
                    for (int r = 0; r < kR; ++r) {
                        if (T == 0 && r >= (int)rows) break;
                        cold += 1u - hot_bit(s_bits, words_per_row, r, v[r], nb);
                        if (cold > max_cold) break;
                    }
                    cand = cold <= max_cold;
                }
            }
            int32_t e = 0;
            bool pass = false;
            if (cand && skip.bits && routed_cell(skip, cx, cy, cz)) cand = false;
            if (cand) {
                if (T == 5) {
                    int32_t r0 = signed_count(__ldg(C + bucket_of(v[0], d.log2w)), v[0], d.log2w);
                    int32_t r1 = signed_count(__ldg(C + d.W + bucket_of(v[1], d.log2w)), v[1], d.log2w);
                    int32_t r2 = signed_count(__ldg(C + 2 * d.W + bucket_of(v[2], d.log2w)), v[2], d.log2w);
                    int32_t r3 = signed_count(__ldg(C + 3 * d.W + bucket_of(v[3], d.log2w)), v[3], d.log2w);
                    int32_t r4 = signed_count(__ldg(C + 4 * d.W + bucket_of(v[4], d.log2w)), v[4], d.log2w);
                    e = median5(r0, r1, r2, r3, r4);
                } else {
                    int32_t ev[kMaxRows];
                    for (uint32_t r = 0; r < rows; ++r)
                        ev[r] = signed_count(__ldg(C + r * d.W + bucket_of(v[r], d.log2w)), v[r],
                                             d.log2w);
                    e = lower_median_dyn(ev, (int)rows);
                }
                pass = passes(e, theta, mode);
            }
            warp_append(pass, key_of(cx, cy, cz, G), e, out, lane);
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                if (T == 0 && r >= (int)rows) break;
                v[r] += step[r];
            }
        }
    }
}

// Hierarchical query (Algorithm 3, CSHi), second layer: every cell of the
// listed super-items (F x F x F blocks on a grid of Gs per axis) is estimated
// from this sketch and kept when it passes theta and its key lies in
// [key_lo, key_hi) and it is not routed to exact counts.  One thread per cell;
// total = ns * F^3 < 2^32.
template <int T>
__global__ void __launch_bounds__(256)
    k_expand(const int32_t *__restrict__ C, const SketchDesc d,
             const uint64_t *__restrict__ skeys, uint32_t total, uint32_t F, uint32_t Gs,
             int32_t theta, uint32_t mode, uint64_t key_lo, uint64_t key_hi, SearchOut out,
             RouteFilter skip) {
    const int lane = threadIdx.x & 31;
    const uint32_t F3 = F * F * F;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total;
         base += stride) {
        const uint32_t i = base + lane;
        bool pass = false;
        int32_t e = 0;
        uint64_t key = 0;
        if (i < total) {
            const uint64_t s = skeys[i / F3];
            const uint32_t l = i % F3;
            const uint32_t sx = (uint32_t)(s % Gs);
            const uint64_t rest = s / Gs;
            const uint32_t sy = (uint32_t)(rest % Gs), sz = (uint32_t)(rest / Gs);
            const uint32_t cx = sx * F + l % F, cy = sy * F + (l / F) % F, cz = sz * F + l / (F * F);
            key = key_of(cx, cy, cz, d.G);
            if (key >= key_lo && key < key_hi && !(skip.bits && routed_cell(skip, cx, cy, cz))) {
                if (T == 5) {
                    int32_t ev[5];
#pragma unroll
                    for (int r = 0; r < 5; ++r) {
                        const uint64_t v = row_value(d.seed[r], cx, cy, cz);
                        ev[r] = signed_count(__ldg(C + r * d.W + bucket_of(v, d.log2w)), v, d.log2w);
                    }
                    e = median5(ev[0], ev[1], ev[2], ev[3], ev[4]);
                } else {
                    int32_t ev[kMaxRows];
                    for (uint32_t r = 0; r < d.rows; ++r) {
                        const uint64_t v = row_value(d.seed[r], cx, cy, cz);
                        ev[r] = signed_count(__ldg(C + r * d.W + bucket_of(v, d.log2w)), v, d.log2w);
                    }
                    e = lower_median_dyn(ev, (int)d.rows);
                }
                pass = passes(e, theta, mode);
            }
        }
        warp_append(pass, key, e, out, lane);
    }
}

__global__ void k_hot_bitmap(const int32_t *__restrict__ C, uint64_t total, uint32_t log2w,
                             uint32_t nb, int32_t theta_hot, uint32_t *__restrict__ bitmap) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t shift = log2w - nb;
    const uint32_t words_per_row = (1u << nb) >> 5 ? (1u << nb) >> 5 : 1u;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        int64_t c = C[i];
        if ((c < 0 ? -c : c) >= (int64_t)theta_hot) {
            uint64_t r = i >> log2w;
            uint32_t sb = (uint32_t)(i & ((1ull << log2w) - 1)) >> shift;
            atomicOr(&bitmap[r * words_per_row + (sb >> 5)], 1u << (sb & 31));
        }
    }
}

__global__ void k_point_query(const int32_t *__restrict__ C, const SketchDesc d,
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
        uint32_t cy = (uint32_t)(rest % d.G);
        uint32_t cz = (uint32_t)(rest / d.G);
        int32_t ev[kMaxRows];
        for (uint32_t r = 0; r < d.rows; ++r) {
            uint64_t v = row_value(d.seed[r], cx, cy, cz);
            ev[r] = signed_count(C[r * d.W + bucket_of(v, d.log2w)], v, d.log2w);
        }
        est[i] = d.rows == 5 ? median5(ev[0], ev[1], ev[2], ev[3], ev[4])
                             : lower_median_dyn(ev, (int)d.rows);
    }
}

__device__ __forceinline__ uint64_t slot_hash(uint64_t k) {
    k ^= k >> 31;
    k *= 0x7FB5D329728EA185ull;
    k ^= k >> 27;
    k *= 0x81DADEF4BC2DD44Dull;
    return k ^ (k >> 33);
}

// Insert every valid probe key into an open-addressing set (CAS, linear
// probing; at most 1/2 full, probe length capped) and list the new ones.
__global__ void k_probe_distinct(const uint64_t *__restrict__ probe, uint64_t m,
                                 unsigned long long *__restrict__ slots, uint64_t mask,
                                 uint64_t *__restrict__ distinct,
                                 unsigned long long *__restrict__ n_distinct,
                                 uint32_t *__restrict__ overflow) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint64_t key = probe[i];
        if (key == kInvalidKey) continue;
        uint64_t h = slot_hash(key) & mask;
        bool done = false;
        for (int p = 0; p < 4096 && !done; ++p) {
            unsigned long long prev = atomicCAS(&slots[h], (unsigned long long)kInvalidKey,
                                                (unsigned long long)key);
            if (prev == kInvalidKey) {
                distinct[atomicAdd(n_distinct, 1ull)] = key;
                done = true;
            } else if (prev == key) {
                done = true;
            } else {
                h = (h + 1) & mask;
            }
        }
        if (!done) atomicOr(overflow, 1u);
    }
}

}  // namespace

uint32_t bitmap_log2_bits(uint32_t rows, uint32_t log2w, size_t smem_budget_bytes) {
    uint64_t bits_per_row = (uint64_t)smem_budget_bytes * 8 / rows;
    uint32_t nb = 5;   // at least one 32-bit word per row
    while (nb + 1 <= log2w && (1ull << (nb + 1)) <= bits_per_row) ++nb;
    if (nb > log2w) nb = log2w;   // log2w < 5: a single partially used word
    return nb;
}

cudaError_t launch_hot_bitmap(const int32_t *C, const SketchDesc &d, uint32_t nb,
                              int32_t theta_hot, uint32_t *bitmap, int max_blocks,
                              cudaStream_t s) {
    uint64_t words_per_row = (1ull << nb) >> 5 ? (1ull << nb) >> 5 : 1;
    cudaError_t e = cudaMemsetAsync(bitmap, 0, (size_t)d.rows * words_per_row * 4, s);
    if (e != cudaSuccess) return e;
    uint64_t total = (uint64_t)d.rows * d.W;
    uint64_t blocks = (total + 255) / 256;
    if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
    k_hot_bitmap<<<(unsigned)blocks, 256, 0, s>>>(C, total, d.log2w, nb, theta_hot, bitmap);
    return cudaGetLastError();
}

cudaError_t launch_full_search(const int32_t *C, const SketchDesc &d, int32_t theta,
                               SearchMode mode, const uint32_t *bitmap, uint32_t nb, int prune,
                               uint64_t line_lo, uint64_t line_hi, SearchOut out, int blocks,
                               cudaStream_t s, RouteFilter skip) {
    if (line_hi <= line_lo) return cudaSuccess;
    uint64_t words_per_row = (1ull << nb) >> 5 ? (1ull << nb) >> 5 : 1;
    size_t smem = prune ? (size_t)d.rows * words_per_row * 4 : 0;
    uint64_t warps_needed = line_hi - line_lo;
    uint64_t b = (warps_needed + 31) / 32;
    if (b > (uint64_t)blocks) b = (uint64_t)blocks;
    if (b < 1) b = 1;
    if (d.rows == 5) {
        auto k = k_full_search<5>;
        ensure_smem_limit(k, smem);
        k<<<(unsigned)b, 1024, smem, s>>>(C, d, theta, mode, bitmap, nb, prune, line_lo, line_hi,
                                         out, skip);
    } else {
        auto k = k_full_search<0>;
        ensure_smem_limit(k, smem);
        k<<<(unsigned)b, 1024, smem, s>>>(C, d, theta, mode, bitmap, nb, prune, line_lo, line_hi,
                                         out, skip);
    }
    return cudaGetLastError();
}

cudaError_t launch_expand(const int32_t *C, const SketchDesc &d, const uint64_t *skeys, uint64_t ns,
                          uint32_t F, uint32_t Gs, int32_t theta, SearchMode mode, uint64_t key_lo,
                          uint64_t key_hi, SearchOut out, int max_blocks, cudaStream_t s,
                          int *launches, RouteFilter skip) {
    const uint64_t F3 = (uint64_t)F * F * F;
    const uint64_t per = ((1ull << 31) / F3);            // super-items per launch: < 2^31 cells
    for (uint64_t s0 = 0; s0 < ns; s0 += per) {
        const uint64_t cnt = std::min<uint64_t>(per, ns - s0);
        const uint32_t total = (uint32_t)(cnt * F3);
        uint64_t blocks = ((uint64_t)total + 255) / 256;
        if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
        if (blocks < 1) blocks = 1;
        if (d.rows == 5)
            k_expand<5><<<(unsigned)blocks, 256, 0, s>>>(C, d, skeys + s0, total, F, Gs, theta, mode,
                                                        key_lo, key_hi, out, skip);
        else
            k_expand<0><<<(unsigned)blocks, 256, 0, s>>>(C, d, skeys + s0, total, F, Gs, theta, mode,
                                                        key_lo, key_hi, out, skip);
        *launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_point_query(const int32_t *C, const SketchDesc &d, const uint64_t *keys,
                               uint64_t m, int32_t *est, uint32_t *bad, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    uint64_t blocks = (m + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_point_query<<<(unsigned)blocks, 256, 0, s>>>(C, d, keys, m, est, bad);
    return cudaGetLastError();
}

cudaError_t launch_probe_distinct(const uint64_t *probe, uint64_t m, uint64_t *slots,
                                  uint32_t log2_slots, uint64_t *distinct,
                                  unsigned long long *n_distinct, uint32_t *overflow,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(slots, 0xFF, (size_t)8 << log2_slots, s);
    if (e != cudaSuccess || m == 0) return e;
    uint64_t blocks = (m + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_probe_distinct<<<(unsigned)blocks, 256, 0, s>>>(
        probe, m, reinterpret_cast<unsigned long long *>(slots), (1ull << log2_slots) - 1, distinct,
        n_distinct, overflow);
    return cudaGetLastError();
}

}  // namespace hs
