// k_select.cu - the k best candidates by (estimate desc, key asc).
//
// Stands in for the paper's top-k bookkeeping (Algorithm 1 keeps a heap of size
// k; Sec. 3.1 "GPU without heap" keeps an array of items above a threshold and
// raises the threshold when it grows past k).  Every candidate gets a 96-bit
// rank value R = ((est XOR 2^31) << 64) | ~key, so a larger R ranks first and
// all R are distinct.  The k-th largest R is found by a most-significant-digit
// radix select (8-bit digits, one histogram pass per digit); the entries with
// R at or above it are then placed by counting, for each, how many others
// rank before it.
#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

__device__ __forceinline__ uint32_t rank_hi(int32_t est) { return (uint32_t)est ^ 0x80000000u; }
__device__ __forceinline__ uint64_t rank_lo(uint64_t key) { return ~key; }

// digit p of R (p = 0 is the most significant); digits 0..3 from hi, 4..11 from lo
__device__ __forceinline__ uint32_t digit_of(uint32_t hi, uint64_t lo, int p) {
    return p < 4 ? (hi >> (24 - 8 * p)) & 0xFFu : (uint32_t)(lo >> (56 - 8 * (p - 4))) & 0xFFu;
}

__device__ __forceinline__ uint32_t hi_mask(int p) {   // digits 0..p-1 of hi decided
    return p <= 0 ? 0u : (p >= 4 ? 0xFFFFFFFFu : 0xFFFFFFFFu << (32 - 8 * p));
}
__device__ __forceinline__ uint64_t lo_mask(int p) {   // digits 4..p-1 decided
    int q = p - 4;
    return q <= 0 ? 0ull : (q >= 8 ? ~0ull : ~0ull << (64 - 8 * q));
}

__global__ void k_select_hist(const uint64_t *__restrict__ key, const int32_t *__restrict__ est,
                              uint64_t m, const SelectState *__restrict__ st, int p,
                              unsigned long long *__restrict__ hist) {
    __shared__ unsigned int sh[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t mh = hi_mask(p);
    const uint64_t ml = lo_mask(p);
    const uint32_t ph = st->hi & mh;   // compare only the digits decided so far
    const uint64_t pl = st->lo & ml;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint32_t hi = rank_hi(est[i]);
        uint64_t lo = rank_lo(key[i]);
        if ((hi & mh) == ph && (lo & ml) == pl) atomicAdd(&sh[digit_of(hi, lo, p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// Choose digit p: the largest d whose bucket holds the k_rem-th best entry.
__global__ void k_select_pick(SelectState *st, int p, unsigned long long *hist) {
    if (threadIdx.x == 0) {
        uint64_t above = 0;
        int d = 255;
        for (; d > 0; --d) {
            if (above + hist[d] >= st->k_rem) break;
            above += hist[d];
        }
        st->k_rem -= above;
        if (p < 4) st->hi |= (uint32_t)d << (24 - 8 * p);
        else st->lo |= (uint64_t)d << (56 - 8 * (p - 4));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

__global__ void k_select_init(SelectState *st, uint64_t k, uint64_t lo_fixed) {
    st->hi = 0;
    st->pad = 0;
    st->lo = lo_fixed;
    st->k_rem = k;
}

// entries with R >= threshold (or all), appended in arbitrary order
__global__ void k_take(const uint64_t *__restrict__ key, const int32_t *__restrict__ est,
                       uint64_t m, const SelectState *__restrict__ st, int all,
                       uint64_t *__restrict__ tk, int32_t *__restrict__ te,
                       unsigned long long *__restrict__ cnt, uint64_t cap) {
    const uint32_t th = st->hi;
    const uint64_t tl = st->lo;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint32_t hi = rank_hi(est[i]);
        uint64_t lo = rank_lo(key[i]);
        if (all || hi > th || (hi == th && lo >= tl)) {
            unsigned long long j = atomicAdd(cnt, 1ull);
            if (j < cap) {
                tk[j] = key[i];
                te[j] = est[i];
            }
        }
    }
}

// rank[i] += number of entries of slice blockIdx.y ranked before entry i: the
// entries are split over blockIdx.x (one per thread) and the slices of the
// comparison range (`slice` entries each) over blockIdx.y, staged through
// shared memory.  Small blocks and slices spread a top-k of 10^4 entries over
// about 400 blocks.
constexpr uint32_t kRankThreads = 256;
constexpr uint32_t kRankSlice = 1024;

__global__ void __launch_bounds__(kRankThreads)
    k_rank_count(const uint64_t *__restrict__ tk, const int32_t *__restrict__ te, uint64_t n,
                 uint64_t slice, uint32_t *__restrict__ rank) {
    __shared__ uint32_t s_hi[kRankThreads];
    __shared__ uint64_t s_lo[kRankThreads];
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t hi = 0;
    uint64_t lo = 0;
    if (i < n) {
        hi = rank_hi(te[i]);
        lo = rank_lo(tk[i]);
    }
    const uint64_t s0 = (uint64_t)blockIdx.y * slice;
    const uint64_t s1 = s0 + slice < n ? s0 + slice : n;
    uint32_t before = 0;
    for (uint64_t base = s0; base < s1; base += blockDim.x) {
        const uint64_t j = base + threadIdx.x;
        __syncthreads();
        if (j < s1) {
            s_hi[threadIdx.x] = rank_hi(te[j]);
            s_lo[threadIdx.x] = rank_lo(tk[j]);
        }
        __syncthreads();
        const uint32_t lim = (uint32_t)(s1 - base < blockDim.x ? s1 - base : blockDim.x);
        for (uint32_t q = 0; q < lim; ++q) {
            const uint32_t h2 = s_hi[q];
            const uint64_t l2 = s_lo[q];
            before += (h2 > hi) || (h2 == hi && l2 > lo);
        }
    }
    if (i < n && before) atomicAdd(&rank[i], before);
}

// out[rank(i)] = entry i
__global__ void k_rank_place(const uint64_t *__restrict__ tk, const int32_t *__restrict__ te,
                             const uint32_t *__restrict__ rank, uint64_t n,
                             uint64_t *__restrict__ ok, int32_t *__restrict__ oe) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        ok[rank[i]] = tk[i];
        oe[rank[i]] = te[i];
    }
}

// The whole radix select in one block, for small entry counts: each digit pass
// builds its histogram in shared memory and thread 0 picks the digit.
__global__ void __launch_bounds__(1024)
    k_select_small(const uint64_t *__restrict__ key, const int32_t *__restrict__ est, uint64_t m,
                   uint64_t k, uint64_t lo_fixed, uint32_t fixed_bytes, SelectState *st) {
    __shared__ unsigned int sh[256];
    __shared__ uint32_t s_hi;
    __shared__ uint64_t s_lo, s_k;
    if (threadIdx.x == 0) {
        s_hi = 0;
        s_lo = lo_fixed;
        s_k = k;
    }
    for (int p = 0; p < 12; ++p) {
        if (p >= 4 && (uint32_t)(p - 4) < fixed_bytes) continue;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
        __syncthreads();
        const uint32_t mh = hi_mask(p);
        const uint64_t ml = lo_mask(p);
        const uint32_t ph = s_hi & mh;
        const uint64_t pl = s_lo & ml;
        for (uint64_t i = threadIdx.x; i < m; i += blockDim.x) {
            uint32_t hi = rank_hi(est[i]);
            uint64_t lo = rank_lo(key[i]);
            if ((hi & mh) == ph && (lo & ml) == pl) atomicAdd(&sh[digit_of(hi, lo, p)], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t above = 0;
            int d = 255;
            for (; d > 0; --d) {
                if (above + sh[d] >= s_k) break;
                above += sh[d];
            }
            s_k -= above;
            if (p < 4) s_hi |= (uint32_t)d << (24 - 8 * p);
            else s_lo |= (uint64_t)d << (56 - 8 * (p - 4));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->hi = s_hi;
        st->pad = 0;
        st->lo = s_lo;
        st->k_rem = s_k;
    }
}

}  // namespace

cudaError_t launch_select_kth(const uint64_t *key, const int32_t *est, uint64_t m, uint64_t k,
                              uint32_t key_bits, SelectState *state, unsigned long long *hist,
                              int blocks, cudaStream_t s, int *launches) {
    // ~key has its top (64 - key_bits) bits set for every key; whole bytes of
    // them are decided up front and their passes skipped.
    uint32_t fixed_bytes = key_bits >= 64 ? 0 : (64 - key_bits) / 8;
    uint64_t lo_fixed = fixed_bytes ? (~0ull << (64 - 8 * fixed_bytes)) : 0ull;
    if (m <= (1ull << 17)) {     // one block: a few hundred entries per thread at most
        k_select_small<<<1, 1024, 0, s>>>(key, est, m, k, lo_fixed, fixed_bytes, state);
        *launches += 1;
        return cudaGetLastError();
    }
    k_select_init<<<1, 1, 0, s>>>(state, k, lo_fixed);
    cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    *launches += 1;
    uint64_t b = (m + 255) / 256;
    if (b > (uint64_t)blocks) b = (uint64_t)blocks;
    if (b < 1) b = 1;
    for (int p = 0; p < 12; ++p) {
        if (p >= 4 && (uint32_t)(p - 4) < fixed_bytes) continue;
        k_select_hist<<<(unsigned)b, 256, 0, s>>>(key, est, m, state, p, hist);
        k_select_pick<<<1, 256, 0, s>>>(state, p, hist);
        *launches += 2;
    }
    return cudaGetLastError();
}

cudaError_t launch_take_sorted(const uint64_t *key, const int32_t *est, uint64_t m,
                               const SelectState *state, int all, uint64_t *tmp_key,
                               int32_t *tmp_est, unsigned long long *tmp_count, uint32_t *tmp_rank,
                               uint64_t n_take, uint64_t *out_key, int32_t *out_est, int blocks,
                               cudaStream_t s, int *launches) {
    cudaError_t e = cudaMemsetAsync(tmp_count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    uint64_t b = (m + 255) / 256;
    if (b > (uint64_t)blocks) b = (uint64_t)blocks;
    if (b < 1) b = 1;
    k_take<<<(unsigned)b, 256, 0, s>>>(key, est, m, state, all, tmp_key, tmp_est, tmp_count,
                                       n_take);
    if (n_take == 0) {
        *launches += 1;
        return cudaGetLastError();
    }
    e = cudaMemsetAsync(tmp_rank, 0, n_take * 4, s);
    if (e != cudaSuccess) return e;
    uint64_t slice = kRankSlice;
    while ((n_take + slice - 1) / slice > 65535) slice *= 2;   // grid.y limit
    const dim3 grid((unsigned)((n_take + kRankThreads - 1) / kRankThreads),
                    (unsigned)((n_take + slice - 1) / slice));
    k_rank_count<<<grid, kRankThreads, 0, s>>>(tmp_key, tmp_est, n_take, slice, tmp_rank);
    k_rank_place<<<(unsigned)((n_take + 255) / 256), 256, 0, s>>>(tmp_key, tmp_est, tmp_rank, n_take,
                                                                 out_key, out_est);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace hs
