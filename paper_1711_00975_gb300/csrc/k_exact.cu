// k_exact.cu - the exact algorithm of Sec. 4.2: one counter per occupied
// cell, kept in an open-addressing hash table in device memory (uint64 key,
// all ones = empty, + int32 count; linear probing from a 64-bit mix of the
// key, at most kTableProbes slots per key).  Used as the ground truth of recall and
// for the router's training labels.
#include <algorithm>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

// count every particle's cell
__global__ void k_exact_count(const float *__restrict__ xyz, uint64_t n, const SketchDesc d,
                              unsigned long long *__restrict__ keys, int32_t *__restrict__ counts,
                              uint64_t mask, uint32_t *__restrict__ overflow) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t cx, cy, cz;
        bool ok = axis_cell(xyz[3 * i], d.inv_cell, d.G, cx);
        ok &= axis_cell(xyz[3 * i + 1], d.inv_cell, d.G, cy);
        ok &= axis_cell(xyz[3 * i + 2], d.inv_cell, d.G, cz);
        if (!ok) continue;
        if (!table_add(keys, counts, mask, key_of(cx, cy, cz, d.G), kTableProbes))
            atomicOr(overflow, 1u);
    }
}

// occupied slots -> (key, count) lists
__global__ void k_table_list(const unsigned long long *__restrict__ keys,
                             const int32_t *__restrict__ counts, uint64_t slots,
                             uint64_t *__restrict__ out_keys, int32_t *__restrict__ out_counts,
                             unsigned long long *__restrict__ n_out, uint64_t cap) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < slots; base += stride) {
        const uint64_t i = base + threadIdx.x;
        const bool on = i < slots && keys[i] != kInvalidKey;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, on);
        if (!m) continue;
        unsigned long long b0 = 0;
        if (lane == __ffs(m) - 1) b0 = atomicAdd(n_out, (unsigned long long)__popc(m));
        b0 = __shfl_sync(0xFFFFFFFFu, b0, __ffs(m) - 1);
        if (on) {
            unsigned long long j = b0 + __popc(m & ((1u << lane) - 1u));
            if (j < cap) {
                out_keys[j] = keys[i];
                out_counts[j] = counts[i];
            }
        }
    }
}

}  // namespace

namespace {

// counts[i] = count of keys[i] (0 if absent): probe until the key or an empty slot
__global__ void k_exact_query(const unsigned long long *__restrict__ tkeys,
                              const int32_t *__restrict__ tcounts, uint64_t mask,
                              const uint64_t *__restrict__ keys, uint64_t m,
                              int32_t *__restrict__ counts) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint64_t key = keys[i];
        uint64_t s = table_hash(key) & mask;
        int32_t c = 0;
        for (int p = 0; p < kTableProbes; ++p) {
            const unsigned long long cur = tkeys[s];
            if (cur == key) {
                c = tcounts[s];
                break;
            }
            if (cur == kInvalidKey) break;
            s = (s + 1) & mask;
        }
        counts[i] = c;
    }
}

}  // namespace

cudaError_t launch_exact_count(const float *xyz, uint64_t n, const SketchDesc &d,
                               unsigned long long *keys, int32_t *counts, uint64_t slots,
                               uint32_t *overflow, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 8192);
    k_exact_count<<<(unsigned)blocks, 256, 0, s>>>(xyz, n, d, keys, counts, slots - 1, overflow);
    return cudaGetLastError();
}

cudaError_t launch_table_list(const unsigned long long *keys, const int32_t *counts, uint64_t slots,
                              uint64_t *out_keys, int32_t *out_counts, unsigned long long *n_out,
                              uint64_t cap, cudaStream_t s) {
    uint64_t blocks = std::min<uint64_t>((slots + 255) / 256, 8192);
    k_table_list<<<(unsigned)blocks, 256, 0, s>>>(keys, counts, slots, out_keys, out_counts, n_out,
                                                  cap);
    return cudaGetLastError();
}

cudaError_t launch_exact_query(const unsigned long long *tkeys, const int32_t *tcounts,
                               uint64_t slots, const uint64_t *keys, uint64_t m, int32_t *counts,
                               cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((m + 255) / 256, 8192);
    k_exact_query<<<(unsigned)blocks, 256, 0, s>>>(tkeys, tcounts, slots - 1, keys, m, counts);
    return cudaGetLastError();
}

}  // namespace hs
