// k_update.cu - the stream-processing kernel (update mode of Count Sketch with
// Full Search, arXiv:1711.00975 Algorithm 1 / Sec. 3.1 "GPU without heap").
//
// Per particle: mesh reduction to a cell (Sec. 2.1), Bernoulli sampling by the
// particle's global index (Sec. 3.1), then Add (Sec. 2.2): for each row r,
// C[r][bucket_r] += sign_r.  The paper's GPU design gives one block per stream
// item and one thread per row (Algorithm 4, Update); here one thread owns four
// particles and all rows, so the particle stream is read with 16-byte
// coalesced loads (three float4 = four xyz triples) marked evict-first, and the
// counter updates are fire-and-forget reductions (RED) that resolve in L2.
// Counters are uint32 so the wrap-around of int32 two's complement is defined.
#include <algorithm>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

struct UpdateArgs {
    uint64_t n;
    uint64_t g0;           // global index of particle 0 of this launch
    uint64_t thr;          // keep iff splitmix64(g) < thr (unless keep_all)
    uint64_t sample_seed;
    uint64_t *probe;       // probe[g - probe_base] = key for probe_base <= g < probe_end
    uint64_t probe_base;
    uint64_t probe_end;
    uint32_t keep_all;
    uint32_t band_lo;      // only buckets in [band_lo, band_hi) are updated
    uint32_t band_hi;
};

template <int T>
__device__ __forceinline__ void add_particle(float x, float y, float z, uint64_t g,
                                             const SketchDesc &d, const UpdateArgs &a,
                                             uint32_t *__restrict__ C) {
    bool keep = a.keep_all || splitmix64_at(a.sample_seed, g) < a.thr;
    uint32_t cx = 0, cy = 0, cz = 0;
    const bool valid = particle_cell(d, x, y, z, cx, cy, cz);
    if (g - a.probe_base < a.probe_end - a.probe_base)
        a.probe[g - a.probe_base] = valid ? key_of(cx, cy, cz, d.G) : kInvalidKey;
    if (!(keep && valid)) return;
    constexpr int kRows = T > 0 ? T : kMaxRows;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (T == 0 && r >= (int)d.rows) break;
        uint64_t v = row_value(d.seed[r], cx, cy, cz);
        uint32_t b = bucket_of(v, d.log2w);
        if (b >= a.band_lo && b < a.band_hi)
            atomicAdd(&C[(uint64_t)r * d.W + b], sign_of(v, d.log2w));
    }
}

// xyz 16-byte aligned: thread q owns particles 4q .. 4q+3 (48 bytes, three float4).
template <int T>
__global__ void __launch_bounds__(256) k_update_vec4(const float *__restrict__ xyz,
                                                     const SketchDesc d, const UpdateArgs a,
                                                     uint32_t *__restrict__ C) {
    const uint64_t ngroups = a.n >> 2;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float4 *p4 = reinterpret_cast<const float4 *>(xyz);
    for (uint64_t q = tid; q < ngroups; q += stride) {
        float4 u = __ldcs(p4 + 3 * q);
        float4 v = __ldcs(p4 + 3 * q + 1);
        float4 w = __ldcs(p4 + 3 * q + 2);
        uint64_t g = a.g0 + 4 * q;
        add_particle<T>(u.x, u.y, u.z, g, d, a, C);
        add_particle<T>(u.w, v.x, v.y, g + 1, d, a, C);
        add_particle<T>(v.z, v.w, w.x, g + 2, d, a, C);
        add_particle<T>(w.y, w.z, w.w, g + 3, d, a, C);
    }
    // the n % 4 particles after the last full group
    uint64_t i = (ngroups << 2) + tid;
    if (i < a.n)
        add_particle<T>(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1), __ldcs(xyz + 3 * i + 2),
                        a.g0 + i, d, a, C);
}

// any 4-byte aligned xyz: one particle per thread per step
template <int T>
__global__ void __launch_bounds__(256) k_update_scalar(const float *__restrict__ xyz,
                                                       const SketchDesc d, const UpdateArgs a,
                                                       uint32_t *__restrict__ C) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        add_particle<T>(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1), __ldcs(xyz + 3 * i + 2),
                        a.g0 + i, d, a, C);
}

// packed records: one 8-byte record per particle
template <int T>
__device__ __forceinline__ void add_record(uint64_t p, uint64_t g, const SketchDesc &d,
                                           const UpdateArgs &a, uint32_t *__restrict__ C) {
    bool keep = a.keep_all || splitmix64_at(a.sample_seed, g) < a.thr;
    uint32_t cx, cy, cz;
    const bool valid = packed_cell(d, p, cx, cy, cz);
    if (g - a.probe_base < a.probe_end - a.probe_base)
        a.probe[g - a.probe_base] = valid ? key_of(cx, cy, cz, d.G) : kInvalidKey;
    if (!(keep && valid)) return;
    constexpr int kRows = T > 0 ? T : kMaxRows;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (T == 0 && r >= (int)d.rows) break;
        uint64_t v = row_value(d.seed[r], cx, cy, cz);
        uint32_t b = bucket_of(v, d.log2w);
        if (b >= a.band_lo && b < a.band_hi)
            atomicAdd(&C[(uint64_t)r * d.W + b], sign_of(v, d.log2w));
    }
}

template <int T>
__global__ void __launch_bounds__(256) k_update_packed(const uint64_t *__restrict__ rec,
                                                       const SketchDesc d, const UpdateArgs a,
                                                       uint32_t *__restrict__ C) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        add_record<T>(__ldcs(reinterpret_cast<const unsigned long long *>(rec) + i), a.g0 + i, d,
                      a, C);
}

// packed records of float32 positions (the quantisation of the mesh reduction
// on a mesh of 2^21 cells per axis)
__global__ void __launch_bounds__(256) k_pack(const float *__restrict__ xyz, uint64_t n,
                                              float inv, uint64_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t q[3];
        bool ok = axis_cell(xyz[3 * i], inv, 1u << kPackBits, q[0]);
        ok &= axis_cell(xyz[3 * i + 1], inv, 1u << kPackBits, q[1]);
        ok &= axis_cell(xyz[3 * i + 2], inv, 1u << kPackBits, q[2]);
        out[i] = ok ? (uint64_t)q[0] | ((uint64_t)q[1] << kPackBits) |
                          ((uint64_t)q[2] << (2 * kPackBits))
                    : kPackInvalid;
    }
}

// A probe entry of the compaction pass: the key of the particle's cell on
// the probe's mesh (the F^3 block holding it when F > 1), or kInvalidKey.
__device__ __forceinline__ void compact_probe(const CompactProbe &p, uint64_t g, bool valid,
                                              uint32_t cx, uint32_t cy, uint32_t cz) {
    if (!p.probe || g - p.base >= p.end - p.base) return;
    uint64_t key = kInvalidKey;
    if (valid) {
        if (p.F > 1) {
            cx = __umulhi(cx, p.fmagic);
            cy = __umulhi(cy, p.fmagic);
            cz = __umulhi(cz, p.fmagic);
        }
        key = key_of(cx, cy, cz, p.G);
    }
    p.probe[g - p.base] = key;
}

// Sample and quantise every particle once (PACKED: decode every packed
// position record); append the cells of the kept, valid ones.  The sampling decision and the cell are the ones the float32
// path takes (splitmix64 of the global index against the same threshold;
// axis_cell on the fine mesh).  A thread takes four particles (three float4
// when the buffer is 16-byte aligned, which page-locked host memory read over
// the host link wants); a warp reserves its records with one atomic.
__device__ __forceinline__ bool compact_cell(bool valid, uint32_t cx, uint32_t cy, uint32_t cz,
                                             uint64_t g, uint64_t thr, int keep_all, uint64_t seed,
                                             const CompactProbe &p0, const CompactProbe &p1,
                                             uint64_t &rec) {
    compact_probe(p0, g, valid, cx, cy, cz);
    compact_probe(p1, g, valid, cx, cy, cz);
    rec = (uint64_t)cx | ((uint64_t)cy << kPackBits) | ((uint64_t)cz << (2 * kPackBits));
    return valid && (keep_all || splitmix64_at(seed, g) < thr);
}

__device__ __forceinline__ bool compact_one(float x, float y, float z, uint64_t g,
                                            const SketchDesc &d, uint64_t thr, int keep_all,
                                            uint64_t seed, const CompactProbe &p0,
                                            const CompactProbe &p1, uint64_t &rec) {
    uint32_t cx = 0, cy = 0, cz = 0;
    const bool valid = particle_cell(d, x, y, z, cx, cy, cz);
    return compact_cell(valid, cx, cy, cz, g, thr, keep_all, seed, p0, p1, rec);
}

// the same for a packed position record (the cell packed_cell gives)
__device__ __forceinline__ bool compact_rec(uint64_t p, uint64_t g, const SketchDesc &d, uint64_t thr,
                                            int keep_all, uint64_t seed, const CompactProbe &p0,
                                            const CompactProbe &p1, uint64_t &rec) {
    uint32_t cx = 0, cy = 0, cz = 0;
    const bool valid = packed_cell(d, p, cx, cy, cz);
    return compact_cell(valid, cx, cy, cz, g, thr, keep_all, seed, p0, p1, rec);
}

template <bool PACKED>
__global__ void __launch_bounds__(256) k_compact(const float *__restrict__ xyz, uint64_t n,
                                                 uint64_t g0, const SketchDesc d, uint64_t thr,
                                                 int keep_all, int vec, uint64_t seed,
                                                 const CompactProbe p0, const CompactProbe p1,
                                                 uint64_t *__restrict__ cells,
                                                 unsigned long long *__restrict__ count) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t groups = (n + 3) / 4, full = vec ? n / 4 : 0;
    const float4 *p4 = reinterpret_cast<const float4 *>(xyz);
    for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5; base < groups;
         base += warps << 5) {                                   // warp-uniform
        const uint64_t q = base + lane;
        uint64_t rec[4] = {0, 0, 0, 0};
        uint32_t keep = 0;
        if (PACKED && q < groups) {                     // four records: two 16-byte loads
            const unsigned long long *r8 = reinterpret_cast<const unsigned long long *>(xyz);
            uint64_t p[4];
            if (q < full) {
                const uint4 ua = __ldcs(reinterpret_cast<const uint4 *>(r8) + 2 * q);
                const uint4 ub = __ldcs(reinterpret_cast<const uint4 *>(r8) + 2 * q + 1);
                p[0] = ua.x | ((uint64_t)ua.y << 32);
                p[1] = ua.z | ((uint64_t)ua.w << 32);
                p[2] = ub.x | ((uint64_t)ub.y << 32);
                p[3] = ub.z | ((uint64_t)ub.w << 32);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) p[j] = 4 * q + j < n ? __ldcs(r8 + 4 * q + j) : 0ull;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (4 * q + j < n)
                    keep |= (uint32_t)compact_rec(p[j], g0 + 4 * q + j, d, thr, keep_all, seed, p0, p1,
                                                  rec[j]) << j;
        } else if (!PACKED && q < full) {
            const float4 u = __ldcs(p4 + 3 * q), v = __ldcs(p4 + 3 * q + 1), w = __ldcs(p4 + 3 * q + 2);
            const float px[4] = {u.x, u.w, v.z, w.y}, py[4] = {u.y, v.x, v.w, w.z},
                        pz[4] = {u.z, v.y, w.x, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                keep |= (uint32_t)compact_one(px[j], py[j], pz[j], g0 + 4 * q + j, d, thr, keep_all,
                                              seed, p0, p1, rec[j]) << j;
        } else if (!PACKED && q < groups) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t i = 4 * q + j;
                if (i < n)
                    keep |= (uint32_t)compact_one(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                                  __ldcs(xyz + 3 * i + 2), g0 + i, d, thr, keep_all,
                                                  seed, p0, p1, rec[j]) << j;
            }
        }
        const uint32_t c = __popc(keep);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        unsigned long long at = 0;
        if (lane == 0 && total) at = atomicAdd(count, (unsigned long long)total);
        at = __shfl_sync(0xFFFFFFFFu, at, 0) + (incl - c);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (keep & (1u << j)) cells[at++] = rec[j];
    }
}

// Random fire-and-forget adds into an n_counters table (power of two): the
// L2 reduction rate that bounds the update when the particle stream does not.
__global__ void __launch_bounds__(256) k_red_rate(uint32_t *__restrict__ T, uint64_t mask,
                                                  uint64_t ops_per_thread, uint64_t salt) {
    uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t s = splitmix64_at(salt, tid);
    for (uint64_t i = 0; i < ops_per_thread; ++i) {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        atomicAdd(&T[(s >> 20) & mask], 1u);
    }
}

__global__ void k_add_counters(uint32_t *__restrict__ dst, const uint32_t *__restrict__ src,
                               uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] += src[i];
}

}  // namespace

cudaError_t launch_add_counters(int32_t *dst, const int32_t *src, uint64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_add_counters<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<uint32_t *>(dst),
                                                   reinterpret_cast<const uint32_t *>(src), n);
    return cudaGetLastError();
}

cudaError_t launch_update(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                          int32_t *C, double rate, uint64_t sample_seed, uint64_t *probe,
                          uint64_t probe_base, uint64_t probe_cap, uint32_t band_lo, uint32_t band_hi, int max_blocks,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    UpdateArgs a;
    a.n = n;
    a.g0 = g0;
    a.keep_all = rate >= 1.0 ? 1u : 0u;
    a.thr = rate >= 1.0 ? 0 : (uint64_t)ldexp(rate, 64);
    a.sample_seed = sample_seed;
    a.probe = probe;
    a.probe_base = probe_base;
    a.probe_end = probe ? probe_base + probe_cap : probe_base;
    a.band_lo = band_lo;
    a.band_hi = band_hi;
    uint32_t *Cu = reinterpret_cast<uint32_t *>(C);
    const int threads = 256;
    bool vec = (reinterpret_cast<uintptr_t>(xyz) & 15u) == 0;
    uint64_t work = vec ? (n >> 2) + 1 : n;
    uint64_t blocks = (work + threads - 1) / threads;
    if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
    if (blocks < 1) blocks = 1;
    if (d.rows == 5) {
        if (vec) k_update_vec4<5><<<(unsigned)blocks, threads, 0, s>>>(xyz, d, a, Cu);
        else k_update_scalar<5><<<(unsigned)blocks, threads, 0, s>>>(xyz, d, a, Cu);
    } else {
        if (vec) k_update_vec4<0><<<(unsigned)blocks, threads, 0, s>>>(xyz, d, a, Cu);
        else k_update_scalar<0><<<(unsigned)blocks, threads, 0, s>>>(xyz, d, a, Cu);
    }
    return cudaGetLastError();
}

cudaError_t launch_update_packed(const uint64_t *rec, uint64_t n, uint64_t g0,
                                 const SketchDesc &d, int32_t *C, double rate,
                                 uint64_t sample_seed, uint64_t *probe, uint64_t probe_base,
                                 uint64_t probe_cap, int max_blocks, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    UpdateArgs a;
    a.n = n;
    a.g0 = g0;
    a.keep_all = rate >= 1.0 ? 1u : 0u;
    a.thr = rate >= 1.0 ? 0 : (uint64_t)ldexp(rate, 64);
    a.sample_seed = sample_seed;
    a.probe = probe;
    a.probe_base = probe_base;
    a.probe_end = probe ? probe_base + probe_cap : probe_base;
    a.band_lo = 0;
    a.band_hi = (uint32_t)d.W;
    uint32_t *Cu = reinterpret_cast<uint32_t *>(C);
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
    if (blocks < 1) blocks = 1;
    if (d.rows == 5) k_update_packed<5><<<(unsigned)blocks, 256, 0, s>>>(rec, d, a, Cu);
    else k_update_packed<0><<<(unsigned)blocks, 256, 0, s>>>(rec, d, a, Cu);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float *xyz, uint64_t n, double box, uint64_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 16384);
    k_pack<<<(unsigned)blocks, 256, 0, s>>>(xyz, n, (float)((double)(1u << kPackBits) / box), out);
    return cudaGetLastError();
}

cudaError_t launch_compact_cells(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                                 double rate, uint64_t sample_seed, const CompactProbe &p0,
                                 const CompactProbe &p1, uint64_t *cells,
                                 unsigned long long *count, int blocks, cudaStream_t s, int packed) {
    if (n == 0) return cudaSuccess;
    if (d.F != 1 || d.Gq >= (1u << kPackBits)) return cudaErrorInvalidValue;
    const bool sampled = rate < 1.0;
    const uint64_t thr = sampled ? (uint64_t)ldexp(rate, 64) : 0;
    const uint64_t want = ((n + 3) / 4 + 255) / 256;
    const int vec = (reinterpret_cast<uintptr_t>(xyz) & 15u) == 0;
    const unsigned grid = (unsigned)std::min<uint64_t>(want, (uint64_t)blocks);
    if (packed)
        k_compact<true><<<grid, 256, 0, s>>>(xyz, n, g0, d, thr, sampled ? 0 : 1, vec, sample_seed,
                                             p0, p1, cells, count);
    else
        k_compact<false><<<grid, 256, 0, s>>>(xyz, n, g0, d, thr, sampled ? 0 : 1, vec, sample_seed,
                                              p0, p1, cells, count);
    return cudaGetLastError();
}

cudaError_t launch_red_rate(uint32_t *table, uint64_t n_counters, uint64_t ops_per_thread,
                            int blocks, cudaStream_t s) {
    k_red_rate<<<blocks, 256, 0, s>>>(table, n_counters - 1, ops_per_thread, 0x1234567ull);
    return cudaGetLastError();
}

}  // namespace hs
