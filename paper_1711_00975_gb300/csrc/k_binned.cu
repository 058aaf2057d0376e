// k_binned.cu - host side of the binned update (layout, launch of the scatter
// variants of k_binned.cuh) and its second pass, the accumulation.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "k_binned.cuh"

namespace hs {

using namespace binned;

namespace {

// One block per bin: the codes of every scatter block's region are added into
// 2^S shared-memory counters, then C[bin range] += the counters and the
// regions' fills are cleared.  Warps take 256-chunk spans
// (a chunk is 8 codes, 16 bytes) of the concatenated regions in turn; lane l
// loads chunks l, l + 32, ... of its warp's span, eight in flight.
constexpr int kAccThreads = 1024;

__global__ void __launch_bounds__(kAccThreads)
    k_bin_accumulate(const BinStore B, uint32_t S, uint32_t gmagic, uint32_t *__restrict__ C) {
    extern __shared__ __align__(16) int32_t acc[];
    const uint32_t nacc = 1u << S;
    uint32_t *pre = reinterpret_cast<uint32_t *>(acc + nacc);   // nblocks + 1 chunk offsets
    const uint32_t bin = blockIdx.x, nblocks = B.nblocks;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t g = B.ngroups > 1 ? __umulhi(bin, gmagic) : 0u;
    const uint32_t cap = B.gcap[g];
    const uint64_t base = B.gbase[g] + (uint64_t)(bin - g * B.bpg) * cap;   // block 0's region
    const uint64_t stride8 = (uint64_t)B.bpg * cap / 8;                      // next block's, in chunks
    for (uint32_t i = threadIdx.x; i < nacc; i += blockDim.x) acc[i] = 0;
    if (warp == 0) {   // exclusive prefix of the regions' chunk counts
        uint32_t carry = 0;
        for (uint32_t b0 = 0; b0 < nblocks; b0 += 32) {
            const uint32_t b = b0 + lane;
            const uint32_t v = b < nblocks ? min(B.fill[(uint64_t)bin * nblocks + b], cap) / 8 : 0;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (b < nblocks) pre[b] = carry + x - v;
            carry += __shfl_sync(0xFFFFFFFFu, x, 31);
        }
        if (lane == 0) pre[nblocks] = carry;
    }
    __syncthreads();
    const uint32_t total = pre[nblocks];
    const uint4 *src = reinterpret_cast<const uint4 *>(B.codes + base);
    for (uint32_t span = warp * 256; span < total; span += nwarps * 256) {
        // region of the span's first chunk (binary search), then upward per chunk
        uint32_t lo = 0, hi = nblocks;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (pre[mid] <= span) lo = mid; else hi = mid;
        }
        uint32_t seg = lo;
        uint4 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t c = span + lane + 32 * u;
            if (c < total) {
                while (pre[seg + 1] <= c) ++seg;
                w[u] = __ldcs(src + (uint64_t)seg * stride8 + (c - pre[seg]));
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (span + lane + 32 * u >= total) break;
            const uint32_t ws[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t c0 = ws[q] & 0xFFFFu, c1 = ws[q] >> 16;
                atomicAdd(&acc[c0 >> 1], (c0 & 1) ? -1 : 1);
                atomicAdd(&acc[c1 >> 1], (c1 & 1) ? -1 : 1);
            }
        }
    }
    __syncthreads();
    // C[bin range] += acc, four counters a lane access and eight accesses of a
    // lane in flight (the counters of a bin are 16-byte aligned when S >= 2);
    // all-zero quads are neither read nor written
    uint32_t *dst = C + ((uint64_t)bin << S);
    if (nacc >= 4) {
        const uint32_t nq = nacc >> 2;
        const int4 *acc4 = reinterpret_cast<const int4 *>(acc);
        uint4 *dst4 = reinterpret_cast<uint4 *>(dst);
        auto any = [](int4 a) { return (a.x | a.y | a.z | a.w) != 0; };
        for (uint32_t i0 = threadIdx.x; i0 < nq; i0 += 8 * blockDim.x) {
            uint4 c[8];
#pragma unroll
            for (uint32_t u = 0; u < 8; ++u) {
                const uint32_t i = i0 + u * blockDim.x;
                if (i < nq && any(acc4[i])) c[u] = dst4[i];
            }
#pragma unroll
            for (uint32_t u = 0; u < 8; ++u) {
                const uint32_t i = i0 + u * blockDim.x;
                if (i < nq) {
                    const int4 a = acc4[i];
                    if (any(a))
                        dst4[i] = make_uint4(c[u].x + (uint32_t)a.x, c[u].y + (uint32_t)a.y,
                                             c[u].z + (uint32_t)a.z, c[u].w + (uint32_t)a.w);
                }
            }
        }
    } else {
        for (uint32_t i = threadIdx.x; i < nacc; i += blockDim.x) {
            const int32_t v = acc[i];
            if (v) dst[i] += (uint32_t)v;
        }
    }
    for (uint32_t b = threadIdx.x; b < nblocks; b += blockDim.x) B.fill[(uint64_t)bin * nblocks + b] = 0;
}

uint32_t magic_of(uint32_t d) { return (uint32_t)((0x100000000ull + d - 1) / d); }

// Per scatter tile of a batch: its first and last particle's volumes
// (first | last << 16; the volume of particle i is the last whose start <= i).
__global__ void k_tile_vols(const VolumeDesc *__restrict__ vols, uint32_t nvol, uint64_t n,
                            uint64_t ntiles, uint32_t *__restrict__ out) {
    auto vol = [&](uint64_t i) {
        uint32_t lo = 0, hi = nvol;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (vols[mid].start <= i) lo = mid; else hi = mid;
        }
        return lo;
    };
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += stride) {
        const uint64_t i0 = t * kScatterTile;
        const uint64_t i1 = (i0 + kScatterTile < n ? i0 + kScatterTile : n) - 1;
        out[t] = vol(i0) | (vol(i1) << 16);
    }
}

}  // namespace

cudaError_t ensure_smem_limit(const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> limits;   // (kernel, device) -> bytes
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = limits[{kernel, dev}];
    if (cur >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

BinLayout bin_layout(const SketchDesc &d, size_t smem_budget, bool single_pass) {
    BinLayout L{};
    L.S = d.log2w < 15 ? d.log2w : 15;
    const uint64_t nb = (uint64_t)d.rows << (d.log2w - L.S);
    if (nb >= 65536) return L;                // bins are 16-bit numbers (group division)
    L.nbins = (uint32_t)nb;
    const uint32_t bpr = 1u << (d.log2w - L.S);
    const size_t budget = std::min<size_t>(smem_budget, kSmemLimit);
    // as many rows a launch as fit even a sampled call's layout (with queues);
    // a sketch whose rings do not fit at once stages its rows in passes
    for (uint32_t rpp = d.rows; rpp >= 1; --rpp) {
        if (ring_slot(rpp * bpr, kMaxBinGroups, 1, budget) != 0) {
            L.rows_per_pass = rpp;
            break;
        }
        if (single_pass) return L;
    }
    if (L.rows_per_pass == 0) return L;
    L.slot = ring_slot(L.rows_per_pass * bpr, kMaxBinGroups, 0, budget);
    L.half = L.slot / 2;
    L.smem = smem_layout(L.rows_per_pass * bpr, L.slot, kMaxBinGroups, 0).total;
    return L;
}

BatchRing batch_ring(const BinLayout &L, const SketchDesc &d, uint32_t ngroups, double rate,
                     uint32_t slot_cap, uint32_t wvols_cap) {
    const uint32_t lbpr = d.log2w - L.S;
    const uint32_t bpv = d.rows << lbpr;
    const bool sampled = rate < 1.0;
    // codes one tile adds to each bin of its volume; a ring holds a half
    // left over from the last flush and one tile's codes
    const double per_tile = kScatterTile * rate / (double)(1u << lbpr);
    BatchRing r{0, 0, 0};
    for (uint32_t wv = wvols_cap >= 4 || wvols_cap == 0 ? 4 : (wvols_cap >= 2 ? 2 : 1); wv >= 1; wv >>= 1) {
        uint32_t slot = ring_slot(wv * bpv, ngroups, sampled ? 1 : 0, kSmemLimit, true);
        if (slot_cap && slot_cap < slot) slot = slot_cap;
        if (slot >= 16 && (slot >= 2.5 * per_tile || wv == 1)) {
            r = BatchRing{wv, wv * bpv, slot};
            break;
        }
    }
    return r;
}

cudaError_t launch_bin_scatter(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                               int32_t *C, double rate, uint64_t sample_seed, uint64_t *probe,
                               uint64_t probe_base, uint64_t probe_cap, const BinLayout &L,
                               const BinStore &B, cudaStream_t s, const VolumeDesc *vols,
                               uint32_t nvol, uint32_t probe_per_vol, const RouteTarget *route,
                               int packed, uint32_t rounds, uint32_t slot, uint32_t *tile_vols,
                               const unsigned long long *n_dev, uint64_t n_base, uint32_t wvols_cap) {
    if (n == 0) return cudaSuccess;
    if (vols && (!tile_vols || nvol == 0 || nvol > 65535)) return cudaErrorInvalidValue;
    if (L.slot == 0 || B.nblocks == 0 || !B.codes || !B.fill || B.ngroups == 0 ||
        B.ngroups > kMaxBinGroups || (uint64_t)B.bpg * B.ngroups != L.nbins)
        return cudaErrorInvalidValue;
    if (packed && (vols || route)) return cudaErrorInvalidValue;   // float input only there
    if (packed == 2 && (!n_dev || rate < 1.0 || probe)) return cudaErrorInvalidValue;   // already sampled
    ScatterArgs a;
    std::memset(&a, 0, sizeof(a));
    const bool sampled = rate < 1.0;
    a.n = n;
    a.n_dev = packed == 2 ? n_dev : nullptr;
    a.n_base = n_base;
    a.g0 = g0;
    a.thr = sampled ? (uint64_t)ldexp(rate, 64) : 0;
    a.sample_seed = sample_seed;
    a.probe = probe;
    a.S = L.S;
    a.hshift = 31 - d.log2w;
    a.code_mask = (2u << L.S) - 1u;
    a.gmagic = magic_of(B.bpg);
    // two tiles between flush phases (about 12 codes a bin at 2560 bins); at
    // sample rate r a tile stages about r times the codes of a full tile
    a.rounds = rounds ? rounds
                      : (sampled ? (uint32_t)std::min(6.0, std::max(2.0, std::floor(2.0 / rate))) : 2u);
    a.B = B;
    a.route = route ? route->filter : RouteFilter{nullptr, 0, 0, 0};
    a.rprefix = route ? route->prefix : nullptr;
    a.rblocks = route ? route->blocks : nullptr;
    a.vols = vols;
    a.nvol = vols ? nvol : 0;
    a.probe_per_vol = probe_per_vol;
    const uint32_t lbpr = d.log2w - L.S;
    const uint32_t rpp = L.rows_per_pass ? L.rows_per_pass : d.rows;
    if (vols && rpp < d.rows) return cudaErrorInvalidValue;   // a batch stages in one pass
    uint32_t *Cu = reinterpret_cast<uint32_t *>(C);
    // one launch per pass over the rows [row0, row0 + nrows); only the first
    // pass records the probe and counts routed particles
    for (uint32_t row0 = 0; row0 < d.rows; row0 += rpp) {
        a.row0 = row0;
        a.nrows = std::min(rpp, d.rows - row0);
        a.bin_base = vols ? 0u : row0 << lbpr;
        a.nbins = vols ? L.nbins : a.nrows << lbpr;
        for (uint32_t i = 0; i < kMaxRows; ++i) a.rbase[i] = i << lbpr;
        a.route_adds = row0 == 0 ? 1u : 0u;
        a.probe_base = probe_base;
        a.probe_end = probe && row0 == 0 ? probe_base + probe_cap : probe_base;
        a.slot = ring_slot(a.nbins, B.ngroups, sampled ? 1 : 0, kSmemLimit);
        if (slot && slot < a.slot) a.slot = slot;     // a shallower ring (power of two)
        if (vols) {   // rings for a window of volumes, one tile between flushes
            const BatchRing br = batch_ring(L, d, B.ngroups, rate, slot, wvols_cap);
            if (br.wvols == 0) return cudaErrorInvalidValue;
            a.wvols = br.wvols;
            a.bpv = d.rows << lbpr;
            a.nbins = br.nslots;
            a.slot = br.slot;
            a.rounds = 1;
            a.tvols = tile_vols;
            const uint64_t ntiles = (n + kScatterTile - 1) / kScatterTile;
            k_tile_vols<<<(unsigned)std::min<uint64_t>((ntiles + 255) / 256, 1024), 256, 0, s>>>(
                vols, nvol, n, ntiles, tile_vols);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        if (a.slot < 16 || (a.slot & (a.slot - 1))) return cudaErrorInvalidValue;
        a.half = a.slot / 2;
        a.team = a.half <= 64 ? 1u : 32u;
        const size_t smem = smem_layout(a.nbins, a.slot, B.ngroups, sampled ? 1 : 0, a.wvols != 0).total;
        cudaError_t e;
        if (vols) {
            e = launch_modes_batch_route(kModeBatch, xyz, d, a, sampled, smem, Cu, s);
        } else if (route) {
            e = launch_modes_batch_route(kModeRoute, xyz, d, a, sampled, smem, Cu, s);
        } else if (packed == 2) {
            e = launch_modes_cells(d.F > 1 ? kModeSuperCells : kModeCells, xyz, d, a, smem, Cu, s);
        } else {
            const int mode = packed ? (d.F > 1 ? kModeSuperPacked : kModePlainPacked)
                                    : (d.F > 1 ? kModeSuper : kModePlain);
            e = launch_modes_sketch(mode, xyz, d, a, sampled, smem, Cu, s);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_bin_accumulate(const BinLayout &L, const BinStore &B, int32_t *C,
                                  cudaStream_t s) {
    if (L.slot == 0 || B.nblocks == 0 || B.ngroups == 0) return cudaErrorInvalidValue;
    const size_t smem = ((size_t)4 << L.S) + 4 * ((size_t)B.nblocks + 1);
    cudaError_t e = ensure_smem_limit(k_bin_accumulate, smem);
    if (e != cudaSuccess) return e;
    k_bin_accumulate<<<L.nbins, kAccThreads, smem, s>>>(B, L.S, magic_of(B.bpg),
                                                        reinterpret_cast<uint32_t *>(C));
    return cudaGetLastError();
}

namespace binned {

// the single-sketch variants: plain, super-item, and both from packed records
cudaError_t launch_modes_sketch(int mode, const float *xyz, const SketchDesc &d, const ScatterArgs &a,
                                bool sampled, size_t smem, uint32_t *C, cudaStream_t s) {
    switch (mode) {
    case kModePlain: return launch_mode<kModePlain>(xyz, d, a, sampled, smem, C, s);
    case kModeSuper: return launch_mode<kModeSuper>(xyz, d, a, sampled, smem, C, s);
    case kModePlainPacked: return launch_mode<kModePlainPacked>(xyz, d, a, sampled, smem, C, s);
    case kModeSuperPacked: return launch_mode<kModeSuperPacked>(xyz, d, a, sampled, smem, C, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace binned
}  // namespace hs
