// k_binned.cu - update mode with shared-memory accumulation (Add of
// arXiv:1711.00975 Sec. 2.2 applied to every kept particle of the stream).
//
// The paper notes that the random counter updates become the bottleneck once
// hashing runs on the GPU (Sec. 3.1, "CPU + hashes on GPU").  On GB300 one
// random 32-bit add resolves in L2 at about 2e11/s (less once the sketch is
// larger than L2), well below the particle stream's HBM rate.  So the update
// is split in two passes over compact 16-bit codes:
//
//  1. scatter: read the particles once; for each kept particle and row, the
//     flat counter index i = r*W + bucket is split into bin = i >> S and a code
//     ((i mod 2^S) << 1 | sign bit).  Codes are write-combined per bin in
//     shared memory and flushed to the bin's global array in 32-byte units.
//  2. accumulate: one block per bin adds its codes into 2^S shared-memory
//     counters with shared atomics, then adds them to the bin's counter range.
//
// Integer addition commutes, so the counters equal those of the direct update
// bit for bit.  Whatever does not fit - a full shared-memory buffer or a full
// global bin - is added directly with a global atomic, so nothing is dropped.
#include <algorithm>
#include <cmath>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

struct ScatterArgs {
    uint64_t n;
    uint64_t g0;
    uint64_t thr;
    uint64_t sample_seed;
    uint64_t *probe;
    uint64_t probe_base;  // probe[g - probe_base] = key for probe_base <= g < probe_end
    uint64_t probe_end;
    uint32_t keep_all;
    uint32_t S;           // log2 of counters per bin
    uint32_t nbins;
    uint32_t slot;        // shared-memory entries per bin (power of two)
    uint32_t unit;        // flush granule (entries), slot / 2
    uint32_t cap;         // global entries per bin
    uint32_t hshift;      // 31 - log2W: top log2W+1 bits of v = bucket and sign bit
    uint32_t code_mask;   // 2^(S+1) - 1
    uint32_t bins_per_row;
    uint32_t log2_slot;
    uint16_t *bins;       // nbins x cap codes
    uint32_t *cursor;     // fill of each global bin (may exceed cap)
    RouteFilter route;        // routed cells go to exact dense blocks instead
    const uint32_t *rprefix;
    int32_t *rblocks;
    uint4 *carry;             // per-block copy of the rings between launches (or nullptr)
    uint32_t carry_in;        // start from the carried rings instead of empty ones
    uint32_t carry_out;       // leave the rings in the carry instead of flushing them
    uint32_t carry16;         // 16-byte words of one block's carry
    uint32_t rounds;          // tiles staged between two flush phases
    const VolumeDesc *vols;   // batch: one entry per volume (nullptr for one sketch)
    uint32_t nvol;
    uint32_t probe_per_vol;   // batch: probe window of each volume
};

// (inlined: a call in the staging path costs register moves around every call
// site, which measured 20 % more instructions than the rare adds it guards)
__device__ __forceinline__ void direct_add(uint32_t *C, const ScatterArgs &a, uint32_t bin,
                                        uint16_t code) {
    uint64_t idx = ((uint64_t)bin << a.S) | (uint64_t)(code >> 1);
    atomicAdd(&C[idx], (code & 1) ? 0xFFFFFFFFu : 1u);
}

// Bin and code of row r for cell (cx, cy, cz).  The top 32 bits of
// v = a0*cx + a1*cy + a2*cz + b (mod 2^64) are the high word of
// b + lo(a0)*cx + lo(a1)*cy + lo(a2)*cz plus hi(a0)*cx + hi(a1)*cy + hi(a2)*cz
// (mod 2^32): three wide multiply-adds and three narrow ones.  Its top
// log2W + 1 bits h are (bucket << 1 | sign bit); the flat counter index is
// r*W + bucket, so bin = r * (W / 2^S) + (h >> (S + 1)) and code = h mod 2^(S+1).
__device__ __forceinline__ void bin_code(const RowSeed &sd, uint32_t cx, uint32_t cy, uint32_t cz,
                                         uint32_t r, const ScatterArgs &a, uint32_t &bin,
                                         uint32_t &code) {
    uint32_t lo;
    uint32_t h = row_value_hi(sd, cx, cy, cz, lo) >> a.hshift;
    code = h & a.code_mask;
    bin = (h >> (a.S + 1)) + r * a.bins_per_row;
}

__device__ __forceinline__ void write_probe(uint64_t *probe, uint64_t g, bool valid, uint32_t cx,
                                         uint32_t cy, uint32_t cz, uint32_t G) {
    probe[g] = valid ? key_of(cx, cy, cz, G) : kInvalidKey;
}

// one exact count for a particle of a routed coarse cell: its block is the
// cell's rank among the routed cells, its counter the fine cell's offset
// (x fastest) inside the coarse cell
__device__ __forceinline__ void route_add(const ScatterArgs &a, uint32_t cx, uint32_t cy,
                                       uint32_t cz) {
    const RouteFilter &f = a.route;
    const uint32_t qx = __umulhi(cx, f.rmagic), qy = __umulhi(cy, f.rmagic),
                   qz = __umulhi(cz, f.rmagic);
    const uint64_t ck = (uint64_t)qx + (uint64_t)f.Gc * (qy + (uint64_t)f.Gc * qz);
    const uint32_t w = (uint32_t)(ck >> 5), b = (uint32_t)(ck & 31);
    const uint32_t blk = __ldg(a.rprefix + w) + __popc(__ldg(f.bits + w) & ((1u << b) - 1u));
    const uint32_t local = (cx - qx * f.R) + f.R * ((cy - qy * f.R) + f.R * (cz - qz * f.R));
    atomicAdd(&a.rblocks[(uint64_t)blk * (f.R * f.R * f.R) + local], 1);
}

// Scatter variants: one plain sketch, a batch of volumes, a learned sketch that
// routes some coarse cells to exact counters, a super-item sketch (Algorithm 3).
constexpr int kModePlain = 0, kModeBatch = 1, kModeRoute = 2, kModeSuper = 3;
// the same for packed 64-bit particle records instead of float32 xyz
constexpr int kModePlainPacked = 4, kModeSuperPacked = 5;

// Mesh reduction, sampling and probe entry of one particle; true when it is
// kept, with its cell packed as cx | cy << 21 | cz << 42 (G <= 2^21).
template <int MODE>
__device__ __forceinline__ bool prep_particle(float x, float y, float z, uint64_t g,
                                              const SketchDesc &d, const ScatterArgs &a,
                                              uint64_t &cell) {
    bool keep = a.keep_all || splitmix64_at(a.sample_seed, g) < a.thr;
    uint32_t cx = 0, cy = 0, cz = 0;
    bool valid = axis_cell(x, d.inv_cell, d.Gq, cx);
    valid &= axis_cell(y, d.inv_cell, d.Gq, cy);
    valid &= axis_cell(z, d.inv_cell, d.Gq, cz);
    if (MODE == kModeSuper) {              // the F^3 block holding the cell
        cx = __umulhi(cx, d.fmagic);
        cy = __umulhi(cy, d.fmagic);
        cz = __umulhi(cz, d.fmagic);
    }
    bool routed = false;
    if (MODE == kModeRoute && valid) routed = routed_cell(a.route, cx, cy, cz);
    if (g - a.probe_base < a.probe_end - a.probe_base)   // the sketch's cells only
        write_probe(a.probe, g - a.probe_base, valid && !routed, cx, cy, cz, d.G);
    cell = (uint64_t)cx | ((uint64_t)cy << 21) | ((uint64_t)cz << 42);
    if (MODE == kModeRoute && routed && keep) {
        route_add(a, cx, cy, cz);
        return false;
    }
    return keep && valid;
}

// prep_particle for a packed record
template <int MODE>
__device__ __forceinline__ bool prep_record(uint64_t p, uint64_t g, const SketchDesc &d,
                                            const ScatterArgs &a, uint64_t &cell) {
    bool keep = a.keep_all || splitmix64_at(a.sample_seed, g) < a.thr;
    uint32_t cx = packed_axis(p, 0, d.Gq), cy = packed_axis(p, 1, d.Gq), cz = packed_axis(p, 2, d.Gq);
    const bool valid = !(p & kPackInvalid);
    if (MODE == kModeSuperPacked) {
        cx = __umulhi(cx, d.fmagic);
        cy = __umulhi(cy, d.fmagic);
        cz = __umulhi(cz, d.fmagic);
    }
    if (g - a.probe_base < a.probe_end - a.probe_base)
        write_probe(a.probe, g - a.probe_base, valid, cx, cy, cz, d.G);
    cell = (uint64_t)cx | ((uint64_t)cy << 21) | ((uint64_t)cz << 42);
    return keep && valid;
}

// Shared-memory staging of bin b: a ring of `slot` (32) codes.  s_fill[b]
// packs the ring's rotation (high 16 bits) and the number of codes staged
// since its last flush (low 16 bits), so one shared atomic returns both.  Code
// number j sits at ring position (j + rot) mod slot; the initial rotations
// differ between bins, which spreads concurrent stores over the banks, and a
// flush of the first half advances the rotation instead of moving the rest.
// The lane that stages code number unit-1 (the first full half) marks the bin
// due in a bitmap (a fire-and-forget shared atomic on a random word).
__device__ __forceinline__ void stage_one(uint32_t bin, uint32_t code, const ScatterArgs &a,
                                          uint32_t w, uint16_t *s_buf, uint32_t *s_due,
                                          uint32_t *C) {
    const uint32_t slot = w & 0xFFFFu, rot = w >> 16;
    if (slot < a.slot) {
        s_buf[(bin << a.log2_slot) + ((slot + rot) & (a.slot - 1))] = (uint16_t)code;
        if (slot == a.unit - 1) atomicOr(&s_due[bin >> 5], 1u << (bin & 31));
    } else {
        direct_add(C, a, bin, (uint16_t)code);
    }
}

// Volume holding particle i of the concatenated buffer (binary search).
__device__ __forceinline__ uint32_t vol_of(const ScatterArgs &a, uint64_t i) {
    uint32_t lo = 0, hi = a.nvol;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (a.vols[mid].start <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Batch variant of prep_particle: particle i of the concatenated buffer
// belongs to volume v (vols[v].start <= i < vols[v+1].start, found from the
// hint v upward); it is sampled with its index inside that volume's stream and
// quantised on that volume's mesh.  The packed cell carries the volume's first
// bin: cx | cy << 16 | cz << 32 | bin0 << 48 (G < 2^16, bins < 2^16).
__device__ __forceinline__ bool prep_particle_batch(float x, float y, float z, uint64_t i,
                                                    const ScatterArgs &a, uint32_t &v,
                                                    uint64_t &cell) {
    while (v + 1 < a.nvol && i >= a.vols[v + 1].start) ++v;
    const VolumeDesc &V = a.vols[v];
    const uint64_t g = V.g0 + (i - V.start);
    bool keep = a.keep_all || splitmix64_at(a.sample_seed, g) < a.thr;
    uint32_t cx = 0, cy = 0, cz = 0;
    bool valid = axis_cell(x, V.inv_cell, V.G, cx);
    valid &= axis_cell(y, V.inv_cell, V.G, cy);
    valid &= axis_cell(z, V.inv_cell, V.G, cz);
    if (a.probe && g - V.probe_base < a.probe_per_vol)
        write_probe(a.probe + (uint64_t)v * a.probe_per_vol, g - V.probe_base, valid, cx, cy, cz,
                    V.G);
    cell = (uint64_t)cx | ((uint64_t)cy << 16) | ((uint64_t)cz << 32) | ((uint64_t)V.bin0 << 48);
    return keep && valid;
}

template <int T, bool BATCH>
__device__ __forceinline__ void stage_cell(uint64_t cell, const SketchDesc &d, const ScatterArgs &a,
                                           uint32_t *s_fill, uint16_t *s_buf, uint32_t *s_due,
                                           uint32_t *C) {
    uint32_t cx, cy, cz, bin0 = 0;
    if (BATCH) {
        cx = (uint32_t)(cell & 0xFFFF);
        cy = (uint32_t)((cell >> 16) & 0xFFFF);
        cz = (uint32_t)((cell >> 32) & 0xFFFF);
        bin0 = (uint32_t)(cell >> 48);
    } else {
        cx = (uint32_t)(cell & 0x1FFFFF);
        cy = (uint32_t)((cell >> 21) & 0x1FFFFF);
        cz = (uint32_t)(cell >> 42);
    }
    if (T > 0) {
        uint32_t bin[T > 0 ? T : 1], code[T > 0 ? T : 1], w[T > 0 ? T : 1];
#pragma unroll
        for (int r = 0; r < T; ++r) {
            bin_code(d.seed[r], cx, cy, cz, (uint32_t)r, a, bin[r], code[r]);
            bin[r] += bin0;
        }
#pragma unroll
        for (int r = 0; r < T; ++r) w[r] = atomicAdd(&s_fill[bin[r]], 1u);
#pragma unroll
        for (int r = 0; r < T; ++r) stage_one(bin[r], code[r], a, w[r], s_buf, s_due, C);
    } else {
        for (uint32_t r = 0; r < d.rows; ++r) {
            uint32_t bin, code;
            bin_code(d.seed[r], cx, cy, cz, r, a, bin, code);
            bin += bin0;
            stage_one(bin, code, a, atomicAdd(&s_fill[bin], 1u), s_buf, s_due, C);
        }
    }
}

// Copy `cnt` (a multiple of 8) codes of a bin's ring, starting at even ring
// position p0, to global memory at position g of the bin's array.
__device__ __forceinline__ void flush_ring(uint32_t *C, const ScatterArgs &a, uint32_t bin,
                                           const uint16_t *ring, uint32_t p0, uint32_t cnt,
                                           uint32_t g) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(ring);
    const uint32_t wmask = (a.slot >> 1) - 1;
    uint16_t *dst = a.bins + (uint64_t)bin * a.cap;
    const bool fits = g < a.cap && cnt <= a.cap - g;
    const bool aligned = (reinterpret_cast<uintptr_t>(dst + g) & 15u) == 0;
    if (fits && aligned) {
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + g);
        for (uint32_t j = 0; j < cnt / 8; ++j) {
            uint32_t q0 = (p0 >> 1) + 4 * j;
            d4[j] = make_uint4(w[q0 & wmask], w[(q0 + 1) & wmask], w[(q0 + 2) & wmask],
                               w[(q0 + 3) & wmask]);
        }
    } else {
        for (uint32_t j = 0; j < cnt; ++j) {
            uint16_t c = ring[(p0 + j) & (a.slot - 1)];
            if (g + j < a.cap) dst[g + j] = c;
            else direct_add(C, a, bin, c);
        }
    }
}

constexpr int kScatterThreads = 1024;  // largest block; the queue area is sized for it
constexpr int kQueuePerWarp = 128;     // 32 lanes x 4 particles

// Up to kMaxFlushPerThread due-bitmap words per warp in the flush phase
// (nbins <= kMaxFlushPerThread * 32 * warps per block).
constexpr int kMaxFlushPerThread = 6;

template <int T, bool VEC, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
    k_bin_scatter(const float *__restrict__ xyz, const SketchDesc d, const ScatterArgs a,
                  uint32_t *__restrict__ C) {
    constexpr bool BATCH = MODE == kModeBatch;
    constexpr bool PACKED = MODE == kModePlainPacked || MODE == kModeSuperPacked;
    // PACKED: xyz holds 64-bit records, two per 16-byte vector
    const uint64_t *rec = reinterpret_cast<const uint64_t *>(xyz);
    const uint4 *r4 = reinterpret_cast<const uint4 *>(xyz);
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *s_fill = reinterpret_cast<uint32_t *>(smem);
    const uint32_t fill_bytes = (a.nbins * 4 + 15) & ~15u;
    uint16_t *s_buf = reinterpret_cast<uint16_t *>(smem + fill_bytes);
    const uint32_t buf_bytes = (a.nbins * a.slot * 2 + 15) & ~15u;
    uint64_t *s_queue = reinterpret_cast<uint64_t *>(smem + fill_bytes + buf_bytes);
    uint32_t *s_due = reinterpret_cast<uint32_t *>(smem + fill_bytes + buf_bytes +
                                                   (kScatterThreads / 32) * kQueuePerWarp * 8);
    const uint32_t ndue = (a.nbins + 31) / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *q = s_queue + warp * kQueuePerWarp;
    if (a.carry_in) {   // the rings this block left at the end of the previous launch
        const uint4 *src = a.carry + (uint64_t)blockIdx.x * a.carry16;
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (uint32_t i = threadIdx.x; i < a.carry16; i += blockDim.x) dst[i] = src[i];
    } else {
        for (uint32_t b = threadIdx.x; b < a.nbins; b += blockDim.x)
            s_fill[b] = ((2u * (b >> 1)) & (a.slot - 1)) << 16;   // rotation, nothing staged
    }
    for (uint32_t i = threadIdx.x; i < ndue; i += blockDim.x) s_due[i] = 0;
    __syncthreads();

    // Tiles of 4 particles per thread (VEC: one 48-byte group as three float4,
    // the next tile's group loaded before this one is processed).  Kept cells
    // are compacted into a per-warp queue so the row updates run with every
    // lane busy whatever the sample rate.
    const uint64_t per_tile = (uint64_t)blockDim.x * 4;
    const uint64_t ntiles = (a.n + per_tile - 1) / per_tile;
    const uint64_t full_groups = a.n >> 2;
    const float4 *p4 = reinterpret_cast<const float4 *>(xyz);
    float4 nu = make_float4(0, 0, 0, 0), nv = nu, nw = nu;
    uint64_t tile = blockIdx.x;
    uint4 na = make_uint4(0, 0, 0, 0), nb = na;
    if (VEC && tile < ntiles) {
        uint64_t g4 = tile * blockDim.x + threadIdx.x;
        if (g4 < full_groups) {
            if (PACKED) {
                na = __ldcs(r4 + 2 * g4);
                nb = __ldcs(r4 + 2 * g4 + 1);
            } else {
                nu = __ldcs(p4 + 3 * g4);
                nv = __ldcs(p4 + 3 * g4 + 1);
                nw = __ldcs(p4 + 3 * g4 + 2);
            }
        }
    }
    const unsigned lt = (1u << lane) - 1u;
    for (; tile < ntiles;) {
      // a.rounds tiles between flushes: at sample rate r about 1/r tiles stage
      // as many codes as one tile at rate 1
      for (uint32_t rnd = 0; rnd < a.rounds && tile < ntiles; ++rnd, tile += gridDim.x) {
        uint64_t cell[4];
        bool ok[4];
        const uint64_t g4 = tile * blockDim.x + threadIdx.x;     // this thread's group
        if (PACKED) {
            if (VEC) {
                const uint4 ua = na, ub = nb;
                const uint64_t gn = (tile + gridDim.x) * blockDim.x + threadIdx.x;
                if (tile + gridDim.x < ntiles && gn < full_groups) {
                    na = __ldcs(r4 + 2 * gn);
                    nb = __ldcs(r4 + 2 * gn + 1);
                }
                if (g4 < full_groups) {
                    const uint64_t g = a.g0 + 4 * g4;
                    ok[0] = prep_record<MODE>(ua.x | ((uint64_t)ua.y << 32), g, d, a, cell[0]);
                    ok[1] = prep_record<MODE>(ua.z | ((uint64_t)ua.w << 32), g + 1, d, a, cell[1]);
                    ok[2] = prep_record<MODE>(ub.x | ((uint64_t)ub.y << 32), g + 2, d, a, cell[2]);
                    ok[3] = prep_record<MODE>(ub.z | ((uint64_t)ub.w << 32), g + 3, d, a, cell[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint64_t i = 4 * g4 + j;
                        ok[j] = i < a.n && prep_record<MODE>(__ldcs(reinterpret_cast<const unsigned long long *>(rec) + i),
                                                             a.g0 + i, d, a, cell[j]);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t i = 4 * g4 + j;
                    ok[j] = i < a.n && prep_record<MODE>(__ldcs(reinterpret_cast<const unsigned long long *>(rec) + i),
                                                         a.g0 + i, d, a, cell[j]);
                }
            }
        } else if (VEC) {
            float4 u = nu, v = nv, w = nw;
            const uint64_t gn = (tile + gridDim.x) * blockDim.x + threadIdx.x;
            if (tile + gridDim.x < ntiles && gn < full_groups) {
                nu = __ldcs(p4 + 3 * gn);
                nv = __ldcs(p4 + 3 * gn + 1);
                nw = __ldcs(p4 + 3 * gn + 2);
            }
            if (g4 < full_groups) {
                if (BATCH) {
                    uint32_t vh = vol_of(a, 4 * g4);
                    ok[0] = prep_particle_batch(u.x, u.y, u.z, 4 * g4, a, vh, cell[0]);
                    ok[1] = prep_particle_batch(u.w, v.x, v.y, 4 * g4 + 1, a, vh, cell[1]);
                    ok[2] = prep_particle_batch(v.z, v.w, w.x, 4 * g4 + 2, a, vh, cell[2]);
                    ok[3] = prep_particle_batch(w.y, w.z, w.w, 4 * g4 + 3, a, vh, cell[3]);
                } else {
                    uint64_t g = a.g0 + 4 * g4;
                    ok[0] = prep_particle<MODE>(u.x, u.y, u.z, g, d, a, cell[0]);
                    ok[1] = prep_particle<MODE>(u.w, v.x, v.y, g + 1, d, a, cell[1]);
                    ok[2] = prep_particle<MODE>(v.z, v.w, w.x, g + 2, d, a, cell[2]);
                    ok[3] = prep_particle<MODE>(w.y, w.z, w.w, g + 3, d, a, cell[3]);
                }
            } else {
                uint32_t vh = BATCH ? vol_of(a, 4 * g4 < a.n ? 4 * g4 : a.n - 1) : 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint64_t i = 4 * g4 + j;
                    if (BATCH)
                        ok[j] = i < a.n &&
                                prep_particle_batch(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                                    __ldcs(xyz + 3 * i + 2), i, a, vh, cell[j]);
                    else
                        ok[j] = i < a.n &&
                                prep_particle<MODE>(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                              __ldcs(xyz + 3 * i + 2), a.g0 + i, d, a, cell[j]);
                }
            }
        } else {
            uint32_t vh = BATCH ? vol_of(a, 4 * g4 < a.n ? 4 * g4 : a.n - 1) : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint64_t i = 4 * g4 + j;
                if (BATCH)
                    ok[j] = i < a.n &&
                            prep_particle_batch(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                                __ldcs(xyz + 3 * i + 2), i, a, vh, cell[j]);
                else
                    ok[j] = i < a.n && prep_particle<MODE>(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                                     __ldcs(xyz + 3 * i + 2), a.g0 + i, d, a,
                                                     cell[j]);
            }
        }
        if (__all_sync(0xFFFFFFFFu, ok[0] & ok[1] & ok[2] & ok[3])) {
            // every particle of the warp is kept: stage straight from registers
#pragma unroll
            for (int j = 0; j < 4; ++j) stage_cell<T, BATCH>(cell[j], d, a, s_fill, s_buf, s_due, C);
        } else {
            uint32_t nq = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                unsigned m = __ballot_sync(0xFFFFFFFFu, ok[j]);
                if (ok[j]) q[nq + __popc(m & lt)] = cell[j];
                nq += __popc(m);
            }
            __syncwarp();
            for (uint32_t i = lane; i < nq; i += 32)
                stage_cell<T, BATCH>(q[i], d, a, s_fill, s_buf, s_due, C);
            __syncwarp();
        }
      }
        __syncthreads();
        // flush the due bins: warp w reads due words w, w + nwarps, ... (one
        // broadcast load each) and lane l flushes the bin of bit l.  All global
        // reservations of a lane are issued before its copies.
        const uint32_t nwarps = blockDim.x >> 5;
        uint32_t wd[kMaxFlushPerThread], gp[kMaxFlushPerThread], nf[kMaxFlushPerThread];
#pragma unroll
        for (int k = 0; k < kMaxFlushPerThread; ++k) {
            const uint32_t wi = warp + k * nwarps;
            nf[k] = 0;
            if (wi >= ndue) break;
            const uint32_t bits = s_due[wi];
            if ((bits >> lane) & 1u) {
                const uint32_t b = wi * 32 + lane;
                wd[k] = s_fill[b];
                const uint32_t f = min(wd[k] & 0xFFFFu, a.slot);
                nf[k] = f >= a.slot ? a.slot : a.unit;   // due: f >= unit
                gp[k] = atomicAdd(&a.cursor[b], nf[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxFlushPerThread; ++k) {
            const uint32_t wi = warp + k * nwarps;
            if (wi >= ndue) break;
            if (nf[k]) {
                const uint32_t b = wi * 32 + lane, rot = wd[k] >> 16;
                const uint32_t f = min(wd[k] & 0xFFFFu, a.slot);
                flush_ring(C, a, b, s_buf + (b << a.log2_slot), rot, nf[k], gp[k]);
                s_fill[b] = (((rot + nf[k]) & (a.slot - 1)) << 16) | (f - nf[k]);
            }
            if (lane == 0) s_due[wi] = 0;
        }
        __syncthreads();
    }
    if (a.carry_out) {   // every ring holds fewer than `unit` codes: keep them for the next launch
        __syncthreads();
        uint4 *dst = a.carry + (uint64_t)blockIdx.x * a.carry16;
        const uint4 *src = reinterpret_cast<const uint4 *>(smem);
        for (uint32_t i = threadIdx.x; i < a.carry16; i += blockDim.x) dst[i] = src[i];
        return;
    }
    // what is left in shared memory
    for (uint32_t b = threadIdx.x; b < a.nbins; b += blockDim.x) {
        uint32_t w = s_fill[b];
        uint32_t f = min(w & 0xFFFFu, a.slot);
        if (f) {
            const uint16_t *ring = s_buf + (b << a.log2_slot);
            uint32_t g = atomicAdd(&a.cursor[b], f);
            uint16_t *dst = a.bins + (uint64_t)b * a.cap;
            for (uint32_t j = 0; j < f; ++j) {
                uint16_t c = ring[((w >> 16) + j) & (a.slot - 1)];
                if (g + j < a.cap) dst[g + j] = c;
                else direct_add(C, a, b, c);
            }
        }
    }
}

// The rings carried out of the last scatter launch of every block, moved to
// the global bins: one thread per (block, bin).
__global__ void k_carry_flush(const uint4 *__restrict__ carry, uint32_t nblocks, ScatterArgs a,
                              uint32_t *__restrict__ C) {
    const uint64_t total = (uint64_t)nblocks * a.nbins;
    const uint32_t fill_bytes = (a.nbins * 4 + 15) & ~15u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint32_t blk = (uint32_t)(t / a.nbins), b = (uint32_t)(t % a.nbins);
        const unsigned char *base =
            reinterpret_cast<const unsigned char *>(carry + (uint64_t)blk * a.carry16);
        const uint32_t w = reinterpret_cast<const uint32_t *>(base)[b];
        const uint32_t f = min(w & 0xFFFFu, a.slot);
        if (!f) continue;
        const uint16_t *ring = reinterpret_cast<const uint16_t *>(base + fill_bytes) + (b << a.log2_slot);
        const uint32_t g = atomicAdd(&a.cursor[b], f);
        uint16_t *dst = a.bins + (uint64_t)b * a.cap;
        for (uint32_t j = 0; j < f; ++j) {
            const uint16_t c = ring[((w >> 16) + j) & (a.slot - 1)];
            if (g + j < a.cap) dst[g + j] = c;
            else direct_add(C, a, b, c);
        }
    }
}

// one block per bin: shared-memory accumulation, then C[bin range] += acc
__global__ void __launch_bounds__(1024)
    k_bin_accumulate(const uint16_t *__restrict__ bins, uint32_t *__restrict__ cursor, uint32_t cap,
                     uint32_t S, uint32_t *__restrict__ C) {
    extern __shared__ __align__(16) int32_t acc[];
    const uint32_t nacc = 1u << S;
    const uint32_t bin = blockIdx.x;
    for (uint32_t i = threadIdx.x; i < nacc; i += blockDim.x) acc[i] = 0;
    __syncthreads();
    const uint32_t len = min(cursor[bin], cap);
    const uint16_t *src = bins + (uint64_t)bin * cap;
    const uint32_t n8 = len / 8;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);   // cap is a multiple of 8
    // eight 16-byte loads in flight per thread before the shared-memory adds
    for (uint32_t j0 = 0; j0 < n8; j0 += 8 * blockDim.x) {
        uint4 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint32_t j = j0 + u * blockDim.x + threadIdx.x;
            w[u] = j < n8 ? __ldcs(s4 + j) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu,
                                                        0xFFFFFFFFu);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (j0 + u * blockDim.x + threadIdx.x >= n8) continue;
            uint32_t ws[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t c0 = ws[q] & 0xFFFFu, c1 = ws[q] >> 16;
                atomicAdd(&acc[c0 >> 1], (c0 & 1) ? -1 : 1);
                atomicAdd(&acc[c1 >> 1], (c1 & 1) ? -1 : 1);
            }
        }
    }
    for (uint32_t j = n8 * 8 + threadIdx.x; j < len; j += blockDim.x) {
        uint32_t c = src[j];
        atomicAdd(&acc[c >> 1], (c & 1) ? -1 : 1);
    }
    __syncthreads();
    uint32_t *dst = C + ((uint64_t)bin << S);
    for (uint32_t i = threadIdx.x; i < nacc; i += blockDim.x) {
        int32_t v = acc[i];
        if (v) dst[i] += (uint32_t)v;
    }
    if (threadIdx.x == 0) cursor[bin] = 0;
}

}  // namespace

uint32_t carry_words16(const BinLayout &L) {
    return (uint32_t)((((size_t)L.nbins * 4 + 15) & ~(size_t)15) +
                      (((size_t)L.nbins * L.slot * 2 + 15) & ~(size_t)15)) / 16;
}

BinLayout bin_layout(const SketchDesc &d, size_t smem_budget) {
    BinLayout L{};
    L.S = d.log2w < 15 ? d.log2w : 15;
    uint64_t nb = (uint64_t)d.rows << (d.log2w - L.S);
    L.nbins = (uint32_t)nb;
    L.slot = 0;
    const size_t queue = (size_t)(kScatterThreads / 32) * kQueuePerWarp * 8;
    for (uint32_t slot = 32; slot >= 16; slot >>= 1) {
        size_t need = ((nb * 4 + 15) & ~15ull) + ((nb * slot * 2 + 15) & ~15ull) + queue +
                      ((nb + 31) / 32) * 4;
        // flush phase: each warp covers at most kMaxFlushPerThread due words
        if (nb <= (uint64_t)kMaxFlushPerThread * kScatterThreads && need <= smem_budget) {
            L.slot = slot;
            L.smem = need;
            break;
        }
    }
    return L;
}

cudaError_t launch_bin_scatter(const float *xyz, uint64_t n, uint64_t g0, const SketchDesc &d,
                               int32_t *C, double rate, uint64_t sample_seed, uint64_t *probe,
                               uint64_t probe_base, uint64_t probe_cap, const BinLayout &L, uint16_t *bins,
                               uint32_t *cursor, uint32_t cap, int blocks, cudaStream_t s,
                               const VolumeDesc *vols, uint32_t nvol, uint32_t probe_per_vol,
                               int threads, const RouteTarget *route, uint4 *carry, int carry_in,
                               int carry_out, int packed) {
    if (n == 0) return cudaSuccess;
    // bin arrays are read and written as 16-byte vectors: every bin must start
    // on a 16-byte boundary
    if ((cap & 7u) != 0 || (reinterpret_cast<uintptr_t>(bins) & 15u) != 0 || L.slot == 0)
        return cudaErrorInvalidValue;
    ScatterArgs a;
    a.n = n;
    a.g0 = g0;
    a.keep_all = rate >= 1.0 ? 1u : 0u;
    a.thr = rate >= 1.0 ? 0 : (uint64_t)ldexp(rate, 64);
    a.sample_seed = sample_seed;
    a.probe = probe;
    a.probe_base = probe_base;
    a.probe_end = probe ? probe_base + probe_cap : probe_base;
    a.S = L.S;
    a.nbins = L.nbins;
    a.slot = L.slot;
    a.unit = L.slot / 2;
    a.cap = cap;
    a.hshift = 31 - d.log2w;
    a.code_mask = (2u << L.S) - 1u;
    a.bins_per_row = 1u << (d.log2w - L.S);
    a.log2_slot = 0;
    while ((1u << a.log2_slot) < L.slot) ++a.log2_slot;
    a.bins = bins;
    a.cursor = cursor;
    a.route = route ? route->filter : RouteFilter{nullptr, 0, 0, 0};
    a.rprefix = route ? route->prefix : nullptr;
    a.rblocks = route ? route->blocks : nullptr;
    a.carry = carry;
    a.carry_in = carry && carry_in ? 1u : 0u;
    a.carry_out = carry && carry_out ? 1u : 0u;
    a.carry16 = carry_words16(L);
    // at sample rate r a tile stages about r times the codes of a full tile
    a.rounds = rate >= 1.0 ? 1u : (uint32_t)std::min(16.0, std::max(1.0, std::floor(1.0 / rate)));
    a.vols = vols;
    a.nvol = vols ? nvol : 0;
    a.probe_per_vol = probe_per_vol;
    uint32_t *Cu = reinterpret_cast<uint32_t *>(C);
    // the flush phase covers kMaxFlushPerThread due words per warp
    // only batches are tuned over the block size
    if (threads != 512 || !vols || L.nbins > (uint32_t)kMaxFlushPerThread * 512)
        threads = kScatterThreads;
    if (packed && (vols || route)) return cudaErrorInvalidValue;   // float input only there
    bool vec = (reinterpret_cast<uintptr_t>(xyz) & 15u) == 0;
    uint64_t per_tile = (uint64_t)threads * 4;
    uint64_t need_blocks = (n + per_tile - 1) / per_tile;
    // a carry belongs to a block index: carrying launches always use every block
    if (!a.carry_in && !a.carry_out && need_blocks < (uint64_t)blocks) blocks = (int)need_blocks;
    if (blocks < 1) blocks = 1;
    auto launch = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        kern<<<blocks, threads, L.smem, s>>>(xyz, d, a, Cu);
    };
#define HS_SCATTER_ROWS(MODE, TH)                                                          \
    if (d.rows == 5) {                                                                     \
        if (vec) launch(k_bin_scatter<5, true, MODE, TH>);                                 \
        else launch(k_bin_scatter<5, false, MODE, TH>);                                    \
    } else {                                                                               \
        if (vec) launch(k_bin_scatter<0, true, MODE, TH>);                                 \
        else launch(k_bin_scatter<0, false, MODE, TH>);                                    \
    }
    if (vols) {
        if (threads == 512) {
            HS_SCATTER_ROWS(kModeBatch, 512)
        } else {
            HS_SCATTER_ROWS(kModeBatch, 1024)
        }
    } else if (route) {
        HS_SCATTER_ROWS(kModeRoute, 1024)
    } else if (packed) {
        if (d.F > 1) {
            HS_SCATTER_ROWS(kModeSuperPacked, 1024)
        } else {
            HS_SCATTER_ROWS(kModePlainPacked, 1024)
        }
    } else if (d.F > 1) {
        HS_SCATTER_ROWS(kModeSuper, 1024)
    } else {
        HS_SCATTER_ROWS(kModePlain, 1024)
    }
#undef HS_SCATTER_ROWS
    return cudaGetLastError();
}

cudaError_t launch_carry_flush(const BinLayout &L, const uint4 *carry, uint32_t nblocks,
                               uint16_t *bins, uint32_t *cursor, uint32_t cap, int32_t *C,
                               cudaStream_t s) {
    ScatterArgs a{};
    a.S = L.S;
    a.nbins = L.nbins;
    a.slot = L.slot;
    a.cap = cap;
    a.log2_slot = 0;
    while ((1u << a.log2_slot) < L.slot) ++a.log2_slot;
    a.bins = bins;
    a.cursor = cursor;
    a.carry16 = carry_words16(L);
    const uint64_t total = (uint64_t)nblocks * L.nbins;
    uint64_t blocks = std::min<uint64_t>((total + 255) / 256, 8192);
    k_carry_flush<<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, s>>>(
        carry, nblocks, a, reinterpret_cast<uint32_t *>(C));
    return cudaGetLastError();
}

cudaError_t launch_bin_accumulate(const BinLayout &L, uint16_t *bins, uint32_t *cursor,
                                  uint32_t cap, int32_t *C, cudaStream_t s) {
    if ((cap & 7u) != 0 || (reinterpret_cast<uintptr_t>(bins) & 15u) != 0)
        return cudaErrorInvalidValue;
    size_t smem = (size_t)4 << L.S;
    cudaFuncSetAttribute(k_bin_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bin_accumulate<<<L.nbins, 1024, smem, s>>>(bins, cursor, cap, L.S,
                                                reinterpret_cast<uint32_t *>(C));
    return cudaGetLastError();
}

}  // namespace hs
