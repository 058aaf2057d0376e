// k_binned.cuh - the scatter of the binned update (Add of arXiv:1711.00975
// Sec. 2.2 applied to every kept particle of the stream), shared by the
// translation units that instantiate its variants.
//
// The paper notes that the random counter updates become the bottleneck once
// hashing runs on the GPU (Sec. 3.1, "CPU + hashes on GPU").  On GB300 one
// random 32-bit add resolves in L2 at about 2e11/s (less once the sketch is
// larger than L2), well below the particle stream's HBM rate.  So the update
// is split in two passes over compact 16-bit codes:
//
//  1. scatter (here): read the particles once; for each kept particle and row,
//     the flat counter index i = r*W + bucket is split into bin = i >> S and a
//     code ((i mod 2^S) << 1 | sign bit).  Codes are write-combined per bin in
//     a shared-memory ring of two halves; between two block barriers every
//     full half is copied to the block's own region of that bin in global
//     memory (no global atomics).  The last, partial half of a launch is padded
//     with pairs of codes that cancel (+1 and -1 on the bin's counter 0).
//  2. accumulate (k_binned.cu): one block per bin adds the codes of every
//     block's region into 2^S shared-memory counters, then adds them to the
//     bin's counters.
//
// Integer addition commutes, so the counters equal those of the direct update
// bit for bit.  Whatever does not fit - a full ring or a full region - is added
// directly with a global atomic, so nothing is dropped.
#pragma once

#include <cstring>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {
namespace binned {

constexpr uint32_t kPadPair = 0x00010000u;   // codes 0 (+1) and 1 (-1) of counter 0: they cancel
// 24 warps: the registers of 85 per thread keep the row seeds and staging
// state out of spills and recomputation (1024 threads, at 64 registers,
// executed 40 % more instructions and measured slower); 3072 particles a tile
constexpr int kScatterThreads = 768;
constexpr int kPPT = 4;                   // particles per thread and tile (three float4)
static_assert(kScatterThreads * kPPT == kScatterTile, "tile size known to the host");
constexpr int kQueue = 64;                // per-warp queue of kept cells (sampled calls)
constexpr uint32_t kSmemLimit = 227 * 1024;   // dynamic shared memory of one block (opt-in)

// Scatter variants: one plain sketch, a batch of volumes, a learned sketch that
// routes some coarse cells to exact counters, a super-item sketch (Algorithm 3).
constexpr int kModePlain = 0, kModeBatch = 1, kModeRoute = 2, kModeSuper = 3;
// the same for packed 64-bit particle records instead of float32 xyz
constexpr int kModePlainPacked = 4, kModeSuperPacked = 5;
// the same for cell records (kept particles' mesh cells, written by the
// compaction pass: cx | cy << 21 | cz << 42, already sampled)
constexpr int kModeCells = 6, kModeSuperCells = 7;

struct ScatterArgs {
    uint64_t n;
    // cell records: the buffer holds *n_dev records (device counter, read at
    // launch) and this launch takes its elements [n_base, n_base + n)
    const unsigned long long *n_dev;
    uint64_t n_base;
    uint64_t g0;
    uint64_t thr;
    uint64_t sample_seed;
    uint64_t *probe;
    uint64_t probe_base;  // probe[g - probe_base] = key for probe_base <= g < probe_end
    uint64_t probe_end;
    uint32_t S;           // log2 of counters per bin
    uint32_t nbins;       // bins staged by this launch (rows row0 .. row0 + nrows - 1)
    uint32_t bin_base;    // global number of this launch's bin 0
    uint32_t row0, nrows; // the rows this launch stages
    uint32_t route_adds;  // routed particles are counted by this launch (the first pass)
    uint32_t slot;        // ring entries per bin (two halves)
    uint32_t half;        // flush granule
    uint32_t hshift;      // 31 - log2W: top log2W+1 bits of v = bucket and sign bit
    uint32_t code_mask;   // 2^(S+1) - 1
    uint32_t rounds;      // tiles between flush phases
    uint32_t team;        // lanes that flush one bin (1 or 32)
    uint32_t gmagic;      // ceil(2^32 / bpg): bin / bpg = umulhi(bin, gmagic)
    uint32_t rbase[kMaxRows];   // first (local) bin of row row0 + i
    BinStore B;
    RouteFilter route;        // routed cells go to exact dense blocks instead
    const uint32_t *rprefix;
    int32_t *rblocks;
    const VolumeDesc *vols;   // batch: one entry per volume (nullptr for one sketch)
    uint32_t nvol;
    uint32_t probe_per_vol;   // batch: probe window of each volume
    // batch window: rings for the bins of `wvols` consecutive volumes only (a
    // power of two; 0: every bin has a ring); volume v's bins use ring slots
    // (v mod wvols) * bpv ... + bpv - 1 while v is in the window
    uint32_t wvols;
    uint32_t bpv;             // bins per volume
    const uint32_t *tvols;    // per tile: first volume | last volume << 16
};

// Byte offsets of the scatter's shared memory (host and device agree).
struct SmemLayout {
    uint32_t fill, cur, gbase, gcap, gbin, ring, queue, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline SmemLayout smem_layout(uint32_t nbins, uint32_t slot, uint32_t ngroups,
                                                  uint32_t queue, bool window = false) {
    SmemLayout L;
    uint32_t off = 0;
    L.fill = off;  off = align16(off + 4 * nbins);
    L.cur = off;   off = align16(off + 4 * nbins);
    L.gbase = off; off = align16(off + 8 * ngroups);
    L.gcap = off;  off = align16(off + 4 * ngroups);
    L.gbin = off;  off = align16(off + (window ? 4 * nbins + 4 : 0u));   // + the next window
    L.ring = off;  off = align16(off + 2 * nbins * slot);
    L.queue = off; off = align16(off + (queue ? 8u * kQueue * (kScatterThreads / 32) : 0u));
    L.total = off;
    return L;
}

// Largest ring (a power of two in [16, 16384] entries per bin) whose layout fits.
inline uint32_t ring_slot(uint32_t nbins, uint32_t ngroups, uint32_t queue, size_t budget,
                          bool window = false) {
    for (uint32_t slot = 16384; slot >= 16; slot >>= 1)
        if (smem_layout(nbins, slot, ngroups, queue, window).total <= budget) return slot;
    return 0;
}

constexpr uint32_t kNoBin = 0xFFFFFFFFu;   // a window's ring slot with no volume behind it

struct Smem {
    uint32_t *fill;    // per bin: (entries not yet flushed << 16) | byte offset of the next entry
    uint32_t *cur;     // per bin: codes this block has written to its region
    uint64_t *gbase;   // per group: region base (codes)
    uint32_t *gcap;    // per group: region capacity (codes)
    uint32_t *gbin;    // batch window: per ring slot, its global bin (or kNoBin); then the next window
    uint16_t *ring;    // per bin: `slot` entries
    uint64_t *queue;   // per warp: kQueue packed cells
};

// global bin of ring slot b (WIN: a batch, whose rings follow a window)
template <bool WIN>
__device__ __forceinline__ uint32_t gbin_of(const ScatterArgs &a, const Smem &s, uint32_t b) {
    return WIN ? s.gbin[b] : b + a.bin_base;
}

// global bin of ring slot b while the window starts at volume w0: slot group
// k = b / bpv holds the window's volume congruent to k modulo wvols
__device__ __forceinline__ uint32_t window_gbin(const ScatterArgs &a, uint32_t w0, uint32_t b) {
    const uint32_t k = b / a.bpv;
    const uint32_t v = w0 + ((k - w0) & (a.wvols - 1));
    return v < a.nvol ? v * a.bpv + (b - k * a.bpv) : kNoBin;
}

// (inlined: a call in the staging path costs register moves around every call
// site, more instructions than the rare adds it guards)
__device__ __forceinline__ void direct_add(uint32_t *C, uint32_t S, uint32_t bin, uint32_t code) {
    const uint64_t idx = ((uint64_t)bin << S) | (uint64_t)(code >> 1);
    atomicAdd(&C[idx], (code & 1u) ? 0xFFFFFFFFu : 1u);
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

// The top 32 bits of v = a0*cx + a1*cy + a2*cz + b (mod 2^64), written as
// plain 64-bit arithmetic (the compiler's own wide multiply-adds measured
// fewer instructions than a hand-written chain).
__device__ __forceinline__ uint32_t row_hi(const RowSeed &sd, uint32_t cx, uint32_t cy, uint32_t cz) {
    return (uint32_t)((sd.a0 * cx + sd.a1 * cy + sd.a2 * cz + sd.b) >> 32);
}

// A particle's cell on the sketch's mesh, ready to hash: coordinates and the
// first bin of its sketch (0 except in a batch).
struct Cell {
    uint32_t cx, cy, cz, bin0;
};

__device__ __forceinline__ uint64_t pack_cell(const Cell &c) {
    return (uint64_t)c.cx | ((uint64_t)c.cy << 21) | ((uint64_t)c.cz << 42);
}
__device__ __forceinline__ Cell unpack_cell(uint64_t v) {
    return Cell{(uint32_t)(v & 0x1FFFFF), (uint32_t)((v >> 21) & 0x1FFFFF), (uint32_t)(v >> 42), 0};
}
// batch cells: G < 2^16 and bins < 2^16
__device__ __forceinline__ uint64_t pack_cell_batch(const Cell &c) {
    return (uint64_t)c.cx | ((uint64_t)c.cy << 16) | ((uint64_t)c.cz << 32) | ((uint64_t)c.bin0 << 48);
}
__device__ __forceinline__ Cell unpack_cell_batch(uint64_t v) {
    return Cell{(uint32_t)(v & 0xFFFF), (uint32_t)((v >> 16) & 0xFFFF), (uint32_t)((v >> 32) & 0xFFFF),
                (uint32_t)(v >> 48)};
}

// Mesh reduction of one position.  A scaled coordinate in [0, G) needs no
// wrap: floor of it is the cell (the same float32 product and floor as
// axis_cell); anything else (outside the box, not finite) takes axis_cell's
// full path.
__device__ __forceinline__ bool mesh_cell(float x, float y, float z, float inv, uint32_t G, float Gf,
                                          Cell &c) {
    const float px = __fmul_rn(x, inv), py = __fmul_rn(y, inv), pz = __fmul_rn(z, inv);
    if (px >= 0.0f && px < Gf && py >= 0.0f && py < Gf && pz >= 0.0f && pz < Gf) {
        c.cx = __float2uint_rd(px);
        c.cy = __float2uint_rd(py);
        c.cz = __float2uint_rd(pz);
        return true;
    }
    bool valid = axis_cell(x, inv, G, c.cx);
    valid &= axis_cell(y, inv, G, c.cy);
    valid &= axis_cell(z, inv, G, c.cz);
    return valid;
}

// Mesh reduction, sampling, probe entry and routing of one particle; true when
// its cell goes to the sketch.
template <int MODE, bool SAMPLED, bool PROBE>
__device__ __forceinline__ bool prep_particle(float x, float y, float z, uint64_t g, float Gf,
                                              const SketchDesc &d, const ScatterArgs &a, Cell &c) {
    const bool keep = !SAMPLED || splitmix64_at(a.sample_seed, g) < a.thr;
    c.bin0 = 0;
    const bool valid = mesh_cell(x, y, z, d.inv_cell, d.Gq, Gf, c);
    if (MODE == kModeSuper) {              // the F^3 block holding the cell
        c.cx = __umulhi(c.cx, d.fmagic);
        c.cy = __umulhi(c.cy, d.fmagic);
        c.cz = __umulhi(c.cz, d.fmagic);
    }
    bool routed = false;
    if (MODE == kModeRoute && valid) routed = routed_cell(a.route, c.cx, c.cy, c.cz);
    if (PROBE && g - a.probe_base < a.probe_end - a.probe_base)   // the sketch's cells only
        write_probe(a.probe, g - a.probe_base, valid && !routed, c.cx, c.cy, c.cz, d.G);
    if (MODE == kModeRoute && routed && keep) {
        if (a.route_adds) route_add(a, c.cx, c.cy, c.cz);
        return false;
    }
    return keep && valid;
}

// prep_particle for a packed record
template <int MODE, bool SAMPLED, bool PROBE>
__device__ __forceinline__ bool prep_record(uint64_t p, uint64_t g, const SketchDesc &d,
                                            const ScatterArgs &a, Cell &c) {
    constexpr bool CELLS = MODE == kModeCells || MODE == kModeSuperCells;
    const bool keep = !SAMPLED || splitmix64_at(a.sample_seed, g) < a.thr;
    c.cx = CELLS ? (uint32_t)(p & kPackMask) : packed_axis(p, 0, d.Gq);
    c.cy = CELLS ? (uint32_t)((p >> kPackBits) & kPackMask) : packed_axis(p, 1, d.Gq);
    c.cz = CELLS ? (uint32_t)((p >> (2 * kPackBits)) & kPackMask) : packed_axis(p, 2, d.Gq);
    c.bin0 = 0;
    const bool valid = !(p & kPackInvalid);
    if (MODE == kModeSuperPacked || MODE == kModeSuperCells) {
        c.cx = __umulhi(c.cx, d.fmagic);
        c.cy = __umulhi(c.cy, d.fmagic);
        c.cz = __umulhi(c.cz, d.fmagic);
    }
    if (PROBE && g - a.probe_base < a.probe_end - a.probe_base)
        write_probe(a.probe, g - a.probe_base, valid, c.cx, c.cy, c.cz, d.G);
    return keep && valid;
}

// Batch variant of prep_particle: particle i of the concatenated buffer
// belongs to volume v (vols[v].start <= i < vols[v+1].start, found from the
// hint v upward); it is sampled with its index inside that volume's stream and
// quantised on that volume's mesh.
// The cell's bins are ring slots of its volume's slot group in the window of
// volumes that have rings; a volume outside the window [w0, w0 + wvols) (a tile spanning
// more volumes than the window holds) adds its rows directly.
template <bool SAMPLED>
__device__ __forceinline__ bool prep_particle_batch(float x, float y, float z, uint64_t i,
                                                    const SketchDesc &d, const ScatterArgs &a,
                                                    uint32_t w0, uint32_t &v, Cell &c, uint32_t *C) {
    while (v + 1 < a.nvol && i >= a.vols[v + 1].start) ++v;
    const VolumeDesc &V = a.vols[v];
    const uint64_t g = V.g0 + (i - V.start);
    const bool keep = !SAMPLED || splitmix64_at(a.sample_seed, g) < a.thr;
    const bool valid = mesh_cell(x, y, z, V.inv_cell, V.G, (float)V.G, c);
    c.bin0 = V.bin0;
    if (a.probe && g - V.probe_base < a.probe_per_vol)
        write_probe(a.probe + (uint64_t)v * a.probe_per_vol, g - V.probe_base, valid, c.cx, c.cy,
                    c.cz, V.G);
    if (v - w0 >= a.wvols) {
        if (keep && valid)
            for (uint32_t r = 0; r < d.rows; ++r) {
                const uint32_t h = row_hi(d.seed[r], c.cx, c.cy, c.cz) >> a.hshift;
                direct_add(C, a.S, (h >> (a.S + 1)) + a.rbase[r] + V.bin0, h & a.code_mask);
            }
        return false;
    }
    c.bin0 = (v & (a.wvols - 1)) * a.bpv;
    return keep && valid;
}

// prep_particle_batch for a tile that lies in one volume of the window: the
// volume's fields are loaded once a tile (vg = g0 - start, probe_v = its
// probe window, pbase = its probe_base, bin0 = its slot group's first ring).
template <bool SAMPLED>
__device__ __forceinline__ bool prep_particle_vol(float x, float y, float z, uint64_t i, uint64_t vg,
                                                  float inv, uint32_t G, uint32_t bin0,
                                                  uint64_t *probe_v, uint64_t pbase,
                                                  const ScatterArgs &a, Cell &c) {
    const uint64_t g = vg + i;
    const bool keep = !SAMPLED || splitmix64_at(a.sample_seed, g) < a.thr;
    const bool valid = mesh_cell(x, y, z, inv, G, (float)G, c);
    c.bin0 = bin0;
    if (probe_v && g - pbase < a.probe_per_vol) write_probe(probe_v, g - pbase, valid, c.cx, c.cy, c.cz, G);
    return keep && valid;
}

// A full ring gives the reservation back (no flush runs while codes are
// staged, so the position is reused) and adds the code directly.
template <bool WIN>
__device__ __forceinline__ void stage_full(uint32_t bin, uint32_t code, const ScatterArgs &a,
                                           const Smem &s, uint32_t *C) {
    atomicAdd(&s.fill[bin], 0xFFFEFFFEu);   // minus (1 << 16 | 2)
    direct_add(C, a.S, gbin_of<WIN>(a, s, bin), code);
}

// Bins and codes of every row of one cell, staged in the bins' rings.  The
// top log2W + 1 bits h of the row's multiply-shift value are
// (bucket << 1 | sign bit); the flat counter index
// is r*W + bucket, so bin = rbase[r] + (h >> (S + 1)) and code = h mod 2^(S+1).
// A reservation (fill += 1 << 16 | 2) returns the entries waiting for a flush
// (w >> 16) and the code's byte offset in the ring (w mod 2 slot); the byte
// offset is kept below 2^16 by the flush phases.
template <int T, bool WIN>
__device__ __forceinline__ void stage_cell(const Cell &c, const SketchDesc &d, const ScatterArgs &a,
                                           const Smem &s, uint32_t *C) {
    unsigned char *ring = reinterpret_cast<unsigned char *>(s.ring);
    const uint32_t rbytes = 2 * a.slot;
    if (T > 0) {
        constexpr int TT = T > 0 ? T : 1;
        uint32_t bin[TT], code[TT], w[TT];
#pragma unroll
        for (int r = 0; r < T; ++r) {
            const uint32_t h = row_hi(d.seed[r], c.cx, c.cy, c.cz) >> a.hshift;
            code[r] = h & a.code_mask;
            bin[r] = (h >> (a.S + 1)) + a.rbase[r] + (WIN ? c.bin0 : 0u);   // bin0 = 0 outside a batch
        }
#pragma unroll
        for (int r = 0; r < T; ++r) w[r] = atomicAdd(&s.fill[bin[r]], 0x10002u);
#pragma unroll
        for (int r = 0; r < T; ++r) {
            if ((w[r] >> 16) < a.slot)
                *reinterpret_cast<uint16_t *>(ring + bin[r] * rbytes + (w[r] & (rbytes - 1))) = (uint16_t)code[r];
            else
                stage_full<WIN>(bin[r], code[r], a, s, C);
        }
    } else {
        for (uint32_t i = 0; i < a.nrows; ++i) {
            const uint32_t h = row_hi(d.seed[a.row0 + i], c.cx, c.cy, c.cz) >> a.hshift;
            const uint32_t bin = (h >> (a.S + 1)) + a.rbase[i] + (WIN ? c.bin0 : 0u);
            const uint32_t code = h & a.code_mask;
            const uint32_t w = atomicAdd(&s.fill[bin], 0x10002u);
            if ((w >> 16) < a.slot)
                *reinterpret_cast<uint16_t *>(ring + bin * rbytes + (w & (rbytes - 1))) = (uint16_t)code;
            else
                stage_full<WIN>(bin, code, a, s, C);
        }
    }
}

// 32 bytes to global memory in one store (address 32-byte aligned).
__device__ __forceinline__ void store32(void *dst, const uint4 &lo, const uint4 &hi) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(dst), "r"(lo.x), "r"(lo.y), "r"(lo.z), "r"(lo.w), "r"(hi.x), "r"(hi.y),
                    "r"(hi.z), "r"(hi.w)
                 : "memory");
}

// Eight ring entries from entry index e (relative to p0, a multiple of 8);
// entries at or after pad_from (even) become cancelling pairs.
__device__ __forceinline__ uint4 ring_chunk(const uint16_t *ring, uint32_t p0, uint32_t e,
                                            uint32_t pad_from, const ScatterArgs &a) {
    uint4 v = *reinterpret_cast<const uint4 *>(ring + ((p0 + e) & (a.slot - 1)));
    if (e + 8 > pad_from) {                            // the padded tail of a last half
        uint32_t q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e + 2 * u >= pad_from) q[u] = kPadPair;
        v = make_uint4(q[0], q[1], q[2], q[3]);
    }
    return v;
}

// Copy `cnt` ring entries of `bin` from ring position p0 (a multiple of 8) to
// the block's region of the bin at code offset rp, shared by the TS lanes of a
// team (lane tl of it); the part past the region's capacity is added directly.
// Entries at or after index pad_from (relative to p0, even) are written as
// cancelling pairs (the last, partial half).  Halves of 16 or more entries
// leave in whole 32-byte sectors, one store each.
__device__ __forceinline__ void write_out(uint32_t bin, uint32_t gbin, uint32_t p0, uint32_t cnt,
                                          uint32_t rp, uint32_t pad_from, uint32_t tl, uint32_t TS,
                                          const ScatterArgs &a, const Smem &s, uint32_t *C) {
    const uint32_t g = a.B.ngroups > 1 ? __umulhi(gbin, a.gmagic) : 0u;
    const uint32_t cap = s.gcap[g];
    uint16_t *dst = a.B.codes + s.gbase[g] +
                    ((uint64_t)blockIdx.x * a.B.bpg + (gbin - g * a.B.bpg)) * cap;
    const uint32_t fit = rp >= cap ? 0u : min(cnt, cap - rp);
    const uint16_t *ring = s.ring + bin * a.slot;
    if (a.half >= 16) {
        for (uint32_t j = tl; j < fit / 16; j += TS)
            store32(dst + rp + 16 * j, ring_chunk(ring, p0, 16 * j, pad_from, a),
                    ring_chunk(ring, p0, 16 * j + 8, pad_from, a));
    } else {
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + rp);
        for (uint32_t j = tl; j < fit / 8; j += TS) d4[j] = ring_chunk(ring, p0, 8 * j, pad_from, a);
    }
    for (uint32_t e = fit + tl; e < cnt && e < pad_from; e += TS)   // region full: add directly
        direct_add(C, a.S, gbin, ring[(p0 + e) & (a.slot - 1)]);
}

// How many entries of a bin to write: every complete half (oldest first);
// final: everything, the last half padded.
__device__ __forceinline__ uint32_t flush_count(uint32_t pend, bool final, const ScatterArgs &a) {
    if (final) return (pend + a.half - 1) & ~(a.half - 1);
    return pend >= a.slot ? a.slot : (pend >= a.half ? a.half : 0u);
}

// Flush ring slot b (global bin gb) whose fill word is w (lane tl of a team
// of TS lanes): returns the entries written.  final: an odd last entry is
// added directly so the padding is whole cancelling pairs.
__device__ __forceinline__ uint32_t flush_bin(uint32_t b, uint32_t gb, uint32_t w, uint32_t rp,
                                              bool final, uint32_t tl, uint32_t TS,
                                              const ScatterArgs &a, const Smem &s, uint32_t *C) {
    const uint32_t pend = w >> 16;
    const uint32_t cnt = flush_count(pend, final, a);
    if (!cnt) return 0;
    const uint32_t p0 = (((w & 0xFFFFu) >> 1) - pend) & (a.slot - 1);   // the oldest entry
    uint32_t pad_from = 0xFFFFFFFFu;
    if (final) {
        pad_from = pend & ~1u;
        if ((pend & 1u) && tl == 0)
            direct_add(C, a.S, gb, s.ring[b * a.slot + ((p0 + pend - 1) & (a.slot - 1))]);
    }
    write_out(b, gb, p0, cnt, rp, pad_from, tl, TS, a, s, C);
    return cnt;
}

// Flush phase, between two block barriers (no code is staged meanwhile):
// every bin whose ring holds a complete half writes it to the block's region,
// and every fill word's byte offset is reduced modulo the ring.  final: every
// bin writes everything it holds and leaves its region fill in global memory.
// A batch window moving to start at volume nw does the same as final for the
// ring slots whose volume leaves, then loads the entering bins' region fills.
// A team of TS lanes takes one bin: one lane while halves are small, a whole
// warp for the large halves of sketches with few bins.
template <bool WIN>
__device__ __forceinline__ void flush_phase(bool final, uint32_t nw, const ScatterArgs &a,
                                            const Smem &s, uint32_t *C) {
    const uint32_t rmask = 2 * a.slot - 1;
    const uint32_t TS = a.team, per = 32 / TS;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t tl = lane & (TS - 1);
    if (!WIN) {   // rings of fixed bins
        for (uint32_t base = warp * per; base < a.nbins; base += nwarps * per) {
            const uint32_t b = base + lane / TS;
            if (b < a.nbins) {   // a team of 32 is the whole warp, so uniform when TS > 1
                const uint32_t w = s.fill[b];
                const uint32_t rp = s.cur[b];
                const uint32_t gb = b + a.bin_base;
                const uint32_t cnt = flush_bin(b, gb, w, rp, final, tl, TS, a, s, C);
                if (TS > 1) __syncwarp();   // the team has read the words lane 0 rewrites
                if (tl == 0) {
                    if (final) {
                        a.B.fill[(uint64_t)gb * a.B.nblocks + blockIdx.x] = rp + cnt;
                    } else {
                        s.cur[b] = rp + cnt;
                        s.fill[b] = (w - (cnt << 16)) & (0xFFFF0000u | rmask);
                    }
                }
            }
        }
        return;
    }
    for (uint32_t base = warp * per; base < a.nbins; base += nwarps * per) {   // warp-uniform
        const uint32_t b = base + lane / TS;
        uint32_t w = 0, rp = 0, cnt = 0, gb = kNoBin, ng = kNoBin;
        bool leave = final;
        if (b < a.nbins) {
            w = s.fill[b];
            rp = s.cur[b];
            gb = gbin_of<WIN>(a, s, b);
            if (WIN && !final) {
                ng = window_gbin(a, nw, b);
                leave = ng != gb;
            }
            if (!WIN || gb != kNoBin) cnt = flush_bin(b, gb, w, rp, leave, tl, TS, a, s, C);
        }
        __syncwarp();          // the team has read the slot's words
        if (b < a.nbins && tl == 0) {
            if (leave) {
                if (!WIN || gb != kNoBin) a.B.fill[(uint64_t)gb * a.B.nblocks + blockIdx.x] = rp + cnt;
                if (WIN && !final) {  // the slot's next volume enters
                    s.gbin[b] = ng;
                    s.fill[b] = 0;
                    s.cur[b] = ng != kNoBin ? a.B.fill[(uint64_t)ng * a.B.nblocks + blockIdx.x] : 0u;
                }
            } else {
                s.cur[b] = rp + cnt;
                s.fill[b] = (w - (cnt << 16)) & (0xFFFF0000u | rmask);
            }
        }
    }
}

// Packed cells of a warp's queue, one per lane for the first `cnt` lanes.
template <int T, bool BATCH>
__device__ __forceinline__ void stage_queue(const uint64_t *q, uint32_t cnt, const SketchDesc &d,
                                            const ScatterArgs &a, const Smem &s, uint32_t *C) {
    const uint32_t lane = threadIdx.x & 31;
    if (lane < cnt) {
        const uint64_t v = q[lane];
        stage_cell<T, BATCH>(BATCH ? unpack_cell_batch(v) : unpack_cell(v), d, a, s, C);
    }
}

// The scatter: a persistent grid of B.nblocks blocks, each taking every
// gridDim.x-th tile of 3072 particles (one group of 4 particles per thread,
// loaded as three float4, the next tile's group loaded before this one is
// processed).  A flush phase between two block barriers follows every
// `rounds` tiles.  SAMPLED: the call's rate is below 1 (kept cells then go
// through per-warp queues); VEC: the input is 16-byte aligned.
template <int T, bool VEC, int MODE, bool SAMPLED>
__global__ void __launch_bounds__(kScatterThreads, 1)
    k_bin_scatter(const float *__restrict__ xyz, const SketchDesc d, const ScatterArgs a,
                  uint32_t *__restrict__ C) {
    constexpr bool BATCH = MODE == kModeBatch;
    constexpr bool PACKED = MODE == kModePlainPacked || MODE == kModeSuperPacked ||
                            MODE == kModeCells || MODE == kModeSuperCells;
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout Ly = smem_layout(a.nbins, a.slot, a.B.ngroups, SAMPLED ? 1u : 0u, BATCH);
    Smem s;
    s.fill = reinterpret_cast<uint32_t *>(smem + Ly.fill);
    s.cur = reinterpret_cast<uint32_t *>(smem + Ly.cur);
    s.gbase = reinterpret_cast<uint64_t *>(smem + Ly.gbase);
    s.gcap = reinterpret_cast<uint32_t *>(smem + Ly.gcap);
    s.gbin = reinterpret_cast<uint32_t *>(smem + Ly.gbin);
    s.ring = reinterpret_cast<uint16_t *>(smem + Ly.ring);
    s.queue = reinterpret_cast<uint64_t *>(smem + Ly.queue);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t per_tile = (uint64_t)blockDim.x * kPPT;
    uint64_t n = a.n;                          // elements this launch takes
    if (a.n_dev) {
        const uint64_t total = *a.n_dev;
        n = total > a.n_base ? min(a.n, total - a.n_base) : 0;
    }
    const uint64_t ntiles = (n + per_tile - 1) / per_tile;
    // batch window: starts at the first volume of the block's first tile
    uint32_t w0 = BATCH && blockIdx.x < ntiles ? (a.tvols[blockIdx.x] & 0xFFFFu) : 0u;
    for (uint32_t b = threadIdx.x; b < a.nbins; b += blockDim.x) {
        const uint32_t gb = BATCH ? window_gbin(a, w0, b) : b + a.bin_base;
        if (BATCH) s.gbin[b] = gb;
        s.fill[b] = 0;
        s.cur[b] = gb != kNoBin ? a.B.fill[(uint64_t)gb * a.B.nblocks + blockIdx.x] : 0u;
    }
    for (uint32_t g = threadIdx.x; g < a.B.ngroups; g += blockDim.x) {
        s.gbase[g] = a.B.gbase[g];
        s.gcap[g] = a.B.gcap[g];
    }
    __syncthreads();

    const float Gf = (float)d.Gq;
    const uint64_t full_groups = n / kPPT;
    const float4 *p4 = reinterpret_cast<const float4 *>(xyz);
    const uint4 *r4 = reinterpret_cast<const uint4 *>(xyz);
    const unsigned long long *rec = reinterpret_cast<const unsigned long long *>(xyz);
    uint64_t *q = s.queue + (uint64_t)warp * kQueue;
    uint32_t nq = 0;                          // cells in this warp's queue
    const unsigned lt = (1u << lane) - 1u;
    float4 nu = make_float4(0, 0, 0, 0), nv = nu, nw = nu;   // next group (float input)
    uint4 na = make_uint4(0, 0, 0, 0), nb = na;              // next group (packed input)
    uint64_t tile = blockIdx.x;
    if (VEC && tile < ntiles) {
        const uint64_t g4 = tile * blockDim.x + threadIdx.x;
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
    while (tile < ntiles) {                   // block-uniform
        for (uint32_t rnd = 0; rnd < a.rounds && tile < ntiles; ++rnd, tile += gridDim.x) {
            const uint64_t g4 = tile * blockDim.x + threadIdx.x;
            // does this tile hold particles of the probe window?
            const uint64_t tg0 = a.g0 + tile * per_tile;
            const bool probe_tile = tg0 < a.probe_end && tg0 + per_tile > a.probe_base;
            Cell c[kPPT];
            bool ok[kPPT];
            const bool full = VEC && g4 < full_groups;
            if (PACKED) {
                const uint4 ua = na, ub = nb;
                const uint64_t gn = (tile + gridDim.x) * blockDim.x + threadIdx.x;
                if (VEC && tile + gridDim.x < ntiles && gn < full_groups) {
                    na = __ldcs(r4 + 2 * gn);
                    nb = __ldcs(r4 + 2 * gn + 1);
                }
                const uint64_t p[kPPT] = {ua.x | ((uint64_t)ua.y << 32), ua.z | ((uint64_t)ua.w << 32),
                                          ub.x | ((uint64_t)ub.y << 32), ub.z | ((uint64_t)ub.w << 32)};
                const uint64_t g = a.g0 + kPPT * g4;
                if (full && !probe_tile) {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) ok[j] = prep_record<MODE, SAMPLED, false>(p[j], g + j, d, a, c[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        const uint64_t i = kPPT * g4 + j;
                        ok[j] = i < n && prep_record<MODE, SAMPLED, true>(full ? p[j] : __ldcs(rec + i),
                                                                            a.g0 + i, d, a, c[j]);
                    }
                }
            } else {
                const float4 u = nu, v = nv, w = nw;
                const uint64_t gn = (tile + gridDim.x) * blockDim.x + threadIdx.x;
                if (VEC && tile + gridDim.x < ntiles && gn < full_groups) {
                    nu = __ldcs(p4 + 3 * gn);
                    nv = __ldcs(p4 + 3 * gn + 1);
                    nw = __ldcs(p4 + 3 * gn + 2);
                }
                const float px[kPPT] = {u.x, u.w, v.z, w.y}, py[kPPT] = {u.y, v.x, v.w, w.z},
                            pz[kPPT] = {u.z, v.y, w.x, w.w};
                const uint32_t tv = BATCH ? a.tvols[tile] : 0u;
                if (BATCH && (tv >> 16) == (tv & 0xFFFFu) && (tv & 0xFFFFu) - w0 < a.wvols) {
                    // the whole tile in one volume of the window (block-uniform)
                    const uint32_t v = tv & 0xFFFFu;
                    const VolumeDesc &V = a.vols[v];
                    const uint64_t vg = V.g0 - V.start, pbase = V.probe_base;
                    const float inv = V.inv_cell;
                    const uint32_t G = V.G, bin0 = (v & (a.wvols - 1)) * a.bpv;
                    uint64_t *probe_v = a.probe ? a.probe + (uint64_t)v * a.probe_per_vol : nullptr;
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        const uint64_t i = kPPT * g4 + j;
                        ok[j] = i < n &&
                                (full ? prep_particle_vol<SAMPLED>(px[j], py[j], pz[j], i, vg, inv, G, bin0,
                                                                   probe_v, pbase, a, c[j])
                                      : prep_particle_vol<SAMPLED>(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                                                   __ldcs(xyz + 3 * i + 2), i, vg, inv, G, bin0,
                                                                   probe_v, pbase, a, c[j]));
                    }
                } else if (BATCH) {   // from the tile's first volume upward per lane
                    uint32_t vh = tv & 0xFFFFu;
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        const uint64_t i = kPPT * g4 + j;
                        ok[j] = i < n &&
                                (full ? prep_particle_batch<SAMPLED>(px[j], py[j], pz[j], i, d, a, w0, vh, c[j], C)
                                      : prep_particle_batch<SAMPLED>(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                                                     __ldcs(xyz + 3 * i + 2), i, d, a, w0, vh,
                                                                     c[j], C));
                    }
                } else if (full && !probe_tile) {
                    const uint64_t g = a.g0 + kPPT * g4;
#pragma unroll
                    for (int j = 0; j < kPPT; ++j)
                        ok[j] = prep_particle<MODE, SAMPLED, false>(px[j], py[j], pz[j], g + j, Gf, d, a, c[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        const uint64_t i = kPPT * g4 + j;
                        ok[j] = i < n &&
                                (full ? prep_particle<MODE, SAMPLED, true>(px[j], py[j], pz[j], a.g0 + i, Gf, d, a, c[j])
                                      : prep_particle<MODE, SAMPLED, true>(__ldcs(xyz + 3 * i), __ldcs(xyz + 3 * i + 1),
                                                                           __ldcs(xyz + 3 * i + 2), a.g0 + i, Gf, d, a,
                                                                           c[j]));
                    }
                }
            }
            if (!SAMPLED) {
                // every particle is kept unless its position is invalid (or the
                // tail): stage straight from registers
                if (__all_sync(0xFFFFFFFFu, ok[0] & ok[1] & ok[2] & ok[3])) {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) stage_cell<T, BATCH>(c[j], d, a, s, C);
                } else {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j)
                        if (ok[j]) stage_cell<T, BATCH>(c[j], d, a, s, C);
                }
            } else {
                // kept cells go through the warp's queue, 32 at a time, so the
                // row updates run with every lane busy whatever the sample rate
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, ok[j]);
                    if (ok[j]) q[nq + __popc(m & lt)] = BATCH ? pack_cell_batch(c[j]) : pack_cell(c[j]);
                    nq += __popc(m);
                    if (nq >= 32) {
                        __syncwarp();
                        stage_queue<T, BATCH>(q, 32, d, a, s, C);
                        __syncwarp();
                        if (lane < nq - 32) q[lane] = q[32 + lane];
                        nq -= 32;
                        __syncwarp();
                    }
                }
            }
        }
        if (SAMPLED && nq) {          // the rest of the queue before the flush
            __syncwarp();
            stage_queue<T, BATCH>(q, nq, d, a, s, C);
            nq = 0;
            __syncwarp();
        }
        // a batch window moves to the next period's first volume when that
        // period's volumes do not all fall in it (one tile a period then)
        if (BATCH && threadIdx.x == 0) {
            uint32_t nw = w0;
            if (tile < ntiles) {
                const uint32_t tv = a.tvols[tile];
                if ((tv & 0xFFFFu) - w0 >= a.wvols || (tv >> 16) - w0 >= a.wvols) nw = tv & 0xFFFFu;
            }
            s.gbin[a.nbins] = nw;
        }
        __syncthreads();
        const uint32_t nw = BATCH ? s.gbin[a.nbins] : 0u;
        flush_phase<BATCH>(false, nw, a, s, C);
        w0 = nw;
        __syncthreads();
    }
    // every bin now holds fewer than `half` staged codes: write the partial
    // half, padded with cancelling pairs, and leave the region fill in global
    flush_phase<BATCH>(true, 0u, a, s, C);
}

// Launch one variant (the caller filled `a`; smem from smem_layout).
// SAMPLING: instantiate the sampled variants too (cell records never sample).
template <int MODE, bool SAMPLING = true>
cudaError_t launch_mode(const float *xyz, const SketchDesc &d, const ScatterArgs &a, bool sampled,
                        size_t smem, uint32_t *C, cudaStream_t s) {
    const bool vec = (reinterpret_cast<uintptr_t>(xyz) & 15u) == 0;
    auto launch = [&](auto kern) {
        cudaError_t e = ensure_smem_limit(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<a.B.nblocks, kScatterThreads, smem, s>>>(xyz, d, a, C);
        return cudaGetLastError();
    };
    // five rows in one pass (every configuration here but the largest
    // sketches) get a fully unrolled variant; row passes and an unaligned
    // buffer (a slice of a larger one) the generic one
    if constexpr (SAMPLING) {
        if (sampled) {
            if (a.nrows == 5 && a.row0 == 0 && vec) return launch(k_bin_scatter<5, true, MODE, true>);
            if (vec) return launch(k_bin_scatter<0, true, MODE, true>);
            return launch(k_bin_scatter<0, false, MODE, true>);
        }
    } else if (sampled) {
        return cudaErrorInvalidValue;
    }
    if (a.nrows == 5 && a.row0 == 0 && vec) return launch(k_bin_scatter<5, true, MODE, false>);
    if (vec) return launch(k_bin_scatter<0, true, MODE, false>);
    return launch(k_bin_scatter<0, false, MODE, false>);
}

// launchers of the variants, one translation unit each group of modes
cudaError_t launch_modes_sketch(int mode, const float *xyz, const SketchDesc &d, const ScatterArgs &a,
                                bool sampled, size_t smem, uint32_t *C, cudaStream_t s);
cudaError_t launch_modes_batch_route(int mode, const float *xyz, const SketchDesc &d,
                                     const ScatterArgs &a, bool sampled, size_t smem, uint32_t *C,
                                     cudaStream_t s);
cudaError_t launch_modes_cells(int mode, const float *xyz, const SketchDesc &d, const ScatterArgs &a,
                               size_t smem, uint32_t *C, cudaStream_t s);

}  // namespace binned
}  // namespace hs
