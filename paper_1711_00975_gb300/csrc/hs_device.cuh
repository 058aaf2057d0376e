// hs_device.cuh - device-side building blocks of the Count Sketch path.
//
// Mesh reduction (arXiv:1711.00975 Sec. 2.1), index-hash sampling (Sec. 3.1)
// and the per-row bucket/sign hash of the Count Sketch (Sec. 2.2), written for
// sm_103a.  The quantisation multiply uses __fmul_rn so it is one IEEE-754
// float32 rounding and can never be contracted into an FMA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hs {

constexpr int kMaxRows = 32;
// learned router: MLP 27 -> 64 -> 64 -> 1, parameters w1[64][27], b1[64],
// w2[64][64], b2[64], w3[64], b3 in that order
constexpr int kMlpIn = 27;
constexpr int kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;
constexpr int kTableProbes = 64;   // slots tried per key in the exact tables
constexpr uint64_t kInvalidKey = 0xFFFFFFFFFFFFFFFFull;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;   // splitmix64 increment

struct RowSeed {
    uint64_t a0, a1, a2, b;
};

// Everything a kernel needs to hash and quantise; passed by value.
struct SketchDesc {
    uint32_t rows;
    uint32_t log2w;
    uint32_t G;          // cells per axis of the keys this sketch counts
    float inv_cell;
    uint64_t W;
    uint32_t Gq;         // cells per axis of the quantisation mesh (G * F)
    uint32_t F;          // super-item side in cells (1: the cells themselves)
    uint32_t fmagic;     // ceil(2^32 / F): c / F = umulhi(c, fmagic) for c, F < 2^16
    uint32_t pad;
    RowSeed seed[kMaxRows];
};

// splitmix64 output number g of the generator seeded with `seed`
// (Steele, Lea & Flood 2014: state advances by the golden gamma, output mixes it).
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t g) {
    uint64_t z = seed + (g + 1) * kGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Division by an invariant G with one high multiply (the multiply-and-shift
// method of Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994).  With M = ceil(2^48 / G) = (2^48 + e) / G,
// 0 <= e < G, x M / 2^48 = x / G + x e / (G 2^48); writing x = q G + r the
// fraction r / G + x e / (G 2^48) stays below 1 when x e < 2^48, so
// floor(x M / 2^48) = q for every x < 2^48 / G.  div_magic(G) = M << 16 (G >= 2,
// so it fits 64 bits); 0 asks for a plain division.
__host__ __device__ inline uint64_t div_magic(uint32_t G) {
    return G >= 2 ? (((1ull << 48) + G - 1) / G) << 16 : 0ull;
}
__device__ __forceinline__ uint64_t div_invariant(uint64_t x, uint32_t G, uint64_t magic) {
    return magic ? __umul64hi(x, magic) : x / G;
}

// Low 64 bits of a * x for a 64-bit a and 32-bit x: one wide and one narrow
// integer multiply-add instead of a full 64x64 product.
__device__ __forceinline__ uint64_t mul_lo64(uint64_t a, uint32_t x) {
    uint64_t lo = (uint64_t)(uint32_t)a * (uint64_t)x;
    uint32_t hi = (uint32_t)(a >> 32) * x;
    return lo + ((uint64_t)hi << 32);
}

// c + a * b with a 64-bit accumulator in one wide multiply-add.
__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// High 32 bits of v = (a0*cx + a1*cy + a2*cz + b) mod 2^64: the low halves of
// the multipliers go through a 64-bit multiply-add chain starting at b; the
// high halves only reach the top word, so they add in 32-bit arithmetic.
__device__ __forceinline__ uint32_t row_value_hi(const RowSeed &s, uint32_t cx, uint32_t cy,
                                                 uint32_t cz, uint32_t &lo) {
    uint64_t acc = mad_wide((uint32_t)s.a0, cx, s.b);
    acc = mad_wide((uint32_t)s.a1, cy, acc);
    acc = mad_wide((uint32_t)s.a2, cz, acc);
    lo = (uint32_t)acc;
    return (uint32_t)(acc >> 32) + (uint32_t)(s.a0 >> 32) * cx + (uint32_t)(s.a1 >> 32) * cy +
           (uint32_t)(s.a2 >> 32) * cz;
}

// v = (a0*cx + a1*cy + a2*cz + b) mod 2^64 (vector multiply-shift before the shift)
__device__ __forceinline__ uint64_t row_value(const RowSeed &s, uint32_t cx, uint32_t cy,
                                              uint32_t cz) {
    uint32_t lo;
    uint32_t hi = row_value_hi(s, cx, cy, cz, lo);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint32_t bucket_of(uint64_t v, uint32_t log2w) {
    return (uint32_t)(v >> (64 - log2w));
}

// +1 or -1 as an unsigned addend (wrap-around arithmetic)
__device__ __forceinline__ uint32_t sign_of(uint64_t v, uint32_t log2w) {
    return ((v >> (63 - log2w)) & 1ull) ? 0xFFFFFFFFu : 1u;
}

// sign * counter with int32 wrap-around
__device__ __forceinline__ int32_t signed_count(int32_t c, uint64_t v, uint32_t log2w) {
    uint32_t u = (uint32_t)c;
    return ((v >> (63 - log2w)) & 1ull) ? (int32_t)(0u - u) : (int32_t)u;
}

// L_r(cy, cz) = a1*cy + a2*cz + b (mod 2^64): row r's value of mesh line
// (cy, cz) without the cx term (v_r = a0*cx + L_r)
__device__ __forceinline__ uint64_t line_value(const RowSeed &s, uint32_t cy, uint32_t cz) {
    return s.b + mul_lo64(s.a1, cy) + mul_lo64(s.a2, cz);
}

// bit `bucket` of row r of a hot-bucket bitmap (words_per_row 32-bit words a row)
__device__ __forceinline__ bool exact_hot(const uint32_t *__restrict__ bits, uint64_t words_per_row,
                                          int r, uint32_t bucket) {
    return (__ldg(bits + (uint64_t)r * words_per_row + (bucket >> 5)) >> (bucket & 31)) & 1u;
}

// Periodic reduction of a cell index outside [0, G) (rare: only particles
// outside the box); kept out of line so the common path stays short.
static __device__ __noinline__ uint32_t wrap_cell(int i, uint32_t G) {
    int m = i % (int)G;
    if (m < 0) m += (int)G;
    return (uint32_t)m;
}

// One axis of the mesh reduction: floor(fl32(x * inv)) reduced into [0, G).
// Returns false when the scaled coordinate is not a finite value in
// [-2^31, 2^31) (then floor(p) is outside int32 or p is NaN/inf).
__device__ __forceinline__ bool axis_cell(float x, float inv, uint32_t G, uint32_t &c) {
    float p = __fmul_rn(x, inv);
    if (!(p >= -2147483648.0f && p < 2147483648.0f)) return false;
    int i = __float2int_rd(p);      // floor, exact for p in range
    c = (unsigned)i < G ? (uint32_t)i : wrap_cell(i, G);
    return true;
}

// Cell of a particle on the quantisation mesh; for a super-item sketch
// (Algorithm 3) the F x F x F block holding that cell.
__device__ __forceinline__ bool particle_cell(const SketchDesc &d, float x, float y, float z,
                                              uint32_t &cx, uint32_t &cy, uint32_t &cz) {
    bool valid = axis_cell(x, d.inv_cell, d.Gq, cx);
    valid &= axis_cell(y, d.inv_cell, d.Gq, cy);
    valid &= axis_cell(z, d.inv_cell, d.Gq, cz);
    if (d.F > 1) {
        cx = __umulhi(cx, d.fmagic);
        cy = __umulhi(cy, d.fmagic);
        cz = __umulhi(cz, d.fmagic);
    }
    return valid;
}

// ---- packed particle records: 64 bits, three 21-bit coordinates ----
// q = floor(fl32(x * fl32(2^21 / L))) reduced into [0, 2^21), x in bits 0-20,
// y in 21-41, z in 42-62; bit 63 marks coordinates that were not finite.  The
// cell on a mesh of G cells per axis is (q * G) >> 21.
constexpr uint32_t kPackBits = 21;
constexpr uint64_t kPackMask = (1ull << kPackBits) - 1;
constexpr uint64_t kPackInvalid = 1ull << 63;

__device__ __forceinline__ uint32_t packed_axis(uint64_t p, uint32_t a, uint32_t G) {
    return (uint32_t)((((p >> (kPackBits * a)) & kPackMask) * (uint64_t)G) >> kPackBits);
}

// Cell of a packed record on the quantisation mesh; for a super-item sketch
// the F x F x F block holding it.
__device__ __forceinline__ bool packed_cell(const SketchDesc &d, uint64_t p, uint32_t &cx,
                                            uint32_t &cy, uint32_t &cz) {
    cx = packed_axis(p, 0, d.Gq);
    cy = packed_axis(p, 1, d.Gq);
    cz = packed_axis(p, 2, d.Gq);
    if (d.F > 1) {
        cx = __umulhi(cx, d.fmagic);
        cy = __umulhi(cy, d.fmagic);
        cz = __umulhi(cz, d.fmagic);
    }
    return !(p & kPackInvalid);
}

__device__ __forceinline__ uint64_t key_of(uint32_t cx, uint32_t cy, uint32_t cz, uint32_t G) {
    return (uint64_t)cx + (uint64_t)G * ((uint64_t)cy + (uint64_t)G * (uint64_t)cz);
}

// Lower median of n values in registers (n <= kMaxRows), insertion sort.
template <int N>
__device__ __forceinline__ int32_t lower_median_fixed(int32_t (&v)[N]) {
#pragma unroll
    for (int i = 1; i < N; ++i) {
#pragma unroll
        for (int j = i; j > 0; --j) {
            int32_t a = v[j - 1], b = v[j];
            v[j - 1] = min(a, b);
            v[j] = max(a, b);
        }
    }
    return v[(N - 1) / 2];
}

__device__ __forceinline__ int32_t lower_median_dyn(int32_t *v, int n) {
    for (int i = 1; i < n; ++i) {
        int32_t x = v[i];
        int j = i;
        while (j > 0 && v[j - 1] > x) {
            v[j] = v[j - 1];
            --j;
        }
        v[j] = x;
    }
    return v[(n - 1) / 2];
}

// Median of five with six comparisons: sort two pairs; the smaller of the two
// pair minima has three values at or above it, so it cannot be the median and
// is replaced by the fifth value; the median is then the second smallest of the
// four that remain.
__host__ __device__ __forceinline__ int32_t median5(int32_t a, int32_t b, int32_t c, int32_t d,
                                                    int32_t e) {
    int32_t t;
    if (a > b) { t = a; a = b; b = t; }
    if (c > d) { t = c; c = d; d = t; }
    if (a < c) {
        a = e;
        if (a > b) { t = a; a = b; b = t; }
    } else {
        c = e;
        if (c > d) { t = c; c = d; d = t; }
    }
    return (a < c) ? (b < c ? b : c) : (a < d ? a : d);
}

// Cells of coarse cells marked in `bits` (one bit per coarse cell, coarse cell =
// fine cell / R per axis on a Gc^3 mesh) are counted outside the sketch.
struct RouteFilter {
    const uint32_t *bits;   // nullptr: nothing is routed
    uint32_t rmagic;        // ceil(2^32 / R): x / R = umulhi(x, rmagic) for x, R < 2^16
    uint32_t Gc;
    uint32_t R;             // coarse factor
};

__device__ __forceinline__ bool routed_cell(const RouteFilter &f, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    const uint32_t qx = __umulhi(cx, f.rmagic), qy = __umulhi(cy, f.rmagic),
                   qz = __umulhi(cz, f.rmagic);
    const uint64_t ck = (uint64_t)qx + (uint64_t)f.Gc * (qy + (uint64_t)f.Gc * qz);
    return (__ldg(f.bits + (ck >> 5)) >> (ck & 31)) & 1u;
}

// ---- exact open-addressing table: uint64 key (empty = all ones) + int32 count ----
__device__ __forceinline__ uint64_t table_hash(uint64_t k) {
    k ^= k >> 33;
    k *= 0xFF51AFD7ED558CCDull;
    k ^= k >> 33;
    k *= 0xC4CEB9FE1A85EC53ull;
    return k ^ (k >> 33);
}

// Count one particle of cell `key`; false when max_probe slots (linear probing
// from the key's hash) were all taken by other keys.
__device__ __forceinline__ bool table_add(unsigned long long *keys, int32_t *counts, uint64_t mask,
                                          uint64_t key, int max_probe) {
    uint64_t s = table_hash(key) & mask;
    for (int p = 0; p < max_probe; ++p) {
        const unsigned long long cur = atomicCAS(&keys[s], (unsigned long long)kInvalidKey,
                                                 (unsigned long long)key);
        if (cur == kInvalidKey || cur == key) {
            atomicAdd(&counts[s], 1);
            return true;
        }
        s = (s + 1) & mask;
    }
    return false;
}

}  // namespace hs
