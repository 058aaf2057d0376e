// k_dir.cu - output-sensitive full search (estimate mode of Algorithm 1,
// arXiv:1711.00975) for large meshes.
//
// The full search must find every cell whose median estimate reaches theta.
// With theta > 0 such a cell has at least need = t - floor((t-1)/2) rows with
// |C[r][bucket_r]| >= theta ("hot" rows), so it is hot in at least one of the
// first F = t - need + 1 rows.  Each cell is therefore reported from the first
// row r < F in which it is hot, and only from there.
//
// Row r's multiply-shift value of cell (cx, cy, cz) splits as
//     v_r = a0*cx + L_r(cy, cz),   L_r = a1*cy + a2*cz + b   (mod 2^64),
// so the cells of a hot bucket h with a given cx are exactly the mesh lines
// (cy, cz) whose L_r falls in the interval [h*2^s - a0*cx, (h+1)*2^s - a0*cx),
// s = 64 - log2W.  A directory of all G^2 lines bucketed by the top D bits of
// L_r (counting sort: count, scan, scatter) answers each such interval by
// reading at most two directory slots.  The work is proportional to
// F * (G^2 + G * |hot buckets|) instead of G^3, and every cell that could pass
// is still examined exactly once, so the result equals the exhaustive search.
#include <algorithm>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

__global__ void k_dir_count(const SketchDesc d, int r, uint32_t D, uint32_t *__restrict__ cnt) {
    const uint64_t lines = (uint64_t)d.G * d.G;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t line = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; line < lines;
         line += stride) {
        uint32_t cy = (uint32_t)(line % d.G), cz = (uint32_t)(line / d.G);
        uint64_t L = line_value(d.seed[r], cy, cz);
        atomicAdd(&cnt[L >> (64 - D)], 1u);
    }
}

__global__ void k_dir_scatter(const SketchDesc d, int r, uint32_t D, uint32_t *__restrict__ cursor,
                              DirRecord *__restrict__ rec) {
    const uint64_t lines = (uint64_t)d.G * d.G;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t line = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; line < lines;
         line += stride) {
        uint32_t cy = (uint32_t)(line % d.G), cz = (uint32_t)(line / d.G);
        uint64_t L = line_value(d.seed[r], cy, cz);
        uint32_t pos = atomicAdd(&cursor[L >> (64 - D)], 1u);
        rec[pos] = cy | (cz << 16);
    }
}

// ---- exclusive scan of uint32 counts (three-phase, recursive over block sums) ----

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 2 * kScanThreads;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp,
                                                         uint32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        s_warp[lane] = s;   // inclusive warp-sum prefix
    }
    __syncthreads();
    uint32_t warp_off = w ? s_warp[w - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    return warp_off + x - v;
}

// out[i] = sum of in[0..i) within each block of kScanItems; sums[b] = block total
__global__ void k_scan_block(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                             uint64_t n, uint32_t *__restrict__ sums) {
    __shared__ uint32_t s_warp[32];
    uint64_t base = (uint64_t)blockIdx.x * kScanItems + 2 * threadIdx.x;
    uint32_t a = base < n ? in[base] : 0;
    uint32_t b = base + 1 < n ? in[base + 1] : 0;
    uint32_t total;
    uint32_t ex = block_exclusive_scan(a + b, s_warp, &total);
    if (base < n) out[base] = ex;
    if (base + 1 < n) out[base + 1] = ex + a;
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t *__restrict__ out, uint64_t n, const uint32_t *__restrict__ off) {
    uint64_t base = (uint64_t)blockIdx.x * kScanItems + 2 * threadIdx.x;
    uint32_t o = off[blockIdx.x];
    if (base < n) out[base] += o;
    if (base + 1 < n) out[base + 1] += o;
}

cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *scratch,
                           cudaStream_t s, int *launches) {
    uint64_t nb = (n + kScanItems - 1) / kScanItems;
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, scratch);
    *launches += 1;
    if (nb > 1) {
        cudaError_t e = exclusive_scan(scratch, scratch, nb, scratch + nb, s, launches);
        if (e != cudaSuccess) return e;
        k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, scratch);
        *launches += 1;
    }
    return cudaGetLastError();
}

// Signed hot bitmaps of every row (one warp a word): bit b of the positive
// map is set when C[b] >= theta, of the negative map when C[b] <= -theta.  A
// cell's signed count in a row, sign * C[bucket], can reach theta only when
// the map of its sign bit (0: positive, 1: negative) has its bucket set.
// bits: rows x W/32 words of the positive map, then as many of the negative.
__global__ void k_signed_bits(const int32_t *__restrict__ C, uint64_t words, int32_t theta,
                              uint32_t *__restrict__ bits) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < words; w += warps) {
        const int32_t c = __ldcs(C + w * 32 + lane);
        const unsigned pos = __ballot_sync(0xFFFFFFFFu, c >= theta);
        const unsigned neg = __ballot_sync(0xFFFFFFFFu, c <= -theta);
        if (lane == 0) {
            bits[w] = pos;
            bits[words + w] = neg;
        }
    }
}

// row r's hot buckets with the sign a cell must have there: entries
// bucket << 1 | sign bit (positive map: 0, negative map: 1)
__global__ void k_hot_list(const uint32_t *__restrict__ bits, uint64_t words_per_row,
                           uint64_t words, int r, uint32_t *__restrict__ list,
                           unsigned long long *__restrict__ count, uint64_t cap) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * words_per_row;
         i += stride) {
        const uint32_t neg = i >= words_per_row;
        const uint64_t w = i - neg * words_per_row;
        uint32_t x = bits[neg * words + (uint64_t)r * words_per_row + w];
        if (!x) continue;
        unsigned long long base = atomicAdd(count, (unsigned long long)__popc(x));
        while (x) {
            int b = __ffs(x) - 1;
            x &= x - 1;
            if (base < cap) list[base] = ((uint32_t)(w * 32 + b) << 1) | neg;
            ++base;
        }
    }
}

// Is row rr of the cell whose row value is v hot for its sign?
__device__ __forceinline__ bool signed_hot(const uint32_t *__restrict__ bits, uint64_t words_per_row,
                                           uint64_t words, uint32_t rr, uint64_t v, uint32_t log2w) {
    const uint32_t b = bucket_of(v, log2w);
    const uint64_t neg = (v >> (63 - log2w)) & 1ull;
    return (__ldg(bits + neg * words + (uint64_t)rr * words_per_row + (b >> 5)) >> (b & 31)) & 1u;
}

// The first records of every slot, inline: slot i's 16-byte entry holds its
// records (up to kInline of them) followed by kEmpty, or kInline times kCrowded
// when the slot has more (then the counting-sorted arrays are read).  A record
// is cy | cz << 16 with cz < G - 1 < 65535, so neither marker is a record.
constexpr uint32_t kInline = 4;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kCrowded = 0xFFFFFFFEu;

__global__ void k_dir_inline(const uint32_t *__restrict__ offsets, const DirRecord *__restrict__ rec,
                             uint64_t nslots, uint4 *__restrict__ inl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += stride) {
        const uint32_t e0 = offsets[i], n = offsets[i + 1] - e0;
        uint4 v;
        if (n > kInline) {
            v = make_uint4(kCrowded, kCrowded, kCrowded, kCrowded);
        } else {
            v.x = n > 0 ? rec[e0] : kEmpty;
            v.y = n > 1 ? rec[e0 + 1] : kEmpty;
            v.z = n > 2 ? rec[e0 + 2] : kEmpty;
            v.w = n > 3 ? rec[e0 + 3] : kEmpty;
        }
        inl[i] = v;
    }
}

// The cells of a warp's lines that fall in their pair's bucket wait in a
// per-warp queue and are checked 32 at a time, every lane busy: a line's
// checks (other rows' hot bits, then the estimate) cost far more than
// finding it, and pairs hold different numbers of lines.
constexpr int kDirWarps = 8;          // 256 threads
constexpr int kLineQueue = 64;

__device__ __forceinline__ uint64_t pack_line(uint32_t cx, uint32_t cy, uint32_t cz) {
    return (uint64_t)cx | ((uint64_t)cy << 16) | ((uint64_t)cz << 32);
}

// One queued cell: reported when row r is its first hot row, at least `need`
// rows are hot and its estimate passes.
template <int T>
__device__ __forceinline__ void dir_check(uint64_t cell, const int32_t *__restrict__ C,
                                          const SketchDesc &d, int r, const uint32_t *__restrict__ bits,
                                          int32_t theta, uint32_t mode, const SearchOut &out) {
    const uint32_t rows = T > 0 ? (uint32_t)T : d.rows;
    const uint32_t need = rows - (rows - 1) / 2;
    const uint64_t words_per_row = d.W >> 5;
    const uint64_t words = (uint64_t)rows * words_per_row;
    const uint32_t cx = (uint32_t)(cell & 0xFFFFu), cy = (uint32_t)((cell >> 16) & 0xFFFFu),
                   cz = (uint32_t)(cell >> 32);
    // the cell is reported from its first hot row r: the rows before r must
    // be cold, so its hot rows are r and rows after r, of which at least
    // `need` must be hot.  The rows after r come first: a line stops as soon
    // as the rows left cannot make `need` (after one cold row for r = t - need,
    // two for r one less, ...); the rows before r, nearly always cold, last.
    uint32_t nhot = 1, left = rows - 1 - (uint32_t)r;
    for (uint32_t rr = (uint32_t)r + 1; rr < rows; ++rr) {
        nhot += signed_hot(bits, words_per_row, words, rr, row_value(d.seed[rr], cx, cy, cz), d.log2w);
        if (nhot + --left < need) return;
    }
    if (nhot < need) return;
    for (uint32_t rr = 0; rr < (uint32_t)r; ++rr)
        if (signed_hot(bits, words_per_row, words, rr, row_value(d.seed[rr], cx, cy, cz), d.log2w)) return;
    int32_t ev[T > 0 ? T : kMaxRows];
    for (uint32_t rr = 0; rr < rows; ++rr) {
        const uint64_t v = row_value(d.seed[rr], cx, cy, cz);
        ev[rr] = signed_count(__ldg(C + rr * d.W + bucket_of(v, d.log2w)), v, d.log2w);
    }
    const int32_t est = T == 5 ? median5(ev[0], ev[1], ev[2], ev[3], ev[4])
                               : lower_median_dyn(ev, (int)rows);
    const bool pass = mode == kGE ? est >= theta : (mode == kGT ? est > theta : est == theta);
    if (!pass) return;
    const unsigned long long idx = atomicAdd(out.count, 1ull);
    if (idx < out.cap) {
        out.key[idx] = key_of(cx, cy, cz, d.G);
        out.est[idx] = est;
    }
}

// one lane per (cx, hot bucket of row r); the warp's items advance together
template <int T>
__global__ void __launch_bounds__(256)
    k_dir_query(const int32_t *__restrict__ C, const SketchDesc d, int r, uint32_t D,
                const uint32_t *__restrict__ offsets, const DirRecord *__restrict__ rec,
                const uint4 *__restrict__ inl, const uint32_t *__restrict__ hot, uint64_t n_hot,
                const uint32_t *__restrict__ bits, int32_t theta, uint32_t mode, uint64_t line_lo,
                uint64_t line_hi, SearchOut out, RouteFilter skip, uint64_t gmagic) {
    __shared__ uint64_t queue[kDirWarps][kLineQueue];
    const uint32_t s = 64 - d.log2w;
    const uint64_t nslots = 1ull << D;
    const uint64_t total = n_hot * d.G;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t *q = queue[warp];
    uint32_t nq = 0;
    // check 32 queued cells (the oldest), keep the rest
    auto drain = [&]() {
        __syncwarp();
        dir_check<T>(q[lane], C, d, r, bits, theta, mode, out);
        __syncwarp();
        if (lane < nq - 32) q[lane] = q[32 + lane];
        nq -= 32;
        __syncwarp();
    };
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5; base < total;
         base += warps << 5) {                                   // warp-uniform
        const uint64_t i = base + lane;
        const bool item = i < total;
        uint32_t h = 0, cx = 0, nslot = 0;
        uint64_t Tx = 0;
        uint4 v[2] = {make_uint4(kEmpty, kEmpty, kEmpty, kEmpty), make_uint4(kEmpty, kEmpty, kEmpty, kEmpty)};
        uint64_t slot0 = 0;
        if (item) {
            const uint64_t hi = div_invariant(i, d.G, gmagic);   // i = hi G + cx
            h = hot[hi];                                         // bucket << 1 | sign bit
            cx = (uint32_t)(i - hi * d.G);
            Tx = d.seed[r].a0 * (uint64_t)cx;
            // the lines whose cell in column cx has bucket and sign bit h: L in
            // [h 2^(s-1) - Tx, (h+1) 2^(s-1) - Tx), one slot or two
            const uint64_t lo = ((uint64_t)h << (s - 1)) - Tx;
            slot0 = lo >> (64 - D);
            nslot = ((lo + ((1ull << (s - 1)) - 1)) >> (64 - D)) == slot0 ? 1u : 2u;
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if ((uint32_t)j < nslot)
                    v[j] = inl ? __ldg(inl + ((slot0 + j) & (nslots - 1))) : make_uint4(kCrowded, 0, 0, 0);
        }
        // a line (cy, cz) whose cell in column cx has bucket and sign h,
        // inside the pass's line window and not routed, is a cell to check
        auto wanted = [&](DirRecord p) {
            const uint32_t cy = p & 0xFFFFu, cz = p >> 16;
            if (((line_value(d.seed[r], cy, cz) + Tx) >> (s - 1)) != h) return false;
            const uint64_t line = (uint64_t)cy + (uint64_t)d.G * cz;
            if (line < line_lo || line >= line_hi) return false;
            return !(skip.bits && routed_cell(skip, cx, cy, cz));
        };
        auto push = [&](bool take, DirRecord p) {            // all lanes of the warp
            const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
            if (take) q[nq + __popc(m & lt)] = pack_line(cx, p & 0xFFFFu, p >> 16);
            nq += __popc(m);
            if (nq >= 32) drain();
        };
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint32_t e[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
            const bool crowded = e[0] == kCrowded;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = item && !crowded && e[u] != kEmpty && wanted(e[u]);
                push(ok, e[u]);
            }
            // a slot with more lines than an inline entry holds: its records,
            // the warp walking the longest list
            uint32_t e0 = 0, e1 = 0;
            if (item && crowded && (uint32_t)j < nslot) {
                const uint64_t slot = (slot0 + j) & (nslots - 1);
                e0 = offsets[slot];
                e1 = offsets[slot + 1];
            }
            const uint32_t len = e1 - e0;
            uint32_t most = len;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) most = max(most, __shfl_xor_sync(0xFFFFFFFFu, most, o));
            for (uint32_t k = 0; k < most; ++k) {
                const DirRecord p = k < len ? rec[e0 + k] : 0u;
                push(k < len && wanted(p), p);
            }
        }
    }
    __syncwarp();
    if (lane < nq) dir_check<T>(q[lane], C, d, r, bits, theta, mode, out);   // the rest
}

}  // namespace

// exclusive prefix sum of n uint32 (in place allowed); scratch: n / 1024 + 4096 words
cudaError_t launch_exclusive_scan(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *scratch,
                                  cudaStream_t s, int *launches) {
    if (n == 0) return cudaSuccess;
    return exclusive_scan(in, out, n, scratch, s, launches);
}

cudaError_t launch_dir_build(const SketchDesc &d, int r, uint32_t D, bool inl, uint32_t *offsets,
                             uint32_t *cursor, DirRecord *rec, uint32_t *scan_scratch,
                             int max_blocks, cudaStream_t s, int *launches) {
    const uint64_t nslots = 1ull << D;
    cudaError_t e = cudaMemsetAsync(cursor, 0, (nslots + 1) * 4, s);
    if (e != cudaSuccess) return e;
    const uint64_t lines = (uint64_t)d.G * d.G;
    uint64_t blocks = (lines + 255) / 256;
    if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
    k_dir_count<<<(unsigned)blocks, 256, 0, s>>>(d, r, D, cursor);
    *launches += 1;
    e = exclusive_scan(cursor, offsets, nslots + 1, scan_scratch, s, launches);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(cursor, offsets, nslots * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    k_dir_scatter<<<(unsigned)blocks, 256, 0, s>>>(d, r, D, cursor, rec);
    *launches += 1;
    if (inl) {
        uint64_t sb = std::min<uint64_t>((nslots + 255) / 256, (uint64_t)max_blocks);
        k_dir_inline<<<(unsigned)std::max<uint64_t>(sb, 1), 256, 0, s>>>(offsets, rec, nslots,
                                                                         dir_inline(offsets, D));
        *launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_signed_bits(const int32_t *C, const SketchDesc &d, int32_t theta, uint32_t *bits,
                               int max_blocks, cudaStream_t s) {
    if (d.W < 32 || theta < 1) return cudaErrorInvalidValue;
    const uint64_t words = (uint64_t)d.rows * (d.W >> 5);
    const uint64_t blocks = std::min<uint64_t>((words * 32 + 255) / 256, (uint64_t)max_blocks);
    k_signed_bits<<<(unsigned)blocks, 256, 0, s>>>(C, words, theta, bits);
    return cudaGetLastError();
}

cudaError_t launch_hot_list(const uint32_t *bits, const SketchDesc &d, int r, uint32_t *list,
                            unsigned long long *count, uint64_t cap, int max_blocks,
                            cudaStream_t s) {
    const uint64_t wpr = d.W >> 5;
    const uint64_t blocks = std::min<uint64_t>((2 * wpr + 255) / 256, (uint64_t)max_blocks);
    k_hot_list<<<(unsigned)blocks, 256, 0, s>>>(bits, wpr, (uint64_t)d.rows * wpr, r, list, count, cap);
    return cudaGetLastError();
}

cudaError_t launch_dir_query(const int32_t *C, const SketchDesc &d, int r, uint32_t D, bool inl,
                             const uint32_t *offsets, const DirRecord *rec, const uint32_t *hot,
                             uint64_t n_hot, const uint32_t *bits, int32_t theta, SearchMode mode,
                             uint64_t line_lo, uint64_t line_hi, SearchOut out, int max_blocks,
                             cudaStream_t s, RouteFilter skip) {
    uint64_t total = n_hot * d.G;
    if (total == 0) return cudaSuccess;
    uint64_t blocks = (total + 255) / 256;
    if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
    // the multiply form of q / G holds for q < 2^48 / G
    const uint64_t gmagic = total < (1ull << 48) / d.G ? div_magic(d.G) : 0ull;
    if (d.rows == 5)
        k_dir_query<5><<<(unsigned)blocks, 256, 0, s>>>(C, d, r, D, offsets, rec,
                                                       inl ? dir_inline(offsets, D) : nullptr,
                                                       hot, n_hot, bits,
                                                       theta, mode, line_lo, line_hi, out, skip,
                                                       gmagic);
    else
        k_dir_query<0><<<(unsigned)blocks, 256, 0, s>>>(C, d, r, D, offsets, rec,
                                                       inl ? dir_inline(offsets, D) : nullptr,
                                                       hot, n_hot, bits,
                                                       theta, mode, line_lo, line_hi, out, skip,
                                                       gmagic);
    return cudaGetLastError();
}

}  // namespace hs
