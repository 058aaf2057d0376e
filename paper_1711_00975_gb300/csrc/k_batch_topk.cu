// k_batch_topk.cu - the top-k query (Algorithm 1's query, the CSFS design of
// arXiv:1711.00975 Sec. 3.1) of every sketch of a batch of sub-volumes in one
// fixed sequence of launches, with no host round trip, so that it is captured
// once as a CUDA graph and replayed.
//
// Per volume v, all volumes at once in each launch:
//  1. the distinct cells of the first particles of v's stream (the probe) and
//     their estimates;
//  2. theta_v = the kk-th largest of those estimates (a lower bound on the
//     kk-th largest estimate over all cells), by a radix select in one block;
//  3. the signed hot maps of every row (C >= theta_v, C <= -theta_v): a cell
//     whose sign in row r is s_r can reach theta_v only where s_r C >= theta_v;
//  4. the hot (bucket, sign) pairs of the first F rows, listed;
//  5. per volume the cheaper search: a scan of its G_v^3 cells, or directory
//     queries (|hot pairs| * G_v a row); the work prefix-summed;
//  6. both searches over all volumes in one persistent grid: every cell with
//     estimate >= theta_v is a candidate;
//  7. one block per volume finds the kk-th best candidate (estimate desc, key
//     asc) by radix selects and sorts the kk candidates ranked at or above it.
// Each step that meets a case outside its fixed capacities (fewer probe cells
// than kk, theta_v < 1, too many hot buckets or candidates) marks the volume
// in `status`; the host answers those volumes by the general path.  Every
// cell with estimate >= theta_v is examined exactly once (the first of the F
// rows in which it is hot reports it), so the kept cells equal the
// exhaustive search's.
#include <algorithm>

#include "hs_device.cuh"
#include "hs_kernels.h"

namespace hs {

namespace {

constexpr uint32_t kProbeFull = 1u;      // fewer distinct probe cells than kk, or theta < 1
constexpr uint32_t kHotFull = 2u;        // a row's hot buckets exceed the list
constexpr uint32_t kCandFull = 4u;       // candidates exceed the buffer (or fewer than kk)
constexpr uint32_t kSetFull = 8u;        // the probe set's probe length ran out

__device__ __forceinline__ void cell_of_key(uint64_t key, uint32_t G, uint32_t &cx, uint32_t &cy,
                                            uint32_t &cz) {
    cx = (uint32_t)(key % G);
    const uint64_t rest = key / G;
    cy = (uint32_t)(rest % G);
    cz = (uint32_t)(rest / G);
}

template <int T>
__device__ __forceinline__ int32_t estimate(const int32_t *__restrict__ C, const SketchDesc &d,
                                            uint32_t rows, uint32_t cx, uint32_t cy, uint32_t cz) {
    int32_t ev[T > 0 ? T : kMaxRows];
    for (uint32_t r = 0; r < rows; ++r) {
        const uint64_t v = row_value(d.seed[r], cx, cy, cz);
        ev[r] = signed_count(__ldg(C + r * d.W + bucket_of(v, d.log2w)), v, d.log2w);
    }
    return T == 5 ? median5(ev[0], ev[1], ev[2], ev[3], ev[4]) : lower_median_dyn(ev, (int)rows);
}

// 1. distinct probe cells of each volume (grid.y = volume) with estimates
template <int T>
__global__ void k_bt_probe(const int32_t *__restrict__ C, const SketchDesc d, BatchTopkBufs b) {
    const uint32_t v = blockIdx.y;
    const BatchTopkVol V = b.vol[v];
    if (!V.use) return;
    const uint64_t mask = (1ull << b.set_log2) - 1;
    unsigned long long *set = b.set + ((uint64_t)v << b.set_log2);
    const uint64_t *probe = b.probe + (uint64_t)v * b.probe_per_vol;
    const int32_t *Cv = C + (uint64_t)v * d.rows * d.W;
    const uint32_t rows = T > 0 ? (uint32_t)T : d.rows;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V.m_probe; i += stride) {
        const uint64_t key = probe[i];
        if (key == kInvalidKey) continue;
        uint64_t h = table_hash(key) & mask;
        bool done = false;
        for (int p = 0; p < 4096 && !done; ++p) {
            // a plain read first: most probe keys repeat a cell already in the set
            unsigned long long prev = *reinterpret_cast<volatile unsigned long long *>(&set[h]);
            if (prev == kInvalidKey)
                prev = atomicCAS(&set[h], (unsigned long long)kInvalidKey, (unsigned long long)key);
            if (prev == kInvalidKey) {
                uint32_t cx, cy, cz;
                cell_of_key(key, V.G, cx, cy, cz);
                const uint32_t at = atomicAdd(&b.dcnt[v], 1u);
                b.dkey[(uint64_t)v * b.probe_per_vol + at] = key;
                b.dest[(uint64_t)v * b.probe_per_vol + at] = estimate<T>(Cv, d, rows, cx, cy, cz);
                done = true;
            } else if (prev == key) {
                done = true;
            } else {
                h = (h + 1) & mask;
            }
        }
        if (!done) atomicOr(&b.status[v], kSetFull);
    }
}

// 2. theta_v: the kk-th largest distinct-probe estimate (radix select over
// the order-preserving unsigned image u = est ^ 2^31, one byte a pass)
__global__ void __launch_bounds__(1024) k_bt_theta(BatchTopkBufs b) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_rem;
    const uint32_t v = blockIdx.x;
    const BatchTopkVol V = b.vol[v];
    if (!V.use) return;
    const uint32_t n = min(b.dcnt[v], (uint32_t)b.probe_per_vol);
    if (n < V.kk || b.status[v]) {
        if (threadIdx.x == 0) {
            b.theta[v] = INT32_MIN;
            atomicOr(&b.status[v], kProbeFull);
        }
        return;
    }
    const int32_t *est = b.dest + (uint64_t)v * b.probe_per_vol;
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_rem = V.kk;
    }
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix;
        const uint32_t himask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t u = (uint32_t)est[i] ^ 0x80000000u;
            if ((u & himask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {   // the digit holding the rem-th largest
            uint32_t above = 0, rem = s_rem;
            int dd = 255;
            for (; dd > 0; --dd) {
                if (above + hist[dd] >= rem) break;
                above += hist[dd];
            }
            s_rem = rem - above;
            s_prefix = prefix | ((uint32_t)dd << shift);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int32_t th = (int32_t)(s_prefix ^ 0x80000000u);
        b.theta[v] = th;
        if (th < 1) atomicOr(&b.status[v], kProbeFull);   // no pruning bound: the general path
    }
}

// 3. signed hot maps of every row of every volume (one warp a 32-bit word;
// W >= 32 so a word lies in one row): the positive map's bit is set when
// C >= theta_v, the negative map's when C <= -theta_v; a cell's signed count
// sign * C can reach theta_v only when the map of its sign bit has its bucket.
// bits: the positive maps of all volumes, then the negative maps.
__global__ void k_bt_bits(const int32_t *__restrict__ C, const SketchDesc d, BatchTopkBufs b,
                          uint64_t words) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t per_vol = (uint64_t)d.rows * (d.W >> 5);
    // four words a warp in flight
    for (uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w0 < words;
         w0 += 4 * warps) {
        int32_t c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t w = w0 + u * warps;
            c[u] = w < words ? __ldcs(C + w * 32 + lane) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t w = w0 + u * warps;
            if (w >= words) break;                               // warp-uniform
            const uint32_t v = (uint32_t)(w / per_vol);
            const bool live = b.vol[v].use && b.status[v] == 0;
            const int64_t x = c[u], th = b.theta[v];
            const unsigned pos = __ballot_sync(0xFFFFFFFFu, live && x >= th);
            const unsigned neg = __ballot_sync(0xFFFFFFFFu, live && x <= -th);
            if (lane == 0) {
                b.bits[w] = pos;
                b.bits[words + w] = neg;
            }
        }
    }
}

// 4. hot buckets of rows 0..F-1 of every volume
__global__ void k_bt_hot(const SketchDesc d, BatchTopkBufs b, uint64_t words) {
    const uint64_t wpr = d.W >> 5;
    const uint64_t all = (uint64_t)b.nvol * d.rows * wpr;       // words of one map
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * words; i += stride) {
        const uint32_t neg = i >= words;
        const uint64_t k = i - neg * words;
        const uint64_t vr = k / wpr, w = k - vr * wpr;   // vr = v * F + r
        const uint32_t v = (uint32_t)(vr / b.F), r = (uint32_t)(vr - (uint64_t)v * b.F);
        if (!b.vol[v].use || b.status[v]) continue;
        uint32_t x = b.bits[neg * all + ((uint64_t)v * d.rows + r) * wpr + w];
        if (!x) continue;
        uint32_t at = atomicAdd(&b.hot_cnt[vr], (uint32_t)__popc(x));
        uint32_t *list = b.hot + vr * b.hot_cap;
        while (x) {
            const int bit = __ffs(x) - 1;
            x &= x - 1;
            if (at < b.hot_cap) list[at] = ((uint32_t)(w * 32 + bit) << 1) | neg;   // bucket, sign bit
            ++at;
        }
    }
}

// Is row rr of the cell with row value val hot for its sign in volume v?
__device__ __forceinline__ bool bt_hot(const BatchTopkBufs &b, const SketchDesc &d, uint32_t v,
                                       uint32_t rr, uint64_t val) {
    const uint64_t wpr = d.W >> 5;
    const uint32_t bk = bucket_of(val, d.log2w);
    const uint64_t neg = (val >> (63 - d.log2w)) & 1ull;
    const uint64_t all = (uint64_t)b.nvol * d.rows * wpr;
    return (__ldg(b.bits + neg * all + ((uint64_t)v * d.rows + rr) * wpr + (bk >> 5)) >> (bk & 31)) & 1u;
}

// 5. each volume's search and the work of each (volume, row) pair, with its
// exclusive prefix (one block).  A volume is scanned (all G^3 cells, the
// work of its pair (v, 0)) when that is cheaper than its directory queries
// (one query of a (hot bucket, sign, cx) triple reads about
// 1 + G^2 / (2 W) + G^2 / 2^D lines; the model counts a whole bucket, G^2 / W)
// or when a row's hot pairs overflowed the list; otherwise every pair (v, r)
// has |hot (bucket, sign) pairs of row r| * G directory queries.
constexpr double kMaxBatchScan = 17179869184.0;   // 2^34 cells

__global__ void __launch_bounds__(1024) k_bt_prefix(BatchTopkBufs b, uint32_t log2w) {
    __shared__ unsigned long long warp_sum[32];
    __shared__ unsigned long long carry;
    const uint32_t n = b.nvol * b.F;
    for (uint32_t v = threadIdx.x; v < b.nvol; v += blockDim.x) {
        uint32_t sc = 0;
        if (b.vol[v].use && b.status[v] == 0) {
            // a query reads the lines of one bucket interval (G^2 / W) and
            // of the part of a slot on each side (G^2 / 2^D)
            const double G = b.vol[v].G;
            const double per_slot = G * G / (double)(1ull << b.vol[v].D) + G * G / (double)(1ull << log2w);
            double dir = 0;
            bool over = false;
            for (uint32_t r = 0; r < b.F; ++r) {
                const uint32_t c = b.hot_cnt[v * b.F + r];
                over |= c > b.hot_cap;
                dir += (double)c * G * (1.0 + per_slot);
            }
            const double scan = G * G * G;
            if (over || scan <= dir) {
                if (scan <= kMaxBatchScan) sc = 1;
                else b.status[v] |= kHotFull;
            }
        }
        b.scan[v] = sc;
    }
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        unsigned long long x = 0;
        if (i < n) {
            const uint32_t v = i / b.F, r = i - v * b.F;
            const uint64_t G = b.vol[v].G;
            if (b.vol[v].use && b.status[v] == 0)
                x = b.scan[v] ? (r == 0 ? G * G * G : 0ull) : (unsigned long long)b.hot_cnt[i] * G;
        }
        unsigned long long incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long sw = lane < (blockDim.x >> 5) ? warp_sum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, sw, o);
                if (lane >= (uint32_t)o) sw += y;
            }
            warp_sum[lane] = sw;
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? warp_sum[warp - 1] : 0) + incl - x;
        if (i < n) b.pre[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) b.pre[n] = carry;
}

// 6. the search of every volume in one persistent grid: a work item is a
// cell of a scanned volume, or a (row r < F, hot bucket, column cx) query of
// a volume's directory, whose cells are reported when r is their first hot
// row.  Either way every cell with estimate >= theta_v becomes a candidate.
template <int T>
__device__ __forceinline__ void bt_candidate(const int32_t *__restrict__ Cv, const SketchDesc &d,
                                             uint32_t rows, uint32_t v, uint32_t G, int32_t theta,
                                             uint32_t cx, uint32_t cy, uint32_t cz,
                                             const BatchTopkBufs &b) {
    const int32_t est = estimate<T>(Cv, d, rows, cx, cy, cz);
    if (est < theta) return;
    const uint32_t at = atomicAdd(&b.ccnt[v], 1u);
    if (at < b.cand_cap) {
        b.ckey[(uint64_t)v * b.cand_cap + at] = key_of(cx, cy, cz, G);
        b.cest[(uint64_t)v * b.cand_cap + at] = est;
    }
}

// A directory record of pair j (volume j / F, row j mod F) whose cell in
// column cx lies in its bucket: reported when row r is the cell's first hot
// row, at least `need` rows are hot and the estimate reaches theta_v.
template <int T>
__device__ __forceinline__ void bt_check(uint64_t cell, const int32_t *__restrict__ C,
                                         const SketchDesc &d, const BatchTopkBufs &b) {
    const uint32_t rows = T > 0 ? (uint32_t)T : d.rows;
    const uint32_t need = rows - (rows - 1) / 2;
    const uint32_t cx = (uint32_t)(cell & 0xFFFFu), cy = (uint32_t)((cell >> 16) & 0xFFFFu),
                   cz = (uint32_t)((cell >> 32) & 0xFFFFu), j = (uint32_t)(cell >> 48);
    const uint32_t v = j / b.F;
    const int r = (int)(j - v * b.F);
    // hot rows (for the cell's sign): r and rows after r (the rows before r
    // must be cold); the rows after r first, stopping once `need` is out of
    // reach, the rows before r last
    uint32_t nhot = 1, left = rows - 1 - (uint32_t)r;
    for (uint32_t rr = (uint32_t)r + 1; rr < rows; ++rr) {
        nhot += bt_hot(b, d, v, rr, row_value(d.seed[rr], cx, cy, cz));
        if (nhot + --left < need) return;
    }
    if (nhot < need) return;
    for (uint32_t rr = 0; rr < (uint32_t)r; ++rr)
        if (bt_hot(b, d, v, rr, row_value(d.seed[rr], cx, cy, cz))) return;
    bt_candidate<T>(C + (uint64_t)v * d.rows * d.W, d, rows, v, b.vol[v].G, b.theta[v], cx, cy, cz, b);
}

constexpr int kBtQueue = 64;   // per-warp queue of records to check

template <int T>
__global__ void __launch_bounds__(256, 5)   // 48 registers, 5 blocks an SM: faster than 6 or 4
    k_bt_query(const int32_t *__restrict__ C, const SketchDesc d, BatchTopkBufs b) {
    __shared__ uint64_t queue[8][kBtQueue];
    const uint32_t n = b.nvol * b.F;
    const uint64_t total = b.pre[n];
    const uint32_t rows = T > 0 ? (uint32_t)T : d.rows;
    const uint32_t need = rows - (rows - 1) / 2;
    const uint32_t s = 64 - d.log2w;
    const uint32_t lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t *qu = queue[threadIdx.x >> 5];
    uint32_t nq = 0;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5; q0 < total;
         q0 += warps << 5) {                                      // warp-uniform
        // the pair holding the warp's first item (the last j with pre[j] <= q0),
        // then upward per lane
        uint32_t j = 0;
        if (lane == 0) {
            uint32_t lo = 0, hi = n;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(b.pre + mid) <= q0) lo = mid; else hi = mid;
            }
            j = lo;
        }
        j = __shfl_sync(0xFFFFFFFFu, j, 0);
        const uint64_t q = q0 + lane;
        const bool item = q < total;
        if (item)
            while (j + 1 < n && __ldg(b.pre + j + 1) <= q) ++j;
        const uint32_t v = j / b.F;
        const int r = (int)(j - v * b.F);
        uint32_t e0 = 0, len = 0, cx = 0, h = 0, wrap = 0xFFFFFFFFu;
        uint64_t Tx = 0;
        const DirRecord *rec = nullptr;
        if (item) {
            const uint32_t G = b.vol[v].G;
            const uint64_t gm = b.vol[v].gmagic;
            const uint64_t local = q - __ldg(b.pre + j);
            if (b.scan[v]) {                 // one cell of a scanned volume: checked here
                const uint64_t rest = div_invariant(local, G, gm), cz = div_invariant(rest, G, gm);
                const uint32_t ccx = (uint32_t)(local - rest * G), cy = (uint32_t)(rest - cz * G);
                uint32_t nhot = 0, left = rows;
                bool skip = false;
                for (uint32_t rr = 0; rr < rows; ++rr) {
                    nhot += bt_hot(b, d, v, rr, row_value(d.seed[rr], ccx, cy, (uint32_t)cz));
                    if (nhot + --left < need) { skip = true; break; }
                }
                if (!skip)
                    bt_candidate<T>(C + (uint64_t)v * d.rows * d.W, d, rows, v, G, b.theta[v], ccx, cy,
                                    (uint32_t)cz, b);
            } else {                         // a (hot bucket, column) query: its run of records
                const uint64_t hi = div_invariant(local, G, gm);      // local = hi G + cx
                h = __ldg(b.hot + (uint64_t)j * b.hot_cap + hi);
                cx = (uint32_t)(local - hi * G);
                const uint32_t *off = b.dir_off[j];
                rec = b.dir_rec[j];
                const uint32_t D = b.vol[v].D;
                Tx = d.seed[r].a0 * (uint64_t)cx;
                // h = bucket << 1 | sign bit: lines with L in [h 2^(s-1) - Tx,
                // (h+1) 2^(s-1) - Tx), the records of slots a .. z, contiguous
                // in the counting-sorted array (a run that wraps past the last
                // slot continues at record 0: index e0 + k taken modulo `wrap`)
                const uint64_t lo = ((uint64_t)h << (s - 1)) - Tx;
                const uint64_t a = lo >> (64 - D), z = (lo + ((1ull << (s - 1)) - 1)) >> (64 - D);
                e0 = __ldg(off + a);
                const uint32_t ez = __ldg(off + z + 1);
                const uint32_t nrec = __ldg(off + (1ull << D));
                len = a <= z ? ez - e0 : (nrec - e0) + ez;
                if (a > z) wrap = nrec;
            }
        }
        // the warp walks the longest run; in-bucket records are queued and
        // checked 32 at a time
        uint32_t most = len;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) most = max(most, __shfl_xor_sync(0xFFFFFFFFu, most, o));
        for (uint32_t k = 0; k < most; k += 4) {
            DirRecord p[4];                  // four records loaded before any is checked
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                uint32_t idx = e0 + k + u;
                if (idx >= wrap) idx -= wrap;
                p[u] = k + u < len ? __ldg(rec + idx) : 0u;
            }
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                bool take = false;
                uint64_t cell = 0;
                if (k + u < len) {
                    const uint32_t cy = p[u] & 0xFFFFu, cz = p[u] >> 16;
                    take = ((line_value(d.seed[r], cy, cz) + Tx) >> (s - 1)) == h;
                    cell = (uint64_t)cx | ((uint64_t)cy << 16) | ((uint64_t)cz << 32) |
                           ((uint64_t)j << 48);
                }
                const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
                if (take) qu[nq + __popc(m & lt)] = cell;
                nq += __popc(m);
                if (nq >= 32) {
                    __syncwarp();
                    bt_check<T>(qu[lane], C, d, b);
                    __syncwarp();
                    if (lane < nq - 32) qu[lane] = qu[32 + lane];
                    nq -= 32;
                    __syncwarp();
                }
            }
        }
    }
    __syncwarp();
    if (lane < nq) bt_check<T>(qu[lane], C, d, b);
}

// 7. the kk best candidates of each volume in rank order, one block a
// volume: the kk-th best (estimate desc, key asc) by a radix select on the
// estimate, then on the key among the estimate's ties; the kk entries ranked
// at or above it gathered in shared memory and sorted (bitonic, next power of
// two >= kk).
__device__ __forceinline__ bool ranks_before(int32_t ea, uint64_t ka, int32_t eb, uint64_t kb) {
    return ea > eb || (ea == eb && ka < kb);
}

// The rank-th (1-based) largest (LARGEST) or smallest value among the
// participating get(i) of i < n, one byte a pass from bit top_shift + 7 down.
template <bool LARGEST, typename Get>
__device__ uint64_t block_select(uint32_t n, uint32_t rank, int top_shift, Get get, uint32_t *hist,
                                 unsigned long long *sh) {
    if (threadIdx.x == 0) {
        sh[0] = 0;      // decided digits
        sh[1] = rank;   // rank still to find among the entries matching them
    }
    for (int shift = top_shift; shift >= 0; shift -= 8) {
        for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t prefix = sh[0];
        const uint64_t himask = shift >= 56 ? 0ull : (~0ull << (shift + 8));
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            bool in = false;
            const uint64_t x = get(i, in);
            if (in && (x & himask) == prefix) atomicAdd(&hist[(x >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t before = 0, rem = sh[1];
            int dd = LARGEST ? 255 : 0;
            for (int step = 0; step < 255; ++step, dd += LARGEST ? -1 : 1) {
                if (before + hist[dd] >= rem) break;
                before += hist[dd];
            }
            sh[1] = rem - before;
            sh[0] = prefix | ((uint64_t)dd << shift);
        }
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(1024) k_bt_final(BatchTopkBufs b, uint32_t sort_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t hist[256];
    __shared__ unsigned long long sh[2];
    __shared__ uint32_t s_above, s_at;
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem);
    int32_t *se = reinterpret_cast<int32_t *>(sk + sort_cap);
    const uint32_t v = blockIdx.x;
    const BatchTopkVol V = b.vol[v];
    const uint32_t m = b.ccnt[v];
    if (!V.use || b.status[v] || m > b.cand_cap || m < V.kk || V.kk > sort_cap) {
        if (threadIdx.x == 0) {
            b.on[v] = 0;
            if (V.use && !b.status[v]) b.status[v] = kCandFull;
        }
        return;
    }
    const uint64_t *ck = b.ckey + (uint64_t)v * b.cand_cap;
    const int32_t *ce = b.cest + (uint64_t)v * b.cand_cap;
    // the kk-th largest estimate (order-preserving unsigned image)
    const uint32_t ue = (uint32_t)block_select<true>(
        m, V.kk, 24, [&](uint32_t i, bool &in) { in = true; return (uint64_t)((uint32_t)ce[i] ^ 0x80000000u); },
        hist, sh);
    if (threadIdx.x == 0) {
        s_above = 0;
        s_at = 0;
    }
    __syncthreads();
    uint32_t above = 0;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) above += ((uint32_t)ce[i] ^ 0x80000000u) > ue;
    atomicAdd(&s_above, above);
    __syncthreads();
    // among the estimate's ties, the (kk - above)-th smallest key
    const uint64_t cells = (uint64_t)V.G * V.G * V.G;
    const int kbits = 64 - __clzll((long long)(cells > 1 ? cells - 1 : 1));
    const uint64_t kth_key = block_select<false>(
        m, V.kk - s_above, ((kbits + 7) / 8 - 1) * 8,
        [&](uint32_t i, bool &in) {
            in = ((uint32_t)ce[i] ^ 0x80000000u) == ue;
            return ck[i];
        },
        hist, sh);
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
        const uint32_t u = (uint32_t)ce[i] ^ 0x80000000u;
        if (u > ue || (u == ue && ck[i] <= kth_key)) {
            const uint32_t at = atomicAdd(&s_at, 1u);
            if (at < sort_cap) {
                sk[at] = ck[i];
                se[at] = ce[i];
            }
        }
    }
    __syncthreads();
    uint32_t N = 1;
    while (N < V.kk) N <<= 1;
    for (uint32_t i = V.kk + threadIdx.x; i < N; i += blockDim.x) {
        sk[i] = kInvalidKey;
        se[i] = INT32_MIN;
    }
    __syncthreads();
    for (uint32_t k = 2; k <= N; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;   // this run in rank order
                    const bool later = ranks_before(se[l], sk[l], se[i], sk[i]);
                    if (later == up) {
                        const uint64_t tk = sk[i];
                        sk[i] = sk[l];
                        sk[l] = tk;
                        const int32_t te = se[i];
                        se[i] = se[l];
                        se[l] = te;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t i = threadIdx.x; i < V.kk; i += blockDim.x) {
        b.okey[(uint64_t)v * b.k + i] = sk[i];
        b.oest[(uint64_t)v * b.k + i] = se[i];
    }
    if (threadIdx.x == 0) b.on[v] = s_at == V.kk ? V.kk : 0u;   // exactly kk gathered
    if (threadIdx.x == 0 && s_at != V.kk) b.status[v] = kCandFull;
}

}  // namespace

// shared memory of the final step: a sort buffer of the next power of two >= k
size_t batch_topk_final_smem(uint32_t k) {
    size_t n = 1;
    while (n < k) n <<= 1;
    return n * 12;
}

cudaError_t launch_batch_topk(const int32_t *C, const SketchDesc &d, const BatchTopkBufs &b,
                              int num_sms, cudaStream_t s, int *launches) {
    if (d.W < 32 || b.F == 0 || b.nvol == 0 || b.k == 0 || b.k > 4096) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.set, 0xFF, ((size_t)b.nvol << b.set_log2) * 8, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.dcnt, 0, b.nvol * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.status, 0, b.nvol * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.hot_cnt, 0, (size_t)b.nvol * b.F * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.ccnt, 0, b.nvol * 4, s)) != cudaSuccess) return e;
    const uint32_t px = (uint32_t)std::min<uint64_t>((b.probe_per_vol + 255) / 256, 64);
    if (d.rows == 5) k_bt_probe<5><<<dim3(px, b.nvol), 256, 0, s>>>(C, d, b);
    else k_bt_probe<0><<<dim3(px, b.nvol), 256, 0, s>>>(C, d, b);
    k_bt_theta<<<b.nvol, 1024, 0, s>>>(b);
    const uint64_t words = (uint64_t)b.nvol * d.rows * (d.W >> 5);
    k_bt_bits<<<num_sms * 8, 256, 0, s>>>(C, d, b, words);
    const uint64_t hwords = (uint64_t)b.nvol * b.F * (d.W >> 5);
    k_bt_hot<<<(unsigned)std::min<uint64_t>((hwords + 255) / 256, (uint64_t)num_sms * 8), 256, 0, s>>>(d, b, hwords);
    k_bt_prefix<<<1, 1024, 0, s>>>(b, d.log2w);
    if (d.rows == 5) k_bt_query<5><<<num_sms * 16, 256, 0, s>>>(C, d, b);
    else k_bt_query<0><<<num_sms * 16, 256, 0, s>>>(C, d, b);
    const size_t smem = batch_topk_final_smem(b.k);
    if ((e = ensure_smem_limit(k_bt_final, smem)) != cudaSuccess) return e;
    k_bt_final<<<b.nvol, 1024, smem, s>>>(b, (uint32_t)(smem / 12));
    *launches += 7;
    return cudaGetLastError();
}

}  // namespace hs
