// capi_noalloc.cu - sketch_query_noalloc (see the comment below).
#include <mutex>

#include "capi_internal.h"

// ---------------------------------------------------------------------------
// sketch_query_noalloc: point queries without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they query: code running
// while a CUDA stream is being captured into a graph (allocation is not a
// capturable operation), processes whose device memory is fully reserved by
// another allocator or a fixed budget, and latency-critical loops where an
// allocation's synchronisation is not acceptable.  sketch_query may allocate
// staging buffers on its first call with host arrays; this variant instead
// uses one file-scope device array, sized for at most
// HS_NOALLOC_QUERY_MAX keys, that every GPU loading this library holds until
// the process exits.
// ---------------------------------------------------------------------------

namespace {

constexpr uint64_t kNoallocMax = HS_NOALLOC_QUERY_MAX;
constexpr size_t kNoallocKeysOff = 0;
constexpr size_t kNoallocEstOff = kNoallocMax * 8;
constexpr size_t kNoallocFlagOff = kNoallocMax * 12;
constexpr size_t kNoallocBytes = kNoallocMax * 12 + 256;
constexpr int kNoallocMaxDevices = 64;

// keys staging | estimates staging | out-of-range flag; shared by every call
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).  The
// host-side name g_noalloc_scratch is only a stand-in, never a device address.
hs_status noalloc_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(HS_ERR_ARG, "device %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(HS_ERR_CUDA, "cudaGetSymbolAddress of the query scratch failed: %s",
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return HS_OK;
}

// Estimate (Sec. 2.2) of each key; keys >= G^3 give 0 and set *bad.
__global__ void k_point_query_noalloc(const int32_t *__restrict__ C, const SketchDesc d,
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
        uint32_t cy = (uint32_t)(rest % d.G), cz = (uint32_t)(rest / d.G);
        int32_t ev[kMaxRows];
        for (uint32_t r = 0; r < d.rows; ++r) {
            uint64_t v = row_value(d.seed[r], cx, cy, cz);
            ev[r] = signed_count(C[r * d.W + bucket_of(v, d.log2w)], v, d.log2w);
        }
        est[i] = d.rows == 5 ? median5(ev[0], ev[1], ev[2], ev[3], ev[4])
                             : lower_median_dyn(ev, (int)d.rows);
    }
}

}  // namespace

extern "C" hs_status sketch_query_noalloc(hs_sketch *h, const uint64_t *keys, uint64_t m,
                                          int32_t *est) {
    if (!h) return fail(HS_ERR_ARG, "handle is NULL");
    if (m == 0) return HS_OK;
    if (!keys || !est) return fail(HS_ERR_ARG, "keys/est is NULL");
    if (m > kNoallocMax)
        return fail(HS_ERR_ARG, "m=%llu exceeds HS_NOALLOC_QUERY_MAX=%llu; split the query",
                    (unsigned long long)m, (unsigned long long)kNoallocMax);
    int dev = -1;
    HS_CUDA(cudaGetDevice(&dev));
    if (dev != h->device)
        return fail(HS_ERR_STATE, "make the sketch's device %d current (current: %d)", h->device,
                    dev);
    unsigned char *scratch = nullptr;
    hs_status st = noalloc_scratch(dev, &scratch);
    if (st != HS_OK) return st;
    st = drain(h);   // pending binned increments use buffers that already exist
    if (st != HS_OK) return st;
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(scratch + kNoallocKeysOff);
    int32_t *s_est = reinterpret_cast<int32_t *>(scratch + kNoallocEstOff);
    uint32_t *s_flag = reinterpret_cast<uint32_t *>(scratch + kNoallocFlagOff);
    const bool kd = is_device_ptr(keys), ed = is_device_ptr(est);
    const uint64_t *dk = keys;
    int32_t *de = ed ? est : s_est;
    if (!kd) {
        HS_CUDA(cudaMemcpyAsync(s_keys, keys, m * 8, cudaMemcpyHostToDevice, h->stream));
        dk = s_keys;
    }
    HS_CUDA(cudaMemsetAsync(s_flag, 0, 4, h->stream));   // the previous call's flag stays otherwise
    uint64_t blocks = std::min<uint64_t>((m + 255) / 256, 65535);
    k_point_query_noalloc<<<(unsigned)blocks, 256, 0, h->stream>>>(h->C, h->d, dk, m, de, s_flag);
    HS_CUDA(cudaGetLastError());
    h->stats.kernel_launches += 1;
    if (!ed) HS_CUDA(cudaMemcpyAsync(est, de, m * 4, cudaMemcpyDeviceToHost, h->stream));
    uint32_t bad = 0;
    HS_CUDA(cudaMemcpyAsync(&bad, s_flag, 4, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    if (bad) return fail(HS_ERR_ARG, "a key is >= G^3 = %llu", (unsigned long long)h->n_cells);
    return HS_OK;
}
