// capi_noalloc.cu - sketch_query_noalloc (see the comment below).
#include <mutex>

#include "capi_internal.h"

// ---------------------------------------------------------------------------
// sketch_query_noalloc: point queries without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they query: processes
// whose device memory is fully reserved by another allocator or held to a
// fixed budget, and query loops that must not pay for an allocation (a
// cudaMalloc may synchronise the device).  sketch_query may allocate staging
// buffers on its first call with host arrays; this variant instead uses one
// file-scope device array, sized for at most HS_NOALLOC_QUERY_MAX keys, that
// every GPU loading this library holds until the process exits.  The call is
// synchronous (it waits for the handle's stream to read back the bad-key
// flag), so it is not for code whose stream is being captured into a graph.
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
    // the same estimate kernel as sketch_query, on the static scratch
    HS_CUDA(launch_point_query(h->C, h->d, dk, m, de, s_flag, h->stream));
    h->stats.kernel_launches += 1;
    if (!ed) HS_CUDA(cudaMemcpyAsync(est, de, m * 4, cudaMemcpyDeviceToHost, h->stream));
    uint32_t bad = 0;
    HS_CUDA(cudaMemcpyAsync(&bad, s_flag, 4, cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    drain_timings(h);
    if (bad) return fail(HS_ERR_ARG, "a key is >= G^3 = %llu", (unsigned long long)h->n_cells);
    return HS_OK;
}
