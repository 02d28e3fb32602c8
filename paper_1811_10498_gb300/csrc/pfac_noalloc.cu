// Allocation-free variant of the packed scan (pfac_match_packed_noalloc in pfac.h).
//
// The ordinary scan keeps its deferred long walks in scratch that the library
// allocates per stream. Here that scratch is one fixed array compiled into the
// library, so a call allocates no device memory at all: for callers under a fixed
// device-memory budget, callers whose device memory belongs to another allocator,
// and latency-sensitive callers that must not meet the device-wide synchronisation
// of cudaMalloc/cudaFree. Every GPU that loads the library holds the array until the
// process exits; all calls share it, so calls that overlap on the GPU race on it.
#include <stdint.h>

#include <mutex>

#include <cuda_runtime.h>

#include "../../include/pfac.h"
#include "pfac_internal.h"

namespace {

constexpr int64_t kItems = int64_t(1) << 18;        // deferred walks the array holds
constexpr int64_t kMaxBases = kItems * 256;          // longest text a call accepts (2^26)
constexpr size_t kHeader = 256;                      // the deferred-walk counter

// Deferred-walk scratch: a counter, then kItems records. In host code this name is
// only a stand-in for the symbol, never a device address: the device address comes
// from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeader + kItems * pfac::kDeferItemBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];

// Device address of the array on the current device, looked up once per device (the
// first call on a device does it; it should come before any stream capture).
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pfac::set_last_cuda_error(e);
    if (dev < 0 || dev >= kMaxDevices) return pfac::set_last_error(PFAC_ERR_UNSUPPORTED);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return pfac::set_last_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PFAC_OK;
}

}  // namespace

extern "C" int pfac_match_packed_noalloc(pfac_handle h, const uint32_t *d_packed, int64_t n_bases,
                                         int32_t *d_out_ids, void *stream)
{
    if (n_bases > kMaxBases) return pfac::set_last_error(PFAC_ERR_SCRATCH_LIMIT);
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != PFAC_OK) return rc;
    pfac::DeferScratch scratch{};
    scratch.count = (unsigned long long *)base;          // zeroed by every launch
    scratch.items = (unsigned char *)base + kHeader;
    scratch.cap = kItems;
    return pfac::scan_packed_with_scratch(h, d_packed, n_bases, d_out_ids, scratch, (cudaStream_t)stream);
}
