// og_noalloc.cu -- a Morton-key sort that performs no device memory allocation.
//
// Why it exists: some callers of this library cannot allocate device memory
// at the moment they need a sort.  A serving process that has committed its
// whole HBM budget to resident trees must not grow its footprint, and a
// latency-critical loop cannot afford cudaMalloc / cudaFree, which can
// synchronise the whole device.  og_sort_keys_noalloc therefore sorts keys
// with a fixed scratch area that is reserved once, when the library is
// loaded, instead of allocating per call.
//
// The scratch is one file-scope static __device__ array (size below).  Every
// GPU that loads the library holds it until the process exits.  Host code
// must not use the array's name as a device address (in host code that name
// refers to a host-side stand-in); the device address is obtained once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call on that device, and cached.
#include <mutex>

#include "og_internal.h"

namespace og {
namespace {

constexpr int64_t kNoAllocMaxN = OG_NOALLOC_MAX_N;
// alternate key buffer, alternate index buffer, then the digit counts and
// scan scratch of the radix sort
constexpr size_t kAltKeysBytes = (size_t)kNoAllocMaxN * sizeof(uint64_t);
constexpr size_t kAltValsBytes = (size_t)kNoAllocMaxN * sizeof(uint32_t);
constexpr size_t kSortScratchBytes = (size_t)4 << 20;  // >= radix_sort_scratch_bytes(max N)
constexpr size_t kScratchBytes = kAltKeysBytes + kAltValsBytes + kSortScratchBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

__global__ void k_iota(int64_t n, uint32_t *v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

}  // namespace
}  // namespace og

using namespace og;

extern "C" og_status og_sort_keys_noalloc(const uint64_t *keys_in, uint64_t *keys_out,
                                          uint32_t *perm_out, int64_t n, void *stream) {
    if (!keys_in || !keys_out || !perm_out) {
        set_error("og_sort_keys_noalloc: NULL pointer");
        return OG_ERR_ARG;
    }
    if (n < 1 || n > kNoAllocMaxN) {
        set_error("og_sort_keys_noalloc: n = %lld outside [1, %lld] (the fixed scratch holds at "
                  "most OG_NOALLOC_MAX_N keys)",
                  (long long)n, (long long)kNoAllocMaxN);
        return OG_ERR_ARG;
    }
    if (radix_sort_scratch_bytes(kNoAllocMaxN) > kSortScratchBytes) {
        set_error("og_sort_keys_noalloc: internal scratch layout too small");
        return OG_ERR_STATE;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "og_sort_keys_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("og_sort_keys_noalloc: device index %d not supported", dev);
        return OG_ERR_ARG;
    }
    void *base = nullptr;
    {
        // once per device, with that device current: the device address of
        // the static scratch array
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                 "og_sort_keys_noalloc: cudaGetSymbolAddress");
            g_scratch_addr[dev] = ptr;
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *sc = static_cast<char *>(base);
    uint64_t *keys_alt = reinterpret_cast<uint64_t *>(sc);
    uint32_t *vals_alt = reinterpret_cast<uint32_t *>(sc + kAltKeysBytes);
    void *sort_scratch = sc + kAltKeysBytes + kAltValsBytes;
    // the scratch keeps no state between calls: every pass rewrites the digit
    // counts and the alternate buffers before reading them
    if (keys_out != keys_in) {
        e = cudaMemcpyAsync(keys_out, keys_in, (size_t)n * sizeof(uint64_t),
                            cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "og_sort_keys_noalloc: copy");
    }
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, perm_out); note_launch();
    // 63-bit keys: eight 8-bit passes, an even count, so the result ends in
    // keys_out / perm_out
    radix_sort_pairs_every_pass(keys_out, perm_out, keys_alt, vals_alt, n, 64, sort_scratch, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "og_sort_keys_noalloc: launch");
    return OG_OK;
}
