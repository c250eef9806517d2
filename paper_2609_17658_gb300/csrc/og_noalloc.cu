// og_noalloc.cu -- a Morton-key sort that performs no device memory allocation.
//
// Why it exists: some callers of this library cannot allocate device memory
// at the moment they need a sort.  A serving process that has committed its
// whole HBM budget to resident trees must not grow its footprint, and a
// latency-critical loop cannot afford cudaMalloc / cudaFree, which can
// synchronise the whole device.  og_sort_keys_noalloc therefore sorts keys
// in a fixed scratch area that belongs to the library's device code instead
// of allocating per call.
//
// The scratch is one file-scope static __device__ array (size below).  Every
// GPU that loads the library's device code holds it until the process exits.
// With CUDA's lazy module loading that can happen at the first call on a
// device (inside its cudaGetSymbolAddress), and if the device has no room
// left then, that first call fails with OG_ERR_CUDA: a caller that is about
// to commit its whole budget makes one call first, at set-up.  Host code
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

// true iff p is device (or managed) memory of device dev
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

// byte ranges [a, a + na) and [b, b + nb) share at least one byte
bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

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
    if (!on_device(keys_in, dev) || !on_device(keys_out, dev) || !on_device(perm_out, dev)) {
        set_error("og_sort_keys_noalloc: keys_in, keys_out and perm_out must be device memory "
                  "of the current device (%d)", dev);
        return OG_ERR_ARG;
    }
    const size_t kb = (size_t)n * sizeof(uint64_t), pb = (size_t)n * sizeof(uint32_t);
    if ((keys_out != keys_in && overlap(keys_in, kb, keys_out, kb)) ||
        overlap(perm_out, pb, keys_in, kb) || overlap(perm_out, pb, keys_out, kb)) {
        set_error("og_sort_keys_noalloc: buffers overlap (keys_out may equal keys_in; no other "
                  "overlap is allowed)");
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
