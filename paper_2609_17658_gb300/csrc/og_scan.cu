// og_scan.cu -- device-wide prefix scans (tile reduce, then a downsweep in which
// every tile adds up the totals of the tiles before it; short scans in one
// kernel with a decoupled look-back).
//
// Tiles of 4096 elements: 512 threads x 8 consecutive items, staged through
// shared memory so that global loads and stores stay coalesced.  Used for the
// node ids of the first splits, the child offsets, the run starts (a maximum
// scan), the group starts (a compaction) and the sort's tile counts.
#include "og_internal.h"

namespace og {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

struct OpSum {
    static __device__ __forceinline__ uint32_t id() { return 0u; }
    static __device__ __forceinline__ uint32_t op(uint32_t a, uint32_t b) { return a + b; }
};
struct OpMax {
    static __device__ __forceinline__ uint32_t id() { return 0u; }
    static __device__ __forceinline__ uint32_t op(uint32_t a, uint32_t b) { return a > b ? a : b; }
};

template <class Op>
__device__ __forceinline__ uint32_t warp_inclusive(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v = Op::op(o, v);
    }
    return v;
}

// Block-wide scan of one value per thread.  Returns the exclusive prefix,
// writes the block total to *total.  s_warp holds 32 words.
template <class Op>
__device__ uint32_t block_exclusive(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t inc = warp_inclusive<Op>(v);
    uint32_t exc_in_warp = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc_in_warp = Op::id();
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nwarps ? s_warp[lane] : Op::id();
        uint32_t wi = warp_inclusive<Op>(w);
        if (lane < nwarps) s_warp[lane] = wi;
    }
    __syncthreads();
    uint32_t warp_pre = warp > 0 ? s_warp[warp - 1] : Op::id();
    *total = s_warp[nwarps - 1];
    __syncthreads();
    return Op::op(warp_pre, exc_in_warp);
}

template <class Op>
__global__ void __launch_bounds__(kScanThreads) k_tile_reduce(const uint32_t *__restrict__ in,
                                                               int64_t n, uint32_t *tile_tot) {
    pdl_wait();
    __shared__ uint32_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t acc = Op::id();
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) acc = Op::op(acc, in[i]);
    }
    uint32_t tot;
    block_exclusive<Op>(acc, s_warp, &tot);
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = tot;
}

template <class Op, bool kExclusive>
__global__ void __launch_bounds__(kScanThreads) k_tile_downsweep(const uint32_t *__restrict__ in,
                                                                  uint32_t *out, int64_t n,
                                                                  const uint32_t *tile_tot,
                                                                  uint32_t *d_total, uint32_t *compact) {
    pdl_wait();
    __shared__ uint32_t s_items[kScanTile];
    __shared__ uint32_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t pre = Op::id();
    for (int64_t t = threadIdx.x; t < (int64_t)blockIdx.x; t += kScanThreads)
        pre = Op::op(pre, tile_tot[t]);
    uint32_t tile_pre;
    block_exclusive<Op>(pre, s_warp, &tile_pre);
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        s_items[k * kScanThreads + threadIdx.x] = i < n ? in[i] : Op::id();
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t acc = Op::id();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = s_items[threadIdx.x * kScanItems + k];
        acc = Op::op(acc, v[k]);
    }
    uint32_t tot;
    uint32_t r = Op::op(tile_pre, block_exclusive<Op>(acc, s_warp, &tot));
    if (d_total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *d_total = Op::op(tile_pre, tot);
    if (compact) {
        // compaction: flagged item i goes to slot (exclusive prefix of i)
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (v[k]) compact[r] = (uint32_t)(base + (int64_t)threadIdx.x * kScanItems + k);
            r = Op::op(r, v[k]);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (kExclusive) {
            s_items[threadIdx.x * kScanItems + k] = r;
            r = Op::op(r, v[k]);
        } else {
            r = Op::op(r, v[k]);
            s_items[threadIdx.x * kScanItems + k] = r;
        }
    }
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = s_items[k * kScanThreads + threadIdx.x];
    }
}

// The same scan in one kernel: tiles numbered in the order their blocks
// start publish their totals, and warp 0 of each tile gathers the totals of
// the tiles before it, 32 at a time, until it meets an inclusive one
// (decoupled look-back).  A look word: flag (2 bits: 1 own total, 2
// inclusive), the use's tag (bits 32..61), the value (low 32 bits); a word
// of another tag reads as not yet published, so one clearing serves
// successive uses with distinct tags.  Every wait is bounded.
constexpr unsigned long long kScanOwn = 1ull << 62, kScanInc = 2ull << 62;
constexpr int kScanSpinLimit = 1 << 20;
// above this many tiles the look-back's waits cost more than the second
// launch they save: the two-kernel scan runs instead
constexpr int64_t kScanLookMaxTiles = 64;

__device__ __forceinline__ void st_word(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <class Op>
__device__ __forceinline__ uint32_t warp_fold(uint32_t v);
template <>
__device__ __forceinline__ uint32_t warp_fold<OpSum>(uint32_t v) { return __reduce_add_sync(0xffffffffu, v); }
template <>
__device__ __forceinline__ uint32_t warp_fold<OpMax>(uint32_t v) { return __reduce_max_sync(0xffffffffu, v); }

template <class Op, bool kExclusive>
__global__ void __launch_bounds__(kScanThreads) k_scan_look(const uint32_t *in, uint32_t *out, int64_t n,
                                                            unsigned long long *look, uint32_t *ctr,
                                                            unsigned long long tag, uint32_t *d_total,
                                                            uint32_t *compact, uint32_t *status) {
    pdl_wait();
    __shared__ uint32_t s_items[kScanTile];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_tile, s_pre;
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        s_items[k * kScanThreads + threadIdx.x] = i < n ? in[i] : Op::id();
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t acc = Op::id();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = s_items[threadIdx.x * kScanItems + k];
        acc = Op::op(acc, v[k]);
    }
    uint32_t tot;
    uint32_t r = block_exclusive<Op>(acc, s_warp, &tot);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned long long tg = tag << 32;
        const unsigned long long tmask = 0x3fffffffull << 32;
        uint32_t pre = Op::id();
        if (tile == 0) {
            if (lane == 0) st_word(&look[0], kScanInc | tg | tot);
        } else {
            if (lane == 0) st_word(&look[tile], kScanOwn | tg | tot);
            int64_t j = tile - 1;
            int spins = 0;
            while (true) {
                const int64_t q = j - lane;
                // before the first tile: an inclusive identity
                const unsigned long long w = q >= 0 ? ld_word(&look[q]) : (kScanInc | tg | Op::id());
                const bool ready = (w & tmask) == tg && (w >> 62) != 0ull;
                const unsigned notready = __ballot_sync(0xffffffffu, !ready);
                const unsigned inc = __ballot_sync(0xffffffffu, ready && (w >> 62) == 2ull);
                const int L = inc ? __ffs(inc) - 1 : 32;        // nearest inclusive word
                const unsigned need = L == 32 ? 0xffffffffu : ((2u << L) - 1u);
                if (notready & need) {
                    if (++spins > kScanSpinLimit) {  // a tile that never publishes: give up
                        if (lane == 0) atomicOr(status, ST_TIMEOUT);
                        break;
                    }
                    if (spins > 32) __nanosleep(32);
                    continue;
                }
                pre = Op::op(pre, warp_fold<Op>(lane <= L ? (uint32_t)w : Op::id()));
                if (L < 32) break;
                j -= 32;
            }
            if (lane == 0) st_word(&look[tile], kScanInc | tg | Op::op(pre, tot));
        }
        if (lane == 0) s_pre = pre;
    }
    __syncthreads();
    const uint32_t tile_pre = s_pre;
    r = Op::op(tile_pre, r);
    if (d_total && threadIdx.x == 0 && base + kScanTile >= n) *d_total = Op::op(tile_pre, tot);
    if (compact) {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (v[k]) compact[r] = (uint32_t)(base + (int64_t)threadIdx.x * kScanItems + k);
            r = Op::op(r, v[k]);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (kExclusive) {
            s_items[threadIdx.x * kScanItems + k] = r;
            r = Op::op(r, v[k]);
        } else {
            r = Op::op(r, v[k]);
            s_items[threadIdx.x * kScanItems + k] = r;
        }
    }
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = s_items[k * kScanThreads + threadIdx.x];
    }
}

template <class Op, bool kExclusive>
void scan_impl(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total, void *scratch,
               cudaStream_t s, uint32_t *compact = nullptr) {
    if (n <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s);
        return;
    }
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    uint32_t *tile = static_cast<uint32_t *>(scratch);
    if (ntiles > 1) {
        launch_pdl(k_tile_reduce<Op>, (unsigned)ntiles, kScanThreads, 0, s, in, n, tile);
    }
    launch_pdl(k_tile_downsweep<Op, kExclusive>, (unsigned)ntiles, kScanThreads, 0, s, in, out, n, tile,
                                                                             d_total, compact);
}

}  // namespace

size_t scan_look_words(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile); }

void scan_exclusive_u32_look(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total,
                             unsigned long long *look, uint32_t *ctr, uint32_t tag, uint32_t *status,
                             void *scratch, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s);
        return;
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > kScanLookMaxTiles) {
        scan_impl<OpSum, true>(in, out, n, d_total, scratch, s);
        return;
    }
    launch_pdl(k_scan_look<OpSum, true>, (unsigned)ntiles, kScanThreads, 0, s, in, out, n, look, ctr,
               (unsigned long long)tag, d_total, (uint32_t *)nullptr, status);
}

void scan_compact_u32_look(const uint32_t *flags, uint32_t *idx, int64_t n, uint32_t *d_total,
                           unsigned long long *look, uint32_t *ctr, uint32_t tag, uint32_t *status, void *scratch,
                           cudaStream_t s) {
    if (n <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s);
        return;
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > kScanLookMaxTiles) {
        scan_impl<OpSum, true>(flags, nullptr, n, d_total, scratch, s, idx);
        return;
    }
    launch_pdl(k_scan_look<OpSum, true>, (unsigned)ntiles, kScanThreads, 0, s, flags, (uint32_t *)nullptr, n, look,
               ctr, (unsigned long long)tag, d_total, idx, status);
}

void scan_inclusive_max_u32_look(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *look,
                                 uint32_t *ctr, uint32_t tag, uint32_t *status, void *scratch,
                                 cudaStream_t s) {
    if (n <= 0) return;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > kScanLookMaxTiles) {
        scan_impl<OpMax, false>(in, out, n, nullptr, scratch, s);
        return;
    }
    launch_pdl(k_scan_look<OpMax, false>, (unsigned)ntiles, kScanThreads, 0, s, in, out, n, look, ctr,
               (unsigned long long)tag, (uint32_t *)nullptr, (uint32_t *)nullptr, status);
}

og_status scan_wait_timeout_probe(og_ctx *c, int64_t n) {
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles < 2 || ntiles > kScanLookMaxTiles) {
        set_error("og_debug_scan_wait_timeout: n must span 2 to %lld tiles of %d", (long long)kScanLookMaxTiles,
                  kScanTile);
        return OG_ERR_ARG;
    }
    cudaStream_t s = c->stream;
    const size_t bytes = (size_t)n * 2 * sizeof(uint32_t) + (size_t)ntiles * 8 + 512;
    void *buf = nullptr;
    cudaError_t e = dev_malloc_async(&buf, bytes, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? OG_ERR_OOM : cuda_fail(e, "cudaMallocAsync (probe)");
    unsigned long long *look = static_cast<unsigned long long *>(buf);   // ntiles words, all 0
    uint32_t *ctr = reinterpret_cast<uint32_t *>(look + ntiles);
    uint32_t *in = ctr + 32;
    uint32_t *out = in + n;
    cudaMemsetAsync(buf, 0, bytes, s);
    // the tile counter starts at 1 and the grid has one block fewer than
    // tiles: tile 0 is never taken, so its look word never carries tag 1 and
    // tile 1 waits until its poll limit runs out
    const uint32_t one = 1u;
    cudaMemcpyAsync(ctr, &one, sizeof(one), cudaMemcpyHostToDevice, s);
    launch_pdl(k_scan_look<OpSum, true>, (unsigned)(ntiles - 1), kScanThreads, 0, s, (const uint32_t *)in, out, n,
               look, ctr, (unsigned long long)1, (uint32_t *)nullptr, (uint32_t *)nullptr, c->d_status);
    cudaFreeAsync(buf, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "scan probe");
    return OG_OK;
}

size_t scan_scratch_bytes(int64_t n) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    return (size_t)(ntiles + 1) * sizeof(uint32_t) + 256;
}

void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total,
                        void *scratch, cudaStream_t s) {
    scan_impl<OpSum, true>(in, out, n, d_total, scratch, s);
}

void scan_inclusive_max_u32(const uint32_t *in, uint32_t *out, int64_t n, void *scratch,
                            cudaStream_t s) {
    scan_impl<OpMax, false>(in, out, n, nullptr, scratch, s);
}

}  // namespace og
