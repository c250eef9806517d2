// og_sort.cu -- stable LSD radix sort of (63-bit Morton key, u32 index) pairs.
//
// The paper builds its tree by inserting the particles one after another in
// Peano-Hilbert order (Sect. 4.1.1); here the order is a Morton order made by a
// least-significant-digit radix sort, 8 bits per pass.  Each pass is
//   1. upsweep:   per 2048-key tile, a 256-bin digit histogram (shared-memory
//                 atomics, one sub-histogram per warp), stored digit-major;
//   2. scan:      exclusive scan over (digit, tile) -> global offsets;
//   3. downsweep: stable in-tile ranking by warp peer masks (each warp owns
//                 256 consecutive keys, 8 rounds of 32), keys staged in shared
//                 memory in digit order, then written out so that runs of one
//                 digit stay contiguous in global memory.
// Passes whose digit is the same for every key (found from one histogram of
// all passes, read by the pass kernels themselves: no host round trip) only
// copy their input.  Sorts of at most kOneSweepMaxTiles tiles (small sorts
// are bound by launch latency) run each pass as one kernel instead: the
// global digit bases come from that histogram, and a tile's offsets within
// its digit from a look-back over the counts the tiles before it publish.
#include "og_internal.h"

namespace og {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;        // 2048 keys per tile
constexpr int kPerWarp = 32 * kItems;           // 256 consecutive keys per warp
constexpr int kRadix = 256;
// sorts of at most this many tiles run each pass as one kernel (k_onesweep);
// larger ones as a count, a scan and a scatter per pass
constexpr int64_t kOneSweepMaxTiles = 384;
static_assert(kThreads == kRadix, "one thread per digit in the pass kernels");

// true in every thread of the block when all n keys share the digit of this
// pass (hist8: the digit histograms of all passes)
__device__ __forceinline__ bool trivial_pass(const uint32_t *hist8, int shift, int64_t n) {
    return __syncthreads_or(hist8 && hist8[(shift / 8) * kRadix + threadIdx.x] == (uint64_t)n) != 0;
}

// exclusive scan of one value per thread over the block (kThreads values)
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += warp_tot[w];
    __syncthreads();
    return wpre + inc - v;
}

__global__ void __launch_bounds__(kThreads) k_upsweep(const uint64_t *__restrict__ keys, int64_t n,
                                                      int shift, uint32_t *counts,
                                                      int64_t ntiles, const uint32_t *hist8) {
    pdl_wait();
    __shared__ uint32_t hist[kWarps][kRadix];
    const int warp = threadIdx.x >> 5;
    if (trivial_pass(hist8, shift, n)) return;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[warp][(uint32_t)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tot += hist[w][threadIdx.x];
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = tot;
}

// histogram of all eight digit positions over all keys (to skip trivial passes)
__global__ void __launch_bounds__(kThreads) k_all_digits(const uint64_t *__restrict__ keys,
                                                         int64_t n, uint32_t *hist8) {
    pdl_wait();
    __shared__ uint32_t h[8][kRadix];
    for (int i = threadIdx.x; i < 8 * kRadix; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
#pragma unroll
        for (int p = 0; p < 8; ++p) atomicAdd(&h[p][(uint32_t)(k >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * kRadix; i += kThreads) {
        uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(&hist8[i], v);
    }
}

struct DownSmem {
    uint64_t keys[kTile];
    uint32_t vals[kTile];
    uint32_t wcnt[kWarps][kRadix];
    uint32_t dstart[kRadix];
    uint32_t gofs[kRadix];
    uint32_t warp_tot[kWarps];
    uint32_t warp_tot2[kWarps];
};

__global__ void __launch_bounds__(kThreads, 4) k_downsweep(const uint64_t *__restrict__ kin,
                                                        const uint32_t *__restrict__ vin,
                                                        uint64_t *__restrict__ kout,
                                                        uint32_t *__restrict__ vout, int64_t n,
                                                        int shift, const uint32_t *offsets,
                                                        int64_t ntiles, const uint32_t *hist8) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem &S = *reinterpret_cast<DownSmem *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (trivial_pass(hist8, shift, n)) {
        // every key has this digit: the stable order is the input order
        const int64_t b0 = (int64_t)blockIdx.x * kTile;
        const int64_t e0 = (n - b0) < kTile ? n : b0 + kTile;
        for (int64_t i = b0 + threadIdx.x; i < e0; i += kThreads) {
            kout[i] = kin[i];
            vout[i] = vin[i];
        }
        return;
    }
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&S.wcnt[0][0])[i] = 0;
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint64_t k[kItems];
    uint32_t v[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + warp * kPerWarp + r * 32 + lane;
        bool valid = i < n;
        k[r] = valid ? kin[i] : 0ull;
        v[r] = valid ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + warp * kPerWarp + r * 32 + lane;
        uint32_t d = (i < n) ? ((uint32_t)(k[r] >> shift) & 0xffu) : (uint32_t)kRadix;
        // lanes with the same digit (9 bits: 256 marks an invalid key), from
        // one ballot per bit plane
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < 9; ++bit) {
            const bool on = (d >> bit) & 1u;
            const unsigned bb = __ballot_sync(0xffffffffu, on);
            peers &= on ? bb : ~bb;
        }
        int leader = __ffs(peers) - 1;
        uint32_t before = (d < kRadix) ? S.wcnt[warp][d] : 0u;
        __syncwarp();
        if (lane == leader && d < kRadix) S.wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: exclusive offsets of the warps, then the digit's tile total
    const int t = threadIdx.x;  // one thread per digit
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t c = S.wcnt[w][t];
        S.wcnt[w][t] = run;
        run += c;
    }
    // block exclusive scan of the digit totals
    uint32_t inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) S.warp_tot[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += S.warp_tot[w];
    S.dstart[t] = wpre + inc - run;
    S.gofs[t] = offsets[(int64_t)t * ntiles + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + warp * kPerWarp + r * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)(k[r] >> shift) & 0xffu;
            uint32_t pos = S.dstart[d] + S.wcnt[warp][d] + rank[r];
            S.keys[pos] = k[r];
            S.vals[pos] = v[r];
        }
    }
    __syncthreads();
    const int64_t cnt = (n - base) < kTile ? (n - base) : kTile;
    for (int p = threadIdx.x; p < cnt; p += kThreads) {
        uint64_t key = S.keys[p];
        uint32_t d = (uint32_t)(key >> shift) & 0xffu;
        uint32_t g = S.gofs[d] + ((uint32_t)p - S.dstart[d]);
        kout[g] = key;
        vout[g] = S.vals[p];
    }
}

// One pass of the sort in a single kernel: the tile's digit counts are
// published, the counts of the tiles before it are gathered by a look-back
// (decoupled: a tile's word first holds its own count, then the inclusive
// count of the tiles up to it), and the digit bases come from the histograms
// of all passes taken before the first pass.  Tiles are numbered in the order
// their blocks start, so every tile waits only on tiles whose blocks already
// run.  A look word: flag (2 bits: 1 own count, 2 inclusive), pass tag
// (6 bits, pass + 1, so that words of the previous pass read as not ready),
// count (low 32 bits).
constexpr unsigned long long kLookOwn = 1ull << 62, kLookInc = 2ull << 62;
constexpr int kLookSpinLimit = 1 << 20;

__device__ __forceinline__ void st_look(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_look(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kThreads, 4) k_onesweep(const uint64_t *__restrict__ kin,
                                                       const uint32_t *__restrict__ vin,
                                                       uint64_t *__restrict__ kout,
                                                       uint32_t *__restrict__ vout, int64_t n, int pass,
                                                       const uint32_t *hist8, unsigned long long *look,
                                                       uint32_t *tile_ctr, uint32_t *status) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem &S = *reinterpret_cast<DownSmem *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int shift = 8 * pass;
    if (threadIdx.x == 0) S.warp_tot2[0] = atomicAdd(&tile_ctr[pass], 1u);
    __syncthreads();
    const int64_t tile = S.warp_tot2[0];
    const int64_t base = tile * kTile;
    if (trivial_pass(hist8, shift, n)) {
        // every key has this digit: the stable order is the input order
        const int64_t e0 = (n - base) < kTile ? n : base + kTile;
        for (int64_t i = base + threadIdx.x; i < e0; i += kThreads) {
            kout[i] = kin[i];
            vout[i] = vin[i];
        }
        return;
    }
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&S.wcnt[0][0])[i] = 0;
    __syncthreads();

    uint64_t k[kItems];
    uint32_t v[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + warp * kPerWarp + r * 32 + lane;
        bool valid = i < n;
        k[r] = valid ? kin[i] : 0ull;
        v[r] = valid ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + warp * kPerWarp + r * 32 + lane;
        uint32_t d = (i < n) ? ((uint32_t)(k[r] >> shift) & 0xffu) : (uint32_t)kRadix;
        // lanes with the same digit (9 bits: 256 marks an invalid key)
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < 9; ++bit) {
            const bool on = (d >> bit) & 1u;
            const unsigned bb = __ballot_sync(0xffffffffu, on);
            peers &= on ? bb : ~bb;
        }
        int leader = __ffs(peers) - 1;
        uint32_t before = (d < kRadix) ? S.wcnt[warp][d] : 0u;
        __syncwarp();
        if (lane == leader && d < kRadix) S.wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit (one thread each): offsets of the warps, the tile's count
    const int t = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t c = S.wcnt[w][t];
        S.wcnt[w][t] = run;
        run += c;
    }
    // publish this tile's count, then gather the counts of the tiles before it
    const unsigned long long tag = (unsigned long long)(pass + 1) << 56;
    const unsigned long long tag_mask = 0x3full << 56;
    uint32_t excl = 0;
    if (tile == 0) {
        st_look(&look[t], kLookInc | tag | run);
    } else {
        st_look(&look[tile * kRadix + t], kLookOwn | tag | run);
        int64_t j = tile - 1;
        int spins = 0;
        while (j >= 0) {
            const unsigned long long w = ld_look(&look[j * kRadix + t]);
            if ((w & tag_mask) != tag || (w >> 62) == 0ull) {
                if (++spins > kLookSpinLimit) {  // a tile that never publishes: give up
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
                if (spins > 32) __nanosleep(64);
                continue;
            }
            excl += (uint32_t)w;
            if ((w >> 62) == 2ull) break;
            --j;
        }
        st_look(&look[tile * kRadix + t], kLookInc | tag | (excl + run));
    }
    // block exclusive scan of the tile's digit counts
    uint32_t inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) S.warp_tot[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += S.warp_tot[w];
    S.dstart[t] = wpre + inc - run;
    // where this tile's keys of digit t go: the keys of smaller digits (all
    // tiles) plus the keys of digit t in the tiles before this one
    S.gofs[t] = block_exclusive(hist8[pass * kRadix + t], S.warp_tot2) + excl;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + warp * kPerWarp + r * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)(k[r] >> shift) & 0xffu;
            uint32_t pos = S.dstart[d] + S.wcnt[warp][d] + rank[r];
            S.keys[pos] = k[r];
            S.vals[pos] = v[r];
        }
    }
    __syncthreads();
    const int64_t cnt = (n - base) < kTile ? (n - base) : kTile;
    for (int p = threadIdx.x; p < cnt; p += kThreads) {
        uint64_t key = S.keys[p];
        uint32_t d = (uint32_t)(key >> shift) & 0xffu;
        uint32_t g = S.gofs[d] + ((uint32_t)p - S.dstart[d]);
        kout[g] = key;
        vout[g] = S.vals[p];
    }
}

}  // namespace

size_t radix_sort_scratch_bytes(int64_t n) {
    int64_t ntiles = (n + kTile - 1) / kTile;
    // every-pass sort: per-tile counts and their scan
    size_t counts = (size_t)kRadix * ntiles * sizeof(uint32_t);
    size_t every = counts + scan_scratch_bytes((int64_t)kRadix * ntiles) + 8 * kRadix * sizeof(uint32_t) +
                   1024;
    // one-kernel passes: histograms, tile counters, one look word per tile and digit
    size_t one = 8 * kRadix * sizeof(uint32_t) + 256 + (size_t)kRadix * ntiles * sizeof(unsigned long long) +
                 1024;
    // large sorts: histograms, counters, the count scans' look words, counts, scan scratch
    size_t large = 8 * kRadix * sizeof(uint32_t) + 256 + scan_look_words((int64_t)kRadix * ntiles) * 8 + 256 +
                   counts + scan_scratch_bytes((int64_t)kRadix * ntiles) + 1024;
    if (large > one) one = large;
    return every > one ? every : one;
}

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                      int64_t n, int bits, void *scratch, cudaStream_t s, bool *result_in_alt,
                      uint32_t *status) {
    *result_in_alt = false;
    if (n <= 1) return;
    int64_t ntiles = (n + kTile - 1) / kTile;
    char *p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(scratch) + 255) & ~(uintptr_t)255);
    uint32_t *hist8 = reinterpret_cast<uint32_t *>(p);
    uint32_t *tile_ctr = hist8 + 8 * kRadix;
    unsigned long long *look = reinterpret_cast<unsigned long long *>(p + 8 * kRadix * sizeof(uint32_t) + 256);
    // large sorts: the look words of the tile counts' one-kernel scans (one
    // tag per pass), then the counts
    const size_t scan_words = scan_look_words((int64_t)kRadix * ntiles);
    const size_t clear = 8 * kRadix * sizeof(uint32_t) + 256 +
                         (ntiles > kOneSweepMaxTiles ? scan_words : (size_t)kRadix * ntiles) *
                             sizeof(unsigned long long);

    // the digit histograms of all passes (they give every pass its digit
    // bases and show which passes are trivial); counters and look words cleared
    cudaMemsetAsync(p, 0, clear, s);
    int grid = (int)((n + kThreads * 16 - 1) / (kThreads * 16));
    if (grid > 1184) grid = 1184;
    launch_pdl(k_all_digits, grid, kThreads, 0, s, keys, n, hist8);

    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(DownSmem));
        cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(DownSmem));
        attr_set = true;
    }
    uint64_t *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    int npasses = (bits + 7) / 8;
    if (ntiles > kOneSweepMaxTiles) {
        // many tiles: the look-back's waits cost more than the count and scan
        // launches they save
        uint32_t *counts = reinterpret_cast<uint32_t *>(
            (reinterpret_cast<uintptr_t>(look + scan_words) + 255) & ~(uintptr_t)255);
        void *scan_scratch = counts + (size_t)kRadix * ntiles;   // the two-kernel form's tile totals
        for (int pass = 0; pass < npasses; ++pass) {
            const int shift = 8 * pass;
            launch_pdl(k_upsweep, (unsigned)ntiles, kThreads, 0, s, (const uint64_t *)kin, n, shift, counts,
                       ntiles, (const uint32_t *)hist8);
            scan_exclusive_u32_look(counts, counts, (int64_t)kRadix * ntiles, nullptr, look, tile_ctr + 8 + pass,
                                    (uint32_t)(pass + 1), status, scan_scratch, s);
            launch_pdl(k_downsweep, (unsigned)ntiles, kThreads, sizeof(DownSmem), s, (const uint64_t *)kin,
                       (const uint32_t *)vin, kout, vout, n, shift, (const uint32_t *)counts, ntiles,
                       (const uint32_t *)hist8);
            uint64_t *tk = kin; kin = kout; kout = tk;
            uint32_t *tv = vin; vin = vout; vout = tv;
        }
        *result_in_alt = (kin == keys_alt);
        return;
    }
    for (int pass = 0; pass < npasses; ++pass) {
        launch_pdl(k_onesweep, (unsigned)ntiles, kThreads, sizeof(DownSmem), s, (const uint64_t *)kin,
                   (const uint32_t *)vin, kout, vout, n, pass, (const uint32_t *)hist8, look, tile_ctr, status);
        uint64_t *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
    *result_in_alt = (kin == keys_alt);
}

void radix_sort_pairs_every_pass(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                                 uint32_t *vals_alt, int64_t n, int bits, void *scratch,
                                 cudaStream_t s) {
    if (n <= 1) return;
    int64_t ntiles = (n + kTile - 1) / kTile;
    char *p = static_cast<char *>(scratch);
    uint32_t *counts = reinterpret_cast<uint32_t *>(p);
    p += (size_t)kRadix * ntiles * sizeof(uint32_t);
    p += 8 * kRadix * sizeof(uint32_t);
    void *scan_scratch = p;
    cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(DownSmem));
    uint64_t *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    const int npasses = (bits + 7) / 8;
    for (int pass = 0; pass < npasses; ++pass) {
        const int shift = 8 * pass;
        launch_pdl(k_upsweep, (unsigned)ntiles, kThreads, 0, s, kin, n, shift, counts, ntiles, nullptr);
        scan_exclusive_u32(counts, counts, (int64_t)kRadix * ntiles, nullptr, scan_scratch, s);
        launch_pdl(k_downsweep, (unsigned)ntiles, kThreads, sizeof(DownSmem), s, kin, vin, kout, vout, n,
                                                                         shift, counts, ntiles, nullptr);
        uint64_t *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
}

}  // namespace og
