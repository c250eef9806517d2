// a5: node moments (mass, sum of m x per axis) and centres of mass, exact.
//
// Monopole moments in double precision from the particles up (paper Sect.
// 4.1.1), read as the exact sums over a node's particles, each rounded once
// to FP64 (ties to even); the centre of mass is the grid point nearest to the
// exact ratio, ties to even; a massless node takes its cell centre.
//
// Exactness: a nonzero mass is m = s 2^e with an integer s < 2^53.  With b the
// lowest set-bit exponent over all masses, m = I 2^b with an integer I < 2^W,
// W the span from b to the top of the largest mass, and m x = (I x) 2^b for an
// integer grid coordinate x.  The node sums are then integer sums: the
// differences of prefix sums over the particles in key order.  The prefix sums
// run modulo 2^192; a node's sum is below 2^(W + 32 + 31), so for W <= 128 the
// differences are exact.  No summation order is involved, so the result does
// not depend on the tree's shape or on the launch, and there is no pass per
// tree level.
//
//   (the lowest and highest set bit over all masses come from the build's
//   k_permute, which reads the masses first)
//   k_mom_tiles      per tile of 512 sorted particles: the sums of the tile
//   k_mom_scan_l1/2  exclusive prefix over the tiles, in two levels (blocks of
//                    256 tiles, then the block totals)
//   k_mom_prefix     per particle: exclusive prefix P[i] = sum over q < i,
//                    and P[n], 96 bytes per entry
//   k_node_moments   per node: P[end] - P[begin], rounded to FP64, and the
//                    rounded ratio for the centre of mass
#include "og_internal.h"

namespace og {
namespace {

constexpr int kMomThreads = 256;
constexpr int kMomItems = 2;                        // consecutive particles per thread
constexpr int kMomTile = kMomThreads * kMomItems;   // 512
constexpr int kScanBlock = 256;                      // tiles per block of the first scan level
constexpr int kScanTop = 512;                        // threads of the second level
// a warp's 64 prefix records staged in shared memory before they are written
// out as contiguous 512-byte runs: 2 records per lane, 16 bytes of padding per
// lane so that the lanes' 16-byte stores fall in distinct banks
constexpr int kLaneStage = 2 * 96 + 16;
constexpr int kWarpStage = 32 * kLaneStage;
constexpr int kMassSpanMax = 128;                   // W above: the 192-bit sums stay exact

struct U192 {
    unsigned long long w0, w1, w2;
};
// mass, m x, m y, m z of a particle range: 96 bytes
struct __align__(16) Mom192 {
    U192 q[4];
};

__device__ __forceinline__ void add192(U192 &a, const U192 &b) {
    asm("add.cc.u64 %0, %0, %3;\n\t"
        "addc.cc.u64 %1, %1, %4;\n\t"
        "addc.u64 %2, %2, %5;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(b.w0), "l"(b.w1), "l"(b.w2));
}

__device__ __forceinline__ void sub192(U192 &a, const U192 &b) {
    asm("sub.cc.u64 %0, %0, %3;\n\t"
        "subc.cc.u64 %1, %1, %4;\n\t"
        "subc.u64 %2, %2, %5;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(b.w0), "l"(b.w1), "l"(b.w2));
}

__device__ __forceinline__ bool is_zero192(const U192 &a) { return (a.w0 | a.w1 | a.w2) == 0ull; }
__device__ __forceinline__ bool is_neg192(const U192 &a) { return (long long)a.w2 < 0; }

// -1, 0, 1 as a < b, a == b, a > b (unsigned)
__device__ __forceinline__ int cmp192(const U192 &a, const U192 &b) {
    if (a.w2 != b.w2) return a.w2 < b.w2 ? -1 : 1;
    if (a.w1 != b.w1) return a.w1 < b.w1 ? -1 : 1;
    if (a.w0 != b.w0) return a.w0 < b.w0 ? -1 : 1;
    return 0;
}

// a * x modulo 2^192, from six 32 x 32 -> 64-bit products
__device__ __forceinline__ U192 mul192(const U192 &a, uint32_t x) {
    const uint32_t h[6] = {(uint32_t)a.w0, (uint32_t)(a.w0 >> 32), (uint32_t)a.w1,
                           (uint32_t)(a.w1 >> 32), (uint32_t)a.w2, (uint32_t)(a.w2 >> 32)};
    uint32_t r[6];
    unsigned long long t = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        t = (t >> 32) + (unsigned long long)h[k] * x;
        r[k] = (uint32_t)t;
    }
    return {((unsigned long long)r[1] << 32) | r[0], ((unsigned long long)r[3] << 32) | r[2],
            ((unsigned long long)r[5] << 32) | r[4]};
}

// index of the highest set bit, -1 for zero
__device__ __forceinline__ int top192(const U192 &a) {
    if (a.w2) return 191 - __clzll((long long)a.w2);
    if (a.w1) return 127 - __clzll((long long)a.w1);
    if (a.w0) return 63 - __clzll((long long)a.w0);
    return -1;
}

// bits [s, s + 64) of a, 0 <= s < 192 (bits above 191 read as zero)
__device__ __forceinline__ unsigned long long bits192(const U192 &a, int s) {
    const int k = s >> 6, o = s & 63;
    const unsigned long long lo = k == 0 ? a.w0 : k == 1 ? a.w1 : a.w2;
    const unsigned long long hi = k == 0 ? a.w1 : k == 1 ? a.w2 : 0ull;
    return o ? (lo >> o) | (hi << (64 - o)) : lo;
}

// any set bit below bit s, 0 <= s < 192
__device__ __forceinline__ bool any_below192(const U192 &a, int s) {
    const int k = s >> 6, o = s & 63;
    const unsigned long long part = k == 0 ? a.w0 : k == 1 ? a.w1 : a.w2;
    const unsigned long long low = o ? (part & ((1ull << o) - 1ull)) : 0ull;
    return low != 0ull || (k >= 1 && a.w0 != 0ull) || (k >= 2 && a.w1 != 0ull);
}

// the mass as an integer in units of 2^b (I < 2^128 when the span is <= 128)
__device__ __forceinline__ U192 mass_units(double m, int b) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    const unsigned E = (unsigned)(bits >> 52) & 0x7ffu;
    if ((bits >> 63) || E == 0x7ffu) return {0ull, 0ull, 0ull};   // rejected input (status set)
    unsigned long long s = bits & ((1ull << 52) - 1ull);
    int ex = -1074;                                                 // m = s 2^ex
    if (E) {
        s |= 1ull << 52;
        ex = (int)E - 1075;
    }
    if (s == 0ull) return {0ull, 0ull, 0ull};
    int sh = ex - b;                     // >= -(trailing zeros of s): those bits are zero
    if (sh < 0) {
        s >>= -sh;
        sh = 0;
    }
    if (sh >= 64) return {0ull, s << (sh - 64), 0ull};
    return {s << sh, sh ? s >> (64 - sh) : 0ull, 0ull};
}

__device__ __forceinline__ void particle_moments(double m, uint32_t x, uint32_t y, uint32_t z,
                                                 int b, Mom192 &v) {
    v.q[0] = mass_units(m, b);
    v.q[1] = mul192(v.q[0], x);
    v.q[2] = mul192(v.q[0], y);
    v.q[3] = mul192(v.q[0], z);
}

__device__ __forceinline__ void mom_add(Mom192 &a, const Mom192 &b) {
#pragma unroll
    for (int k = 0; k < 4; ++k) add192(a.q[k], b.q[k]);
}

__device__ __forceinline__ void mom_zero(Mom192 &a) {
#pragma unroll
    for (int k = 0; k < 4; ++k) a.q[k] = {0ull, 0ull, 0ull};
}

__device__ __forceinline__ Mom192 mom_shfl_up(const Mom192 &a, int d) {
    Mom192 r;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        r.q[k].w0 = __shfl_up_sync(0xffffffffu, a.q[k].w0, d);
        r.q[k].w1 = __shfl_up_sync(0xffffffffu, a.q[k].w1, d);
        r.q[k].w2 = __shfl_up_sync(0xffffffffu, a.q[k].w2, d);
    }
    return r;
}

__device__ __forceinline__ Mom192 load_mom(const Mom192 *p) {
    const ulonglong2 *v = reinterpret_cast<const ulonglong2 *>(p);
    const ulonglong2 a = v[0], b = v[1], c = v[2], d = v[3], e = v[4], f = v[5];
    Mom192 r;
    r.q[0] = {a.x, a.y, b.x};
    r.q[1] = {b.y, c.x, c.y};
    r.q[2] = {d.x, d.y, e.x};
    r.q[3] = {e.y, f.x, f.y};
    return r;
}

__device__ __forceinline__ void store_mom(Mom192 *p, const Mom192 &r) {
    ulonglong2 *v = reinterpret_cast<ulonglong2 *>(p);
    v[0] = make_ulonglong2(r.q[0].w0, r.q[0].w1);
    v[1] = make_ulonglong2(r.q[0].w2, r.q[1].w0);
    v[2] = make_ulonglong2(r.q[1].w1, r.q[1].w2);
    v[3] = make_ulonglong2(r.q[2].w0, r.q[2].w1);
    v[4] = make_ulonglong2(r.q[2].w2, r.q[3].w0);
    v[5] = make_ulonglong2(r.q[3].w1, r.q[3].w2);
}

// The per-particle prefixes P are stored modulo 2^128 (64-byte records: the
// two low words of each sum) when the mass span W is at most kMassSpanShort:
// a node's sums are then below 2^(W + 26 + 32) <= 2^128 (at most 2^26
// particles, coordinates below 2^32), so the differences of the truncated
// prefixes are still the exact sums.  Wider spans keep the 96-byte records.
constexpr int kMassSpanShort = 70;

__device__ __forceinline__ bool short_prefix(const int *mbits) {
    // an empty span (lowest above highest) counts as short
    return (long long)mbits[1] - (long long)mbits[0] <= kMassSpanShort;
}

__device__ __forceinline__ void store_prefix(unsigned char *P, int64_t i, const Mom192 &r, bool shrt) {
    if (shrt) {
        ulonglong2 *v = reinterpret_cast<ulonglong2 *>(P + (size_t)i * 64);
        v[0] = make_ulonglong2(r.q[0].w0, r.q[0].w1);
        v[1] = make_ulonglong2(r.q[1].w0, r.q[1].w1);
        v[2] = make_ulonglong2(r.q[2].w0, r.q[2].w1);
        v[3] = make_ulonglong2(r.q[3].w0, r.q[3].w1);
    } else {
        store_mom(reinterpret_cast<Mom192 *>(P + (size_t)i * 96), r);
    }
}

// P[q1] - P[q0], the exact sums of the particles q0 .. q1 - 1
__device__ __forceinline__ Mom192 prefix_diff(const unsigned char *P, int64_t q0, int64_t q1, bool shrt) {
    Mom192 D;
    if (shrt) {
        const ulonglong2 *a = reinterpret_cast<const ulonglong2 *>(P + (size_t)q1 * 64);
        const ulonglong2 *c = reinterpret_cast<const ulonglong2 *>(P + (size_t)q0 * 64);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const ulonglong2 x = a[k], y = c[k];
            unsigned long long lo, hi;
            asm("sub.cc.u64 %0, %2, %4;\n\t"
                "subc.u64 %1, %3, %5;"
                : "=l"(lo), "=l"(hi)
                : "l"(x.x), "l"(x.y), "l"(y.x), "l"(y.y));
            D.q[k] = {lo, hi, 0ull};
        }
    } else {
        D = load_mom(reinterpret_cast<const Mom192 *>(P + (size_t)q1 * 96));
        const Mom192 Pb = load_mom(reinterpret_cast<const Mom192 *>(P + (size_t)q0 * 96));
#pragma unroll
        for (int k = 0; k < 4; ++k) sub192(D.q[k], Pb.q[k]);
    }
    return D;
}

// Inclusive scan of one value per thread over the block; returns the thread's
// exclusive prefix and the block total.
template <int kThreads>
__device__ __forceinline__ void block_scan(const Mom192 &x, Mom192 &excl, Mom192 &total) {
    constexpr int kWarps = kThreads / 32;
    __shared__ Mom192 wsum[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Mom192 inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Mom192 o = mom_shfl_up(inc, d);
        if (lane >= d) mom_add(inc, o);
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        Mom192 w;
        if (lane < kWarps) w = wsum[lane];
        else mom_zero(w);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Mom192 o = mom_shfl_up(w, d);
            if (lane >= d) mom_add(w, o);
        }
        if (lane < kWarps) wsum[lane] = w;     // inclusive over the warps
    }
    __syncthreads();
    total = wsum[kWarps - 1];
    Mom192 before;
    mom_zero(before);
    if (warp > 0) before = wsum[warp - 1];
    // exclusive within the warp: the inclusive value of the lane below
    Mom192 below = mom_shfl_up(inc, 1);
    if (lane == 0) mom_zero(below);
    mom_add(before, below);
    excl = before;
    __syncthreads();                           // wsum may be reused by the caller
}

__device__ __forceinline__ bool span_ok(const int *mbits, uint32_t *status) {
    const int lo = mbits[0], hi = mbits[1];
    if (hi >= lo && hi - lo > kMassSpanMax) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_MASS_RANGE);
        return false;
    }
    return true;
}

// this thread's kMomItems consecutive particles q0, q0 + 1 (vector loads);
// items past n have mass 0
__device__ __forceinline__ void load_pair(int64_t n, int64_t q0, const double *__restrict__ pm64,
                                          const uint32_t *__restrict__ px,
                                          const uint32_t *__restrict__ py,
                                          const uint32_t *__restrict__ pz, int b, Mom192 &v0,
                                          Mom192 &v1) {
    double2 m = make_double2(0.0, 0.0);
    uint2 x = make_uint2(0u, 0u), y = x, z = x;
    if (q0 + 1 < n) {
        m = *reinterpret_cast<const double2 *>(pm64 + q0);
        x = *reinterpret_cast<const uint2 *>(px + q0);
        y = *reinterpret_cast<const uint2 *>(py + q0);
        z = *reinterpret_cast<const uint2 *>(pz + q0);
    } else if (q0 < n) {
        m.x = pm64[q0];
        x.x = px[q0];
        y.x = py[q0];
        z.x = pz[q0];
    }
    particle_moments(m.x, x.x, y.x, z.x, b, v0);
    particle_moments(m.y, x.y, y.y, z.y, b, v1);
}

// the sums of one tile (the order of the additions does not matter: exact)
__global__ void __launch_bounds__(kMomThreads) k_mom_tiles(int64_t n, const double *__restrict__ pm64,
                                                           const uint32_t *__restrict__ px,
                                                           const uint32_t *__restrict__ py,
                                                           const uint32_t *__restrict__ pz,
                                                           const int *__restrict__ mbits,
                                                           Mom192 *tile_sum, uint32_t *status) {
    pdl_wait();
    if (!span_ok(mbits, status)) return;
    const int b = mbits[0];
    const int64_t q0 = (int64_t)blockIdx.x * kMomTile + (int64_t)threadIdx.x * kMomItems;
    __shared__ Mom192 wsum[kMomThreads / 32];
    Mom192 v0, v1;
    load_pair(n, q0, pm64, px, py, pz, b, v0, v1);
    mom_add(v0, v1);
    // the tile's total: a butterfly over the warp (sums modulo 2^192 do not
    // depend on the order), then the warps' totals
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        Mom192 o;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o.q[k].w0 = __shfl_xor_sync(0xffffffffu, v0.q[k].w0, d);
            o.q[k].w1 = __shfl_xor_sync(0xffffffffu, v0.q[k].w1, d);
            o.q[k].w2 = __shfl_xor_sync(0xffffffffu, v0.q[k].w2, d);
        }
        mom_add(v0, o);
    }
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v0;
    __syncthreads();
    if (threadIdx.x == 0) {
        Mom192 t = wsum[0];
#pragma unroll
        for (int w = 1; w < kMomThreads / 32; ++w) mom_add(t, wsum[w]);
        store_mom(&tile_sum[blockIdx.x], t);
    }
}

// first level: each block turns its kScanBlock tile sums into exclusive
// prefixes within the block (in place) and stores its total
__global__ void __launch_bounds__(kScanBlock) k_mom_scan_l1(int64_t ntiles, const int *__restrict__ mbits,
                                                            Mom192 *tile_sum, Mom192 *block_sum,
                                                            uint32_t *status) {
    pdl_wait();
    if (!span_ok(mbits, status)) return;
    const int64_t k = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    Mom192 v, excl, total;
    if (k < ntiles) v = load_mom(&tile_sum[k]);
    else mom_zero(v);
    block_scan<kScanBlock>(v, excl, total);
    if (k < ntiles) store_mom(&tile_sum[k], excl);
    if (threadIdx.x == 0) store_mom(&block_sum[blockIdx.x], total);
}

// second level: exclusive prefixes of the block totals (in place, several
// per thread when there are more than kScanTop), the grand total to P[n]
__global__ void __launch_bounds__(kScanTop) k_mom_scan_l2(int64_t nblocks, const int *__restrict__ mbits,
                                                          Mom192 *block_sum, unsigned char *P, int64_t n,
                                                          uint32_t *status) {
    pdl_wait();
    if (!span_ok(mbits, status)) return;
    const int64_t per = (nblocks + kScanTop - 1) / kScanTop;
    const int64_t k0 = (int64_t)threadIdx.x * per;
    const int64_t k1 = k0 + per < nblocks ? k0 + per : nblocks;
    Mom192 s, excl, total;
    mom_zero(s);
    for (int64_t k = k0; k < k1; ++k) mom_add(s, load_mom(&block_sum[k]));
    block_scan<kScanTop>(s, excl, total);
    for (int64_t k = k0; k < k1; ++k) {
        const Mom192 v = load_mom(&block_sum[k]);
        store_mom(&block_sum[k], excl);
        mom_add(excl, v);
    }
    if (threadIdx.x == 0) store_prefix(P, n, total, short_prefix(mbits));
}

// Per particle the exclusive prefix: the tile's offset (both scan levels)
// plus the prefix within the tile.  Thread t owns the items 2t, 2t + 1 of the
// tile; each warp stages its 64 records in shared memory and writes them out
// as contiguous 16-byte chunks, so that every store request covers whole
// sectors.
__global__ void __launch_bounds__(kMomThreads) k_mom_prefix(int64_t n, const double *__restrict__ pm64,
                                                            const uint32_t *__restrict__ px,
                                                            const uint32_t *__restrict__ py,
                                                            const uint32_t *__restrict__ pz,
                                                            const int *__restrict__ mbits,
                                                            const Mom192 *__restrict__ tile_off,
                                                            const Mom192 *__restrict__ block_off,
                                                            unsigned char *P, uint32_t *status) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char stage_all[];
    if (!span_ok(mbits, status)) return;
    const int b = mbits[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile0 = (int64_t)blockIdx.x * kMomTile;
    const int64_t q0 = tile0 + (int64_t)threadIdx.x * kMomItems;
    Mom192 v0, v1, s, excl, total;
    load_pair(n, q0, pm64, px, py, pz, b, v0, v1);
    s = v0;
    mom_add(s, v1);
    block_scan<kMomThreads>(s, excl, total);
    Mom192 run = load_mom(&tile_off[blockIdx.x]);
    mom_add(run, load_mom(&block_off[blockIdx.x / kScanBlock]));
    mom_add(run, excl);
    unsigned char *stage = stage_all + warp * kWarpStage;
    const int64_t wq0 = tile0 + (int64_t)warp * 64;
    if (short_prefix(mbits)) {
        // 64 records of 64 bytes: 256 chunks of 16 bytes, contiguous in P
        store_prefix(stage + lane * kLaneStage, 0, run, true);
        mom_add(run, v0);
        store_prefix(stage + lane * kLaneStage, 1, run, true);
        __syncwarp();
        unsigned char *dst = P + (size_t)wq0 * 64;
#pragma unroll 4
        for (int k = 0; k < 8; ++k) {
            const int c = k * 32 + lane;
            const int r = c >> 2, part = c & 3;
            if (wq0 + r < n) {
                const uint4 u = *reinterpret_cast<const uint4 *>(stage + (r >> 1) * kLaneStage + (r & 1) * 64 +
                                                                part * 16);
                *reinterpret_cast<uint4 *>(dst + (size_t)c * 16) = u;
            }
        }
    } else {
        // 64 records of 96 bytes: 384 chunks of 16 bytes
        store_mom(reinterpret_cast<Mom192 *>(stage + lane * kLaneStage), run);
        mom_add(run, v0);
        store_mom(reinterpret_cast<Mom192 *>(stage + lane * kLaneStage + 96), run);
        __syncwarp();
        unsigned char *dst = P + (size_t)wq0 * 96;
#pragma unroll 4
        for (int k = 0; k < 12; ++k) {
            const int c = k * 32 + lane;
            const int r = c / 6, part = c - 6 * r;
            if (wq0 + r < n) {
                const uint4 u = *reinterpret_cast<const uint4 *>(stage + (r >> 1) * kLaneStage + (r & 1) * 96 +
                                                                part * 16);
                *reinterpret_cast<uint4 *>(dst + (size_t)c * 16) = u;
            }
        }
    }
}

// a 2^b rounded to the nearest double, ties to even; overflow to infinity
__device__ __forceinline__ double to_double(const U192 &a, int b) {
    const int p = top192(a);
    if (p < 0) return 0.0;
    const int E = p + b;                       // a 2^b in [2^E, 2^(E+1))
    const bool normal = E >= -1022;
    const int lsb = normal ? p - 52 : -1074 - b;   // last kept bit of a
    unsigned long long mant;
    if (lsb <= 0) {
        mant = a.w0 << (-lsb);                 // exact: a < 2^(53 + lsb)
    } else {
        mant = bits192(a, lsb) & ((1ull << 53) - 1ull);
        const bool half = (bits192(a, lsb - 1) & 1ull) != 0ull;
        if (half && ((mant & 1ull) || any_below192(a, lsb - 1))) ++mant;
    }
    unsigned long long out;
    if (normal) {
        // mant in [2^52, 2^53]; a carry into 2^53 raises the exponent field
        // (E + 1022) << 52 plus the hidden bit is the biased exponent field;
        // E <= 1087 here, so the shift cannot leave 64 bits
        out = ((unsigned long long)(E + 1022) << 52) + mant;
        if (out >= 0x7ff0000000000000ull) out = 0x7ff0000000000000ull;   // infinity
    } else {
        out = mant;                            // subnormal; 2^52 encodes 2^-1022
    }
    return __longlong_as_double((long long)out);
}

// the top 24 bits of a nonzero a (top bit p) as a float in [2^23, 2^24)
__device__ __forceinline__ float top24(const U192 &a, int p) {
    const unsigned long long t = p >= 23 ? bits192(a, p - 23) : (a.w0 << (23 - p));
    return (float)(uint32_t)(t & 0xffffffull);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// v 2^k for a float v in [0, 4) and |k| small enough for no overflow
__device__ __forceinline__ float scale2(float v, int k) {
    if (k < -126) return 0.0f;
    return v * __int_as_float((127 + k) << 23);
}

// |a| / M as a float from the leading bits (relative error below 2^-20)
__device__ __forceinline__ float ratio_estimate(const U192 &a, int pM, float rM) {
    const int p = top192(a);
    if (p < 0) return 0.0f;
    return scale2(top24(a, p) * rM, p - pM);
}

// the integer nearest to S / M, ties to even (M > 0, S / M < 2^32); pM is
// the top bit of M and rM the reciprocal of its leading 24 bits
__device__ __forceinline__ uint32_t round_ratio(const U192 &S, const U192 &M, int pM, float rM,
                                                uint32_t *status) {
    // first estimate: within 2^12 of S / M
    const float q0f = fminf(ratio_estimate(S, pM, rM), 4294967040.0f);
    long long q = (long long)(unsigned)__float2uint_rd(q0f);
    U192 R = S;
    sub192(R, mul192(M, (uint32_t)q));          // |R| < 2^13 M: exact as a signed value
    // second estimate of the remainder's quotient: within 1 of it
    const bool neg = is_neg192(R);
    U192 A = R;
    if (neg) {
        A = {0ull, 0ull, 0ull};
        sub192(A, R);
    }
    const float df = ratio_estimate(A, pM, rM);
    const long long d = neg ? -(long long)ceilf(df) : (long long)floorf(df);
    if (d != 0) {
        q += d;
        if (d > 0) sub192(R, mul192(M, (uint32_t)d));
        else add192(R, mul192(M, (uint32_t)(-d)));
    }
    // exact: 0 <= S - q M < M
    for (int it = 0; it < 3; ++it) {
        if (is_neg192(R)) {
            --q;
            add192(R, M);
        } else if (cmp192(R, M) >= 0) {
            ++q;
            sub192(R, M);
        } else {
            break;
        }
    }
    if (is_neg192(R) || cmp192(R, M) >= 0 || q < 0 || q > 0xffffffffll) {
        atomicOr(status, ST_INTERNAL);
        return 0u;
    }
    U192 twoR = R;
    add192(twoR, R);
    const int c = cmp192(twoR, M);
    if (c > 0 || (c == 0 && (q & 1))) ++q;
    return (uint32_t)q;
}

// one thread per node; m = B + *nsplit (the build) or m_host (a refit)
__global__ void __launch_bounds__(kMomThreads) k_node_moments(
    const uint32_t *__restrict__ nsplit, int64_t B, int64_t m_host, int64_t mcap,
    const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ nend,
    const uint8_t *__restrict__ nlev, const uint32_t *__restrict__ px,
    const uint32_t *__restrict__ py, const uint32_t *__restrict__ pz,
    const unsigned char *__restrict__ P, const int *__restrict__ mbits, NodeMom *nmom, uint32_t *ncom,
    uint32_t *status) {
    pdl_wait();
    if (!span_ok(mbits, status)) return;
    int64_t m = nsplit ? B + (int64_t)*nsplit : m_host;
    if (m > mcap) m = mcap;                    // the host reports the overflow
    const int b = mbits[0];
    const bool shrt = short_prefix(mbits);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q0 = nbeg[j], q1 = nend[j];
        const Mom192 D = prefix_diff(P, q0, q1, shrt);
        nmom[j] = NodeMom{to_double(D.q[0], b), to_double(D.q[1], b), to_double(D.q[2], b),
                          to_double(D.q[3], b)};
        uint32_t c[3];
        if (!is_zero192(D.q[0])) {
            const int pM = top192(D.q[0]);
            const float rM = rcp_approx(top24(D.q[0], pM));
            c[0] = round_ratio(D.q[1], D.q[0], pM, rM, status);
            c[1] = round_ratio(D.q[2], D.q[0], pM, rM, status);
            c[2] = round_ratio(D.q[3], D.q[0], pM, rM, status);
        } else {
            // massless node: the cell centre
            const int level = nlev[j];
            const uint64_t mask = level == 0 ? 0ull : ~((1ull << (32 - level)) - 1ull);
            const uint32_t pc[3] = {px[q0], py[q0], pz[q0]};
            for (int a = 0; a < 3; ++a)
                c[a] = (uint32_t)(((uint64_t)pc[a] & mask) + (1ull << (31 - level)));
        }
        ncom[3 * j + 0] = c[0];
        ncom[3 * j + 1] = c[1];
        ncom[3 * j + 2] = c[2];
    }
}

inline int64_t mom_tiles(int64_t n) { return (n + kMomTile - 1) / kMomTile; }

}  // namespace

size_t moments_scratch_bytes(int64_t n) {
    const auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nt = (size_t)(mom_tiles(n) > 0 ? mom_tiles(n) : 1);
    const size_t nb = (nt + kScanBlock - 1) / kScanBlock;
    return up((size_t)(n + 1) * sizeof(Mom192)) + up(nt * sizeof(Mom192)) + up(nb * sizeof(Mom192)) + 256;
}

void node_moments(og_tree *t, const uint32_t *d_nsplit, int64_t mcap, void *scratch, cudaStream_t s) {
    const int64_t n = t->n;
    const int64_t ntiles = mom_tiles(n);
    const int64_t nblocks = (ntiles + kScanBlock - 1) / kScanBlock;
    const auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char *q = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(scratch) + 255) & ~(uintptr_t)255);
    unsigned char *P = reinterpret_cast<unsigned char *>(q);   // 64- or 96-byte records
    q += up((size_t)(n + 1) * sizeof(Mom192));
    Mom192 *tiles = reinterpret_cast<Mom192 *>(q);
    q += up((size_t)ntiles * sizeof(Mom192));
    Mom192 *blocks = reinterpret_cast<Mom192 *>(q);
    uint32_t *status = t->ctx->d_status;
    launch_pdl(k_mom_tiles, (unsigned)ntiles, kMomThreads, 0, s, n, t->pm64, t->px, t->py, t->pz, t->mbits,
                                                         tiles, status);
    launch_pdl(k_mom_scan_l1, (unsigned)nblocks, kScanBlock, 0, s, ntiles, t->mbits, tiles, blocks, status);
    launch_pdl(k_mom_scan_l2, 1, kScanTop, 0, s, nblocks, t->mbits, blocks, P, n, status);
    // the stage is above the default 48 KB of shared memory (set per call: the
    // attribute belongs to the current device)
    cudaFuncSetAttribute(k_mom_prefix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (kMomThreads / 32) * kWarpStage);
    launch_pdl(k_mom_prefix, (unsigned)ntiles, kMomThreads, (kMomThreads / 32) * kWarpStage, s, 
        n, t->pm64, t->px, t->py, t->pz, t->mbits, tiles, blocks, P, status);
    const int64_t mb = (mcap + kMomThreads - 1) / kMomThreads;
    const unsigned grid = (unsigned)(mb < 4096 ? (mb > 0 ? mb : 1) : 4096);
    launch_pdl(k_node_moments, grid, kMomThreads, 0, s, d_nsplit, t->nseg, t->nnodes, mcap, t->nbeg, t->nend,
                                                t->nlev, t->px, t->py, t->pz, P, t->mbits, t->nmom,
                                                t->ncom, status);
}

}  // namespace og
