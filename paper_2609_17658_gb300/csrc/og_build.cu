// og_build.cu -- tree construction on the GPU (Sect. 4.1.1 "Tree construction").
//
// The paper builds the tree by inserting particles one at a time in
// space-filling-curve order and then computing moments bottom-up.  Here the
// same tree is built fully in parallel from the sorted keys, for a forest of
// B independent periodic boxes (segments) at once: the particles of all boxes
// are concatenated, sorted by (box, key), and every box gets its own root
// (node ids 0..B-1).  A single system is the forest with B = 1.  Splits
// between two boxes are separators: no node spans them.
//
//   a1/a2  k_quantize_keys   f64 positions -> u32 fixed point -> 63-bit Morton key
//   a3     radix sort (og_sort.cu), k_permute gathers sorted SoA positions/masses
//                           and the masses' set-bit span
//   a4     k_split_tiles    level of every adjacent-key split (shared 3-bit digits)
//          k_split_carry    and, per level threshold, the nearest lower split
//          k_split_ranges   across tiles; the node a split belongs to: its key
//                           range (nearest lower splits on both sides) and whether
//                           it is the node's first split; first splits are
//                           numbered by a scan
//          k_node_init      nodes of first splits, node id of every split
//          k_link           parent of every node, owner node of every particle,
//                           octant-occupancy bits of every node
//          k_place          child array in key order, grouped by parent
//          k_threading      nextnode / sibling threading (unified index space)
//   a5     exact node moments and centres of mass (og_moments.cu): prefix
//                           sums over the sorted particles, one pass over the nodes
//          k_level_hist .. k_level_scatter   node ids bucketed by tree level (a
//                           refit's extents only, made on the first refit)
//          k_extents_level  a refit's node extents, one launch per large level
//          k_extents_run    a run of small levels in one block (a barrier per level)
//   a6     k_frontier       frontier node, unit and run start mark of every particle
//          k_groupmark      group starts (then compacted into gbeg by a scan)
//          k_group_fin      group ends, boxes and box index
//          k_records        32-byte child records read by the walk
//          k_cell_origin    node cell origins, made when extents are first needed
//
// Every decision is integer or exact, so the result is identical to the
// oracle's recursive construction.
#include <cmath>
#include <cstdio>
#include <vector>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kT = 256;
constexpr uint8_t kSep = 0xff;  // split level of a boundary between two boxes

__device__ __forceinline__ uint64_t spread21(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ int lcp_levels(uint64_t a, uint64_t b) {
    uint64_t x = a ^ b;
    return x == 0 ? kLevels : (__clzll((long long)x) - 1) / 3;
}

__device__ __forceinline__ int digit_at(uint64_t key, int lev) {
    return (int)((key >> (3 * (kLevels - lev))) & 7u);
}

// u = floor(frac(t) * 2^32), t = x / L, evaluated exactly as
// floor(t * 2^32) mod 2^32: t * 2^32 is an exact scaling and, for |t| < 2^31,
// fits a signed 64-bit integer after the round-down conversion.  When L is a
// power of two, x * (1/L) equals the correctly rounded quotient exactly.
// floor(v * 2^s) mod 2^32 for a finite v, from the bits of v: |v| = M 2^e with
// an integer mantissa M, so |v| 2^s = M 2^(e + s) is a shift of M.  Negative v:
// floor(-a) = -(floor(a) + [a not an integer]).  Integer operations only (the
// FP64 rate of the GPU is 1/64 of its FP32 rate), except for a negative v of
// magnitude below one grid unit: there the FP64 quotient v / L the reading
// starts from may underflow to -0 (then 0, else -1), so that product decides.
__device__ __forceinline__ uint32_t fixed_shift(double v, int s, double inv_box) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7ffu);
    unsigned long long M = b & 0xfffffffffffffull;
    int e = -1074;                                   // subnormal
    if (E != 0) {
        M |= 1ull << 52;
        e = E - 1075;
    }
    if (M == 0) return 0u;                           // +0 and -0
    const int sh = e + s;
    uint32_t mag = 0;
    bool frac = false;
    if (sh >= 32) {
        mag = 0;                                     // a multiple of 2^32
    } else if (sh >= 0) {
        mag = (uint32_t)(M << sh);                   // the low 32 bits survive the wrap
    } else if (sh > -64) {
        mag = (uint32_t)(M >> -sh);
        frac = (M & ((1ull << -sh) - 1ull)) != 0ull;
    } else {
        frac = true;                                 // 0 < a < 1
    }
    if (!(b >> 63)) return mag;
    if (mag == 0u && frac) return (v * inv_box == 0.0) ? 0u : 0xffffffffu;
    return 0u - (mag + (frac ? 1u : 0u));
}

__device__ __forceinline__ uint32_t quantize(double v, double box, double inv_box, bool pow2,
                                             int shift, uint32_t *status) {
    if (!isfinite(v)) {
        atomicOr(status, ST_BAD_INPUT);
        return 0;
    }
    if (pow2) return fixed_shift(v, shift, inv_box);
    const double t = __ddiv_rn(v, box);
    if (fabs(t) < 2147483648.0) return (uint32_t)(unsigned long long)__double2ll_rd(t * 4294967296.0);
    const double f = t - floor(t);  // exact for |t| >= 1
    return (uint32_t)floor(f * 4294967296.0);
}

// segment (box) of every particle of the concatenated input
__global__ void k_fill_seg(int64_t n, int64_t B, const uint32_t *__restrict__ seg_off, uint32_t *pseg) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t lo = 0, hi = B;  // seg_off[lo] <= i < seg_off[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if ((uint64_t)seg_off[mid] <= (uint64_t)i) lo = mid; else hi = mid;
    }
    pseg[i] = (uint32_t)lo;
}

// In a build (d_tot set) it also clears what later kernels accumulate into:
// the device totals, the masses' set-bit span (empty: lowest 0x7f7f7f7f
// above highest 0x80808080), the scans' look words and tile counters, and with
// one box its sorted box indices (all 0).
__global__ void k_quantize_keys(const double *__restrict__ pos, int64_t n, const uint32_t *__restrict__ pseg,
                                const SegGeom *__restrict__ geom, uint4 *q4, uint64_t *key,
                                uint64_t *key_copy, uint32_t *idx,
                                uint32_t *sseg_zero, uint32_t *d_tot, int *mbits,
                                unsigned long long *scan_look, int64_t nlook, uint32_t *status) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the look words and tile counters of the build's one-kernel scans
    for (int64_t k = i; k < nlook; k += (int64_t)gridDim.x * blockDim.x) scan_look[k] = 0ull;
    if (i == 0 && d_tot) {
        d_tot[0] = d_tot[1] = d_tot[2] = d_tot[3] = 0u;
        mbits[0] = 0x7f7f7f7f;
        mbits[1] = (int)0x80808080u;
    }
    if (i >= n) return;
    if (sseg_zero) sseg_zero[i] = 0u;
    const SegGeom g = geom[pseg ? pseg[i] : 0];
    const double box = g.box, inv_box = g.inv_box;
    const bool pow2 = g.pow2 != 0;
    uint32_t x = quantize(pos[3 * i + 0], box, inv_box, pow2, g.shift, status);
    uint32_t y = quantize(pos[3 * i + 1], box, inv_box, pow2, g.shift, status);
    uint32_t z = quantize(pos[3 * i + 2], box, inv_box, pow2, g.shift, status);
    q4[i] = make_uint4(x, y, z, 0u);   // one 16-byte record: the permute gathers it whole
    const uint64_t k = (spread21(x >> 11) << 2) | (spread21(y >> 11) << 1) | spread21(z >> 11);
    key[i] = k;
    if (key_copy) key_copy[i] = k;
    idx[i] = (uint32_t)i;
}

// after the key sort: sort key = box index of each particle (stable second pass)
__global__ void k_seg_keys(int64_t n, const uint32_t *__restrict__ idx,
                           const uint32_t *__restrict__ pseg, uint64_t *segkey) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    segkey[i] = pseg[idx[i]];
}

__global__ void k_gather_keys(int64_t n, const uint32_t *__restrict__ perm,
                              const uint64_t *__restrict__ key0, const uint32_t *__restrict__ pseg,
                              uint64_t *skey, uint32_t *sseg) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    skey[i] = key0[j];
    sseg[i] = pseg[j];
}

// Positions and masses in key order, and the inverse permutation (the force
// call gathers its caller-order outputs through it); the masses are checked here, and their
// set-bit span (the units of the exact moments) is gathered: a block's lowest
// and highest exponents, merged by atomics only where they widen the span.
__global__ void __launch_bounds__(kT) k_permute(int64_t n, const uint32_t *__restrict__ perm,
                                                const uint4 *__restrict__ q4, const double *__restrict__ mass,
                                                uint32_t *px, uint32_t *py, uint32_t *pz, float *pm32,
                                                double *pm64, uint32_t *inv, int *mbits, uint32_t *status) {
    pdl_wait();
    __shared__ int wlo[kT / 32], whi[kT / 32];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int lo = 0x7fffffff, hi = (int)0x80000000;
    if (i < n) {
        uint32_t j = perm[i];
        inv[j] = (uint32_t)i;
        const uint4 q = q4[j];
        px[i] = q.x;
        py[i] = q.y;
        pz[i] = q.z;
        double m = mass[j];
        if (!isfinite(m) || m < 0.0) atomicOr(status, ST_BAD_INPUT);
        pm64[i] = m;
        pm32[i] = __double2float_rn(m);
        mass_bit_span(m, lo, hi);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31u) == 0u) {
        wlo[threadIdx.x >> 5] = lo;
        whi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kT / 32; ++w) {
            lo = min(lo, wlo[w]);
            hi = max(hi, whi[w]);
        }
        if (lo <= hi) {
            if (lo < __ldcg(&mbits[0])) atomicMin(&mbits[0], lo);
            if (hi > __ldcg(&mbits[1])) atomicMax(&mbits[1], hi);
        }
    }
}

// The node of a split of level L is the key range around it whose adjacent
// splits all have levels >= L (the lcp of two sorted keys is the smallest
// split level between them); so its ends are the nearest splits of a level
// below L on either side (a box boundary counts as below every level).  The
// levels take 23 values, so "nearest split below t" is answered for every
// threshold t at once: a ballot per threshold inside a warp, a fold over the
// warps of a tile, and a scan over the tiles.
constexpr int kSplitTile = 1024;       // splits per block
constexpr int kNT = kLevels + 2;       // thresholds t = 0 .. kLevels + 1: level < t
constexpr int kNone = 0x7fffffff;      // no split below t on the right

// a split's level as an ordered value: a box boundary below every level
__device__ __forceinline__ int split_rank(uint8_t v) { return v == kSep ? -1 : (int)v; }

// The lanes of a warp whose split lies below threshold t, for a t of each
// lane's own choosing: the values u = rank + 1 (0 .. kNT + 1, five bits) go
// out as five bit-plane ballots, and each lane compares them with its own
// threshold bit by bit, from the top (u < t + 1 iff the split's level < t).
struct WarpLevels {
    unsigned b[5];
};
__device__ __forceinline__ WarpLevels warp_levels(int v) {
    const unsigned u = (unsigned)(v + 1);
    WarpLevels w;
#pragma unroll
    for (int k = 0; k < 5; ++k) w.b[k] = __ballot_sync(0xffffffffu, (u >> k) & 1u);
    return w;
}
__device__ __forceinline__ unsigned lanes_below(const WarpLevels &w, int t) {
    const unsigned c = (unsigned)(t + 1);   // t <= kNT - 1, so c < 32
    unsigned less = 0u, eq = 0xffffffffu;
#pragma unroll
    for (int k = 4; k >= 0; --k) {
        const bool cb = (c >> k) & 1u;
        less |= cb ? (eq & ~w.b[k]) : 0u;
        eq &= cb ? w.b[k] : ~w.b[k];
    }
    return less;
}

// levels of all splits; per tile and threshold, its last and first split below t
__global__ void __launch_bounds__(kSplitTile) k_split_tiles(const uint64_t *__restrict__ skey,
                                                            const uint32_t *__restrict__ sseg, int64_t nsplit,
                                                            uint8_t *lv, int *tlast, int *tfirst) {
    pdl_wait();
    __shared__ int wl[32][kNT], wf[32][kNT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kSplitTile + threadIdx.x;
    int v = kNT;  // past the last split: below no threshold
    // key i and box i of every lane (i <= nsplit = n - 1 is a particle); the
    // next particle's from the lane above, the warp's last lane loads its own
    const int64_t ic = i <= nsplit ? i : nsplit;
    const uint64_t k0 = skey[ic];
    const uint32_t s0 = sseg[ic];
    uint64_t k1 = __shfl_down_sync(0xffffffffu, k0, 1);
    uint32_t s1 = __shfl_down_sync(0xffffffffu, s0, 1);
    if (lane == 31 && i < nsplit) {
        k1 = skey[i + 1];
        s1 = sseg[i + 1];
    }
    if (i < nsplit) {
        const uint8_t l = (s0 != s1) ? kSep : (uint8_t)lcp_levels(k0, k1);
        lv[i] = l;
        v = split_rank(l);
    }
    // lane t < kNT: this warp's last and first split below threshold t
    const int64_t base = (int64_t)blockIdx.x * kSplitTile + warp * 32;
    const unsigned m = lanes_below(warp_levels(v), lane < kNT ? lane : 0);
    if (lane < kNT) {
        wl[warp][lane] = m ? (int)(base + 31 - __clz(m)) : -1;
        wf[warp][lane] = m ? (int)(base + __ffs(m) - 1) : kNone;
    }
    __syncthreads();
    // warp t folds threshold t over the 32 warps of the tile
    if (warp < kNT) {
        int l = wl[lane][warp], f = wf[lane][warp];
        l = __reduce_max_sync(0xffffffffu, l);
        f = __reduce_min_sync(0xffffffffu, f);
        if (lane == 0) {
            tlast[blockIdx.x * kNT + warp] = l;
            tfirst[blockIdx.x * kNT + warp] = f;
        }
    }
}

// per tile and threshold t: the last split below t in the tiles before it and
// the first one in the tiles after it (one block per threshold)
__global__ void __launch_bounds__(kSplitTile) k_split_carry(int64_t ntiles, const int *__restrict__ tlast,
                                                            const int *__restrict__ tfirst, int *clast,
                                                            int *cfirst) {
    pdl_wait();
    __shared__ int ws[32];
    const int t = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // left to right: exclusive running maximum of tlast
    int run = -1;
    for (int64_t c0 = 0; c0 < ntiles; c0 += kSplitTile) {
        const int64_t k = c0 + threadIdx.x;
        const int x = k < ntiles ? tlast[k * kNT + t] : -1;
        int inc = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc = max(inc, o);
        }
        if (lane == 31) ws[warp] = inc;
        __syncthreads();
        int before = run;
        for (int w = 0; w < warp; ++w) before = max(before, ws[w]);
        const int ex = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane > 0) before = max(before, ex);
        if (k < ntiles) clast[k * kNT + t] = before;
        for (int w = 0; w < 32; ++w) run = max(run, ws[w]);
        __syncthreads();
    }
    // right to left: exclusive running minimum of tfirst
    run = kNone;
    for (int64_t c0 = 0; c0 < ntiles; c0 += kSplitTile) {
        const int64_t k = ntiles - 1 - (c0 + threadIdx.x);  // thread 0 takes the last tile
        const int x = k >= 0 ? tfirst[k * kNT + t] : kNone;
        int inc = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc = min(inc, o);
        }
        if (lane == 31) ws[warp] = inc;
        __syncthreads();
        int after = run;
        for (int w = 0; w < warp; ++w) after = min(after, ws[w]);
        const int ex = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane > 0) after = min(after, ex);
        if (k >= 0) cfirst[k * kNT + t] = after;
        for (int w = 0; w < 32; ++w) run = min(run, ws[w]);
        __syncthreads();
    }
}

// Node of every split: its key range [sb, se) (written for first splits), and
// whether it is its node's first split: no split of the same level between the
// range start and it.  A later split of the node keeps the nearest split to
// its left of a level <= L (prevle), which is the node's previous split, or
// at level kLevels the node's first split.
__global__ void __launch_bounds__(kSplitTile) k_split_ranges(const uint8_t *__restrict__ lv, int64_t nsplit,
                                                             const int *__restrict__ clast,
                                                             const int *__restrict__ cfirst, uint32_t *sb,
                                                             uint32_t *se, uint32_t *first, uint32_t *prevle) {
    pdl_wait();
    __shared__ int wl[32][kNT], wf[32][kNT];
    __shared__ int pl[32][kNT], pf[32][kNT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kSplitTile + threadIdx.x;
    const int v = i < nsplit ? split_rank(lv[i]) : kNT;
    // warp t's carries for threshold t, loaded first so that their latency
    // passes while the warp works on its ballots
    int cl = -1, cf = kNone;
    if (warp < kNT) {
        cl = clast[blockIdx.x * kNT + warp];
        cf = cfirst[blockIdx.x * kNT + warp];
    }
    const int64_t base = (int64_t)blockIdx.x * kSplitTile + warp * 32;
    const WarpLevels W = warp_levels(v);
    {
        const unsigned m = lanes_below(W, lane < kNT ? lane : 0);
        if (lane < kNT) {
            wl[warp][lane] = m ? (int)(base + 31 - __clz(m)) : -1;
            wf[warp][lane] = m ? (int)(base + __ffs(m) - 1) : kNone;
        }
    }
    __syncthreads();
    // warp t: for threshold t, the nearest split below t in the warps (and
    // tiles) before each warp and after it
    if (warp < kNT) {
        const int t = warp;
        int l = wl[lane][t];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, l, d);
            if (lane >= d) l = max(l, o);
        }
        int lex = __shfl_up_sync(0xffffffffu, l, 1);
        pl[lane][t] = lane == 0 ? cl : max(cl, lex);
        int f = wf[lane][t];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_down_sync(0xffffffffu, f, d);
            if (lane + d < 32) f = min(f, o);
        }
        int fex = __shfl_down_sync(0xffffffffu, f, 1);
        pf[lane][t] = lane == 31 ? cf : min(cf, fex);
    }
    __syncthreads();
    if (i >= nsplit) return;
    if (v < 0) {  // a boundary between two boxes
        first[i] = 0u;
        return;
    }
    const int L = v;
    const unsigned below = (1u << lane) - 1u;
    const unsigned above = lane == 31 ? 0u : (0xfffffffeu << lane);
    const unsigned mL = lanes_below(W, L), mL1 = lanes_below(W, L + 1);
    // nearest split of a level < L to the left (or -1) and to the right (or the end)
    const int left = (mL & below) ? (int)(base + 31 - __clz(mL & below)) : pl[warp][L];
    int right = (mL & above) ? (int)(base + __ffs(mL & above) - 1) : pf[warp][L];
    if (right > (int)nsplit) right = (int)nsplit;
    // nearest split of a level <= L to the left
    const int le = (mL1 & below) ? (int)(base + 31 - __clz(mL1 & below)) : pl[warp][L + 1];
    const bool isfirst = L >= 1 && le == left;
    first[i] = isfirst ? 1u : 0u;
    if (isfirst) {
        sb[i] = (uint32_t)(left + 1);
        se[i] = (uint32_t)(right + 1);
    } else {
        // a node of level < kLevels has at most 7 splits of its level; one of
        // level kLevels (a run of equal keys) any number, and its first split
        // is the range start
        // when the range starts in this warp, its first split is the lowest
        // split of a level <= L after the range start, found from the mask
        uint32_t f = (uint32_t)le;
        if (L == kLevels) {
            f = (uint32_t)(left + 1);
        } else if (left + 1 >= base) {
            const int sh = left - (int)base;   // -1 .. 30: the lanes after left
            const unsigned after = sh < 0 ? 0xffffffffu : ~((2u << sh) - 1u);
            f = (uint32_t)(base + __ffs(mL1 & after) - 1);
        }
        prevle[i] = f;
    }
}

// Roots, the nodes of first splits (level, key range), cleared
// per-node accumulators, and the node id of every split: its box's root at level 0, else the node of the
// first split reached along prevle (at most 7 steps).
__global__ void k_node_init(int64_t n, int64_t B, const uint32_t *__restrict__ seg_off,
                            const uint32_t *__restrict__ first, const uint32_t *__restrict__ nid,
                            const uint8_t *__restrict__ lv, const uint32_t *__restrict__ sb,
                            const uint32_t *__restrict__ se, const uint32_t *__restrict__ prevle,
                            const uint32_t *__restrict__ sseg,
                            uint8_t *nlev, uint32_t *nbeg, uint32_t *nend, uint32_t *sid,
                            int64_t mcap, uint32_t *occ, uint32_t *nnc, uint32_t *nccnt, uint32_t *status) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < mcap) {  // per-node accumulators of the kernels that follow
        occ[i] = 0u;
        nnc[i] = 0u;
        nccnt[i] = 0u;
    }
    if (i < B) {  // the root of box i covers the whole box
        nlev[i] = 0;
        nbeg[i] = seg_off[i];
        nend[i] = seg_off[i + 1];
    }
    if (i >= n - 1) return;
    const int L = lv[i];
    if (L == kSep) { sid[i] = 0xffffffffu; return; }
    if (L == 0) { sid[i] = sseg[i]; return; }  // the root of this box
    if (first[i]) {
        const uint32_t id = (uint32_t)B + nid[i];
        sid[i] = id;
        nlev[id] = (uint8_t)L;
        nbeg[id] = sb[i];
        nend[id] = se[i];
        return;
    }
    uint32_t j = prevle[i];
    for (int guard = 0;; ++guard) {
        if (guard > 7 || (int64_t)j >= n - 1) {
            atomicOr(status, ST_INTERNAL);
            sid[i] = sseg[i];
            return;
        }
        if (first[j]) break;
        j = prevle[j];
    }
    sid[i] = (uint32_t)B + nid[j];
}

__device__ __forceinline__ int split_at(const uint8_t *lv, int64_t j, int64_t n) {
    if (j < 0 || j >= n - 1) return -1;
    const uint8_t v = lv[j];
    return v == kSep ? -1 : (int)v;
}

// parent of every non-root node, owner of every particle, octant occupancy
__global__ void k_link(int64_t n, const uint32_t *__restrict__ nsplit, int64_t B,
                       const uint64_t *__restrict__ skey,
                       const uint8_t *__restrict__ lv, const uint32_t *__restrict__ sid,
                       const uint32_t *__restrict__ sseg, const uint8_t *__restrict__ nlev,
                       const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ nend,
                       int32_t *npar, uint32_t *owner, uint32_t *occ, uint32_t *nnc,
                       uint32_t *status) {
    pdl_wait();
    const int64_t m = B + (int64_t)*nsplit;  // nodes: the roots and one per first split
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const int64_t p = t;
        const int dl = split_at(lv, p - 1, n), dr = split_at(lv, p, n);
        uint32_t own;
        if (dl < 0 && dr < 0) own = sseg[p];  // alone in its box: hangs from the root
        else own = sid[dl >= dr ? p - 1 : p];
        if (own >= (uint32_t)m) {
            atomicOr(status, ST_INTERNAL);
            own = sseg[p];
        }
        owner[p] = own;
        int lo = nlev[own];
        if (lo < kLevels) atomicOr(&occ[own], 1u << digit_at(skey[p], lo + 1));
    } else if (t < n + (m - B)) {
        const int64_t id = B + (t - n);
        const int64_t b = nbeg[id], e = nend[id];
        const int dl = split_at(lv, b - 1, n), dr = split_at(lv, e - 1, n);
        uint32_t par;
        if (dl < 0 && dr < 0) par = sseg[b];  // the whole box: child of its root
        else par = sid[dl >= dr ? b - 1 : e - 1];
        npar[id] = (int32_t)par;
        if (par >= (uint32_t)m || nlev[par] >= nlev[id] || nlev[par] >= kLevels) {
            atomicOr(status, ST_INTERNAL);
            return;
        }
        atomicOr(&occ[par], 1u << digit_at(skey[b], nlev[par] + 1));
        atomicAdd(&nnc[par], 1u);
    } else if (t < n + m) {
        npar[t - n - (m - B)] = -1;  // roots
    }
}

__global__ void k_ccnt(const uint32_t *__restrict__ nsplit, int64_t B, const uint8_t *__restrict__ nlev,
                       const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ nend,
                       const uint32_t *__restrict__ occ, uint32_t *nccnt) {
    pdl_wait();
    const int64_t m = B + (int64_t)*nsplit;
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= m) return;
    nccnt[id] = nlev[id] == kLevels ? nend[id] - nbeg[id] : (uint32_t)__popc(occ[id]);
}

__global__ void k_place(int64_t n, const uint32_t *__restrict__ nsplit, int64_t B,
                        const uint64_t *__restrict__ skey,
                        const uint8_t *__restrict__ nlev, const uint32_t *__restrict__ nbeg,
                        const uint32_t *__restrict__ ncbeg, const uint32_t *__restrict__ occ,
                        const int32_t *__restrict__ npar, const uint32_t *__restrict__ owner,
                        uint32_t *child, uint32_t *npos, uint32_t *status) {
    pdl_wait();
    const int64_t m = B + (int64_t)*nsplit;
    const int64_t nchild = n + (m - B);
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const int64_t p = t;
        uint32_t own = owner[p];
        int lo = nlev[own];
        uint32_t slot;
        if (lo == kLevels) {
            slot = ncbeg[own] + (uint32_t)(p - nbeg[own]);
        } else {
            int d = digit_at(skey[p], lo + 1);
            slot = ncbeg[own] + __popc(occ[own] & ((1u << d) - 1u));
        }
        if (slot >= (uint64_t)nchild) { atomicOr(status, ST_INTERNAL); return; }
        child[slot] = (uint32_t)p;
    } else if (t < n + m - B) {
        const int64_t id = B + (t - n);
        uint32_t par = (uint32_t)npar[id];
        int d = digit_at(skey[nbeg[id]], nlev[par] + 1);
        uint32_t slot = ncbeg[par] + __popc(occ[par] & ((1u << d) - 1u));
        if (slot >= (uint64_t)nchild) { atomicOr(status, ST_INTERNAL); return; }
        child[slot] = (uint32_t)(n + id);
        npos[id] = slot;
    }
}

__global__ void k_threading(int64_t n, const uint32_t *__restrict__ nsplit, int64_t B,
                            const uint32_t *__restrict__ child,
                            const uint32_t *__restrict__ ncbeg, const uint32_t *__restrict__ nccnt,
                            const int32_t *__restrict__ npar, const uint32_t *__restrict__ npos,
                            const uint32_t *__restrict__ owner, int32_t *nnext, int32_t *nsib,
                            int32_t *pnext, uint32_t *status) {
    pdl_wait();
    const int64_t m = B + (int64_t)*nsplit;
    const int64_t nchild = n + (m - B);
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < m) {
        nnext[c] = (int32_t)child[ncbeg[c]];
        if (c < B) nsib[c] = -1;  // a root ends its box's threading
    }
    if (c >= nchild) return;
    const uint32_t item = child[c];
    int64_t par = item < n ? (int64_t)owner[item] : (int64_t)npar[item - n];
    int64_t cc = c;
    int32_t after = -1;
    for (int guard = 0;; ++guard) {
        if (guard > 2 * kLevels + 2 || par < 0 || par >= m) { atomicOr(status, ST_INTERNAL); break; }
        if (cc + 1 < (int64_t)ncbeg[par] + nccnt[par]) { after = (int32_t)child[cc + 1]; break; }
        if (par < B) { after = -1; break; }
        cc = npos[par];
        par = npar[par];
    }
    if (item < n) pnext[item] = after;
    else nsib[item - n] = after;
}

// Node ids bucketed by tree level, for the bottom-up pass of a refit's
// extents (a node's extent joins its children's).
constexpr int kLvItems = 16;  // nodes per thread in the level bucketing

// per-block shared-memory histograms, one global atomic per level and block
__global__ void __launch_bounds__(kT) k_level_hist(const uint32_t *__restrict__ nsplit, int64_t B,
                                                   const uint8_t *__restrict__ nlev,
                                                   uint32_t *lcount) {
    pdl_wait();
    const int64_t m = B + (int64_t)*nsplit;
    __shared__ uint32_t h[kLevels + 1];
    if (threadIdx.x <= kLevels) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * kLvItems;
    for (int k = 0; k < kLvItems; ++k) {
        const int64_t id = base + (int64_t)k * blockDim.x + threadIdx.x;
        if (id < m) atomicAdd(&h[nlev[id]], 1u);
    }
    __syncthreads();
    if (threadIdx.x <= kLevels && h[threadIdx.x]) atomicAdd(&lcount[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_level_offsets(uint32_t *lcount, uint32_t *loff, uint32_t *lcursor) {
    pdl_wait();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t run = 0;
    for (int l = 0; l <= kLevels; ++l) {
        loff[l] = run;
        lcursor[l] = 0;
        run += lcount[l];
    }
    loff[kLevels + 1] = run;
}

__global__ void __launch_bounds__(kT) k_level_scatter(const uint32_t *__restrict__ nsplit, int64_t B,
                                                      const uint8_t *__restrict__ nlev,
                                                      const uint32_t *__restrict__ loff,
                                                      uint32_t *lcursor, uint32_t *lnodes) {
    pdl_wait();
    const int64_t m = B + (int64_t)*nsplit;
    __shared__ uint32_t h[kLevels + 1], hb[kLevels + 1];
    if (threadIdx.x <= kLevels) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * kLvItems;
    uint32_t pos[kLvItems];
    uint8_t lev[kLvItems];
#pragma unroll
    for (int k = 0; k < kLvItems; ++k) {
        const int64_t id = base + (int64_t)k * blockDim.x + threadIdx.x;
        lev[k] = id < m ? nlev[id] : 0;
        pos[k] = id < m ? atomicAdd(&h[lev[k]], 1u) : 0u;
    }
    __syncthreads();
    if (threadIdx.x <= kLevels) hb[threadIdx.x] = h[threadIdx.x] ? atomicAdd(&lcursor[threadIdx.x], h[threadIdx.x]) : 0u;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kLvItems; ++k) {
        const int64_t id = base + (int64_t)k * blockDim.x + threadIdx.x;
        if (id < m) lnodes[loff[lev[k]] + hb[lev[k]] + pos[k]] = (uint32_t)id;
    }
}

// extent of one node of this level after a refit: its cell joined with its
// members' positions, as 32-bit offsets from the cell origin (drift stays
// local across the periodic boundary); the nodes of deeper levels are done
__device__ __forceinline__ void extent_node(
    int64_t n, const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ nend,
    const uint32_t *__restrict__ ncbeg, const uint32_t *__restrict__ occ,
    const uint32_t *__restrict__ child, const uint32_t *__restrict__ px,
    const uint32_t *__restrict__ py, const uint32_t *__restrict__ pz, int64_t nchild,
    const uint32_t *__restrict__ norg, uint32_t *ext_s, uint32_t *ext_l, uint32_t node, int level) {
    const uint32_t o[3] = {norg[3 * node + 0], norg[3 * node + 1], norg[3 * node + 2]};
    const int64_t side = (int64_t)1 << (32 - level);
    int64_t lo[3] = {0, 0, 0}, hi[3] = {side - 1, side - 1, side - 1};
    auto add_point = [&](uint32_t x, uint32_t y, uint32_t z) {
        const int64_t d[3] = {(int64_t)(int32_t)(x - o[0]), (int64_t)(int32_t)(y - o[1]),
                              (int64_t)(int32_t)(z - o[2])};
        for (int a = 0; a < 3; ++a) {
            lo[a] = d[a] < lo[a] ? d[a] : lo[a];
            hi[a] = d[a] > hi[a] ? d[a] : hi[a];
        }
    };
    if (level == kLevels) {
        for (uint32_t q = nbeg[node]; q < nend[node]; ++q) add_point(px[q], py[q], pz[q]);
    } else {
        const uint32_t oc = occ[node];
        const uint32_t cb = ncbeg[node];
        for (int sidx = 0; sidx < 8; ++sidx) {
            const uint32_t slot = cb + __popc(oc & ((1u << sidx) - 1u));
            if (!((oc >> sidx) & 1u) || slot >= (uint64_t)nchild) continue;
            const uint32_t item = child[slot];
            if (item < n) {
                add_point(px[item], py[item], pz[item]);
            } else {
                const int64_t j = item - n;
                for (int a = 0; a < 3; ++a) {
                    const int64_t clo = (int64_t)(int32_t)(ext_s[3 * j + a] - o[a]);
                    const int64_t chi = clo + (int64_t)ext_l[3 * j + a];
                    lo[a] = clo < lo[a] ? clo : lo[a];
                    hi[a] = chi > hi[a] ? chi : hi[a];
                }
            }
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (hi[a] - lo[a] >= (int64_t)0xffffffffll) {
            ext_s[3 * node + a] = 0u;  // the whole circle
            ext_l[3 * node + a] = 0xffffffffu;
        } else {
            ext_s[3 * node + a] = o[a] + (uint32_t)lo[a];
            ext_l[3 * node + a] = (uint32_t)(hi[a] - lo[a]);
        }
    }
}

#define OG_EXTENT_ARGS n, nbeg, nend, ncbeg, occ, child, px, py, pz, nchild, norg, ext_s, ext_l

// one level with many nodes: a thread per node
__global__ void __launch_bounds__(kT) k_extents_level(
    int64_t n, int64_t m, const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ nend,
    const uint32_t *__restrict__ ncbeg, const uint32_t *__restrict__ occ,
    const uint32_t *__restrict__ child, const uint32_t *__restrict__ px,
    const uint32_t *__restrict__ py, const uint32_t *__restrict__ pz, int64_t nchild,
    uint32_t *status, const uint32_t *__restrict__ norg, uint32_t *ext_s, uint32_t *ext_l, int level,
    const uint32_t *__restrict__ lnodes, uint32_t cnt) {
    pdl_wait();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    const uint32_t node = lnodes[k];
    if (node >= (uint64_t)m) {
        atomicOr(status, ST_INTERNAL);
        return;
    }
    extent_node(OG_EXTENT_ARGS, node, level);
}

// consecutive levels with few nodes each, deepest first, in one block: a level
// starts after the block barrier that ends the level below it (the block's
// own global writes are visible to it after the barrier), which saves a
// launch per level
struct LevelRun {
    int lo, hi;                                // levels hi, hi - 1, ..., lo
    uint32_t off[kLevels + 1], cnt[kLevels + 1];
};
constexpr int kRunThreads = 512;
constexpr uint32_t kRunMaxNodes = 256;         // larger levels get a grid of their own

__global__ void __launch_bounds__(kRunThreads) k_extents_run(
    int64_t n, int64_t m, const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ nend,
    const uint32_t *__restrict__ ncbeg, const uint32_t *__restrict__ occ,
    const uint32_t *__restrict__ child, const uint32_t *__restrict__ px,
    const uint32_t *__restrict__ py, const uint32_t *__restrict__ pz, int64_t nchild,
    uint32_t *status, const uint32_t *__restrict__ norg, uint32_t *ext_s, uint32_t *ext_l,
    const uint32_t *__restrict__ lnodes, LevelRun run) {
    pdl_wait();
    for (int l = run.hi; l >= run.lo; --l) {
        for (uint32_t k = threadIdx.x; k < run.cnt[l]; k += blockDim.x) {
            const uint32_t node = lnodes[run.off[l] + k];
            if (node >= (uint64_t)m) {
                atomicOr(status, ST_INTERNAL);
                continue;
            }
            extent_node(OG_EXTENT_ARGS, node, l);
        }
        __syncthreads();
    }
}

// frontier node of p: the deepest node with more than G particles containing
// p (or its box's root); unit: the child of the frontier node that contains p
// (its first particle), or p itself when p hangs directly from it
// the frontier node of particle p (its nearest ancestor above G particles, or
// its box's root) and its unit (the start of the largest ancestor of at most G
// particles below it, or p itself)
__device__ __forceinline__ uint32_t frontier_of(int64_t p, int64_t B, int G, const uint32_t *__restrict__ owner,
                                                const int32_t *__restrict__ npar,
                                                const uint32_t *__restrict__ nbeg,
                                                const uint32_t *__restrict__ nend, int64_t &prev) {
    uint32_t node = owner[p];
    prev = -1;
    for (int guard = 0; node >= (uint64_t)B && nend[node] - nbeg[node] <= (uint32_t)G &&
                        guard <= kLevels + 2;
         ++guard) {
        prev = node;
        node = (uint32_t)npar[node];
    }
    return node;
}

// frontier node and unit of every particle, and the run marks: p where the
// frontier node changes (else 0), for the maximum scan that gives each
// particle the start of its run
__global__ void k_frontier(int64_t n, int64_t B, int G, const uint32_t *__restrict__ owner,
                           const int32_t *__restrict__ npar, const uint32_t *__restrict__ nbeg,
                           const uint32_t *__restrict__ nend, uint32_t *fp, uint32_t *unit, uint32_t *rs) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t pc = p < n ? p : n - 1;          // every lane takes part in the shuffle
    int64_t prev;
    const uint32_t f = frontier_of(pc, B, G, owner, npar, nbeg, nend, prev);
    uint32_t fl = __shfl_up_sync(0xffffffffu, f, 1);
    if ((threadIdx.x & 31) == 0 && pc > 0) {
        int64_t unused;
        fl = frontier_of(pc - 1, B, G, owner, npar, nbeg, nend, unused);
    }
    if (p >= n) return;
    fp[p] = f;
    unit[p] = prev < 0 ? (uint32_t)p : nbeg[prev];
    rs[p] = (p == 0 || f != fl) ? (uint32_t)p : 0u;
}

// group starts: inside a frontier node of at most 8G particles, runs of
// consecutive particles are cut every G; inside a larger frontier node every
// unit (a small child node or a single particle) starts a group of its own
__global__ void k_groupmark(int64_t n, int G, const uint32_t *__restrict__ runstart,
                            const uint32_t *__restrict__ fp, const uint32_t *__restrict__ unit,
                            const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ nend,
                            uint32_t *gs) {
    pdl_wait();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t f = fp[p];
    const bool merge = (uint64_t)(nend[f] - nbeg[f]) <= 8ull * (uint64_t)G;
    if (merge) gs[p] = ((p - runstart[p]) % G == 0) ? 1u : 0u;
    else gs[p] = (unit[p] == (uint32_t)p) ? 1u : 0u;
}

__device__ __forceinline__ void group_box(int64_t n, int64_t ng, int64_t g,
                                          const uint32_t *__restrict__ gbeg, uint32_t *gend,
                                          const uint32_t *__restrict__ px,
                                          const uint32_t *__restrict__ py,
                                          const uint32_t *__restrict__ pz,
                                          const uint32_t *__restrict__ sseg, uint32_t *gbox,
                                          uint32_t *gseg) {
    uint32_t b = gbeg[g];
    gseg[g] = sseg[b];
    uint32_t e = (g + 1 < ng) ? gbeg[g + 1] : (uint32_t)n;
    gend[g] = e;
    // per axis an interval on the circle: member offsets from the first
    // member, min to max (a drifted group may wrap through 0)
    const uint32_t ref[3] = {px[b], py[b], pz[b]};
    int32_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (uint32_t q = b; q < e; ++q) {
        const uint32_t v[3] = {px[q], py[q], pz[q]};
        for (int a = 0; a < 3; ++a) {
            const int32_t d = (int32_t)(v[a] - ref[a]);
            lo[a] = min(lo[a], d);
            hi[a] = max(hi[a], d);
        }
    }
    for (int a = 0; a < 3; ++a) {
        gbox[6 * g + a] = ref[a] + (uint32_t)lo[a];
        gbox[6 * g + 3 + a] = ref[a] + (uint32_t)hi[a];
    }
}


// group ends and boxes; the group count is *d_ng (the build, before the host
// knows it) or ng (a refit)
__global__ void k_group_fin(int64_t n, const uint32_t *__restrict__ d_ng, int64_t ng_host,
                            const uint32_t *__restrict__ gbeg, uint32_t *gend,
                            const uint32_t *__restrict__ px, const uint32_t *__restrict__ py,
                            const uint32_t *__restrict__ pz, const uint32_t *__restrict__ sseg,
                            uint32_t *gbox, uint32_t *gseg) {
    pdl_wait();
    int64_t ng = d_ng ? (int64_t)*d_ng : ng_host;
    if (ng > n) ng = n;                        // the host reports a bad count
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x)
        group_box(n, ng, g, gbeg, gend, px, py, pz, sseg, gbox, gseg);
}

__global__ void k_ext_records(int64_t n, int64_t nchild, const uint32_t *__restrict__ child,
                              const uint32_t *__restrict__ ext_s, const uint32_t *__restrict__ ext_l,
                              CExt *cext) {
    pdl_wait();
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchild) return;
    const uint32_t item = child[c];
    CExt x = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (item >= n) {
        const int64_t j = item - n;
        x = {ext_s[3 * j], ext_s[3 * j + 1], ext_s[3 * j + 2], 0u,
             ext_l[3 * j], ext_l[3 * j + 1], ext_l[3 * j + 2], 0u};
    }
    cext[c] = x;
}

// a built tree's node extents: its cells
__global__ void k_cell_ext(int64_t m, const uint8_t *__restrict__ nlev, const uint32_t *__restrict__ norg,
                           uint32_t *ext_s, uint32_t *ext_l) {
    pdl_wait();
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int L = nlev[j];
    for (int a = 0; a < 3; ++a) {
        ext_s[3 * j + a] = norg[3 * j + a];
        ext_l[3 * j + a] = (uint32_t)((1ull << (32 - L)) - 1ull);
    }
}

// refit: drifted fixed-point positions into sorted order (masses unchanged)
__global__ void k_repos(int64_t n, const uint32_t *__restrict__ perm, const uint4 *__restrict__ q4,
                        uint32_t *px, uint32_t *py, uint32_t *pz) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 q = q4[perm[i]];
    px[i] = q.x;
    py[i] = q.y;
    pz[i] = q.z;
}

// the walk's child records; the child count is *d_nchild (the build) or
// nchild_host (a refit), at most ccap
__global__ void k_records(int64_t n, const uint32_t *__restrict__ d_nchild, int64_t nchild_host,
                          int64_t ccap, const uint32_t *__restrict__ child,
                          const uint32_t *__restrict__ px, const uint32_t *__restrict__ py,
                          const uint32_t *__restrict__ pz, const float *__restrict__ pm32,
                          const double *__restrict__ pm64, const uint8_t *__restrict__ nlev,
                          const uint32_t *__restrict__ ncbeg, const uint32_t *__restrict__ nccnt,
                          const NodeMom *__restrict__ nmom, const uint32_t *__restrict__ ncom,
                          CRec *crec, uint32_t *status) {
    pdl_wait();
    int64_t nchild = d_nchild ? (int64_t)*d_nchild : nchild_host;
    if (nchild > ccap) nchild = ccap;          // the host reports a bad count
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchild;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t item = child[c];
        CRec r;
        if (item < n) {
            r.x = px[item];
            r.y = py[item];
            r.z = pz[item];
            r.m = pm32[item];
            r.M = pm64[item];
            r.info = 0;
            r.ref = item;
        } else {
            int64_t j = item - n;
            r.x = ncom[3 * j + 0];
            r.y = ncom[3 * j + 1];
            r.z = ncom[3 * j + 2];
            r.M = nmom[j].M;
            r.m = __double2float_rn(r.M);
            r.info = (1u << 31) | ((uint32_t)nlev[j] << 26) | (nccnt[j] & 0x3ffffffu);
            r.ref = ncbeg[j];
            // the walk pushes (ref, count) unchecked: a node has children, inside
            // the child array, and is never a root
            if (nccnt[j] == 0u || nccnt[j] > 0x3ffffffu || nlev[j] == 0u || nlev[j] > kLevels ||
                (uint64_t)ncbeg[j] + nccnt[j] > (uint64_t)nchild)
                atomicOr(status, ST_INTERNAL);
        }
        crec[c] = r;
    }
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

// bump allocator inside one device allocation
struct Bump {
    char *base;
    size_t off = 0, cap;
    Bump(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
    template <class T>
    T *take(int64_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += (size_t)(count > 0 ? count : 1) * sizeof(T);
        return p;
    }
};

}  // namespace

// Bytes of the persistent arrays of a forest with n particles in B boxes.
static size_t tree_bytes(int64_t n, int64_t B) {
    int64_t m = n + B;        // nodes: B roots + at most n - B split nodes
    int64_t c = n + m;        // children = n + (m - B)
    size_t b = 0;
    auto add = [&](size_t sz, int64_t cnt) { b += ((size_t)(cnt > 0 ? cnt : 1) * sz + 255) & ~(size_t)255; };
    add(8, n); add(4, n); add(4, n); add(4, n); add(4, n); add(4, n); add(8, n); add(4, n);  // particles
    add(4, n);                                                                      // inv
    add(1, m); add(4, m); add(4, m); add(4, m); add(4, m); add(4, m);               // nlev..npos
    add(4, m); add(4, m); add(4, m); add(32, m); add(4, 3 * m);                     // npar.. ncom
    add(4, n); add(4, n);                                                           // pnext, owner
    add(4, c); add(32, c);                                                          // child, crec
    add(4, n); add(4, n); add(4, 6 * n); add(4, n); add(4, n); add(4, n);           // groups
    add(4, 3 * n); add(4, 3 * n); add(4, n); add(4, n);                             // force arrays
    add(4, B + 1); add(sizeof(SegGeom), B); add(sizeof(WalkParams), 2 * B);         // boxes
    add(4, 3 * m); add(4, m); add(4, m); add(4, 2);                                 // norg nocc lnodes mbits
    return b + 4096;
}

// Node ids by level (t->lnodes) and the count of each level (t->h_lcount),
// for the bottom-up pass over a refit's extents; once per tree.  lcount holds
// 3 (kLevels + 2) words of device scratch.
static og_status level_lists(og_tree *t, uint32_t *lcount) {
    if (!t->h_lcount.empty()) return OG_OK;
    cudaStream_t s = t->ctx->stream;
    const int64_t B = t->nseg, m = t->nnodes;
    uint32_t *loff = lcount + (kLevels + 2), *lcursor = lcount + 2 * (kLevels + 2);
    uint32_t *d_nsplit = lcount + 3 * (kLevels + 2);
    const uint32_t nsplit = (uint32_t)(m - B);
    cudaMemsetAsync(lcount, 0, (kLevels + 2) * sizeof(uint32_t), s);
    cudaMemcpyAsync(d_nsplit, &nsplit, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    const unsigned lv_blocks = (unsigned)((m + (int64_t)kT * kLvItems - 1) / ((int64_t)kT * kLvItems));
    launch_pdl(k_level_hist, lv_blocks, kT, 0, s, d_nsplit, B, t->nlev, lcount);
    launch_pdl(k_level_offsets, 1, 32, 0, s, lcount, loff, lcursor);
    launch_pdl(k_level_scatter, lv_blocks, kT, 0, s, d_nsplit, B, t->nlev, loff, lcursor, t->lnodes);
    uint32_t h[kLevels + 2];
    cudaMemcpyAsync(h, lcount, (kLevels + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "level lists");
    t->h_lcount.assign(h, h + kLevels + 1);
    return OG_OK;
}

// A refit's node extents, level by level from the deepest level up; each level
// reads only nodes of deeper levels, finished by the previous launches (or,
// inside a run of small levels, before the block barrier).
static void extents_bottom_up(og_tree *t, uint32_t *ext_s, uint32_t *ext_l) {
    cudaStream_t s = t->ctx->stream;
    const int64_t n = t->n, m = t->nnodes;
    uint32_t off = 0;
    uint32_t offs[kLevels + 1];
    for (int l = 0; l <= kLevels; ++l) {
        offs[l] = off;
        off += t->h_lcount[l];
    }
    // runs of small levels go to one block each; a large level to a grid
    LevelRun run{};
    run.hi = -1;
    auto flush = [&]() {
        if (run.hi < 0) return;
        launch_pdl(k_extents_run, 1, kRunThreads, 0, s, n, m, t->nbeg, t->nend, t->ncbeg, t->nocc, t->child,
                                                t->px, t->py, t->pz, t->nchild, t->ctx->d_status,
                                                t->norg, ext_s, ext_l, t->lnodes, run);
        run.hi = -1;
    };
    for (int l = kLevels; l >= 0; --l) {
        const uint32_t cnt = t->h_lcount[l];
        if (cnt == 0) continue;
        if (cnt <= kRunMaxNodes) {
            if (run.hi < 0) run.hi = l;
            run.lo = l;
            run.off[l] = offs[l];
            run.cnt[l] = cnt;
            continue;
        }
        flush();
        launch_pdl(k_extents_level, nblk(cnt), kT, 0, s, n, m, t->nbeg, t->nend, t->ncbeg, t->nocc, t->child,
                                                 t->px, t->py, t->pz, t->nchild, t->ctx->d_status,
                                                 t->norg, ext_s, ext_l, l, t->lnodes + offs[l], cnt);
    }
    flush();
}

static og_status alloc_extents(og_tree *t) {
    if (t->cext) return OG_OK;
    cudaStream_t s = t->ctx->stream;
    const int64_t m = t->nnodes;
    cudaError_t err;
    size_t bytes = (size_t)m * 6 * sizeof(uint32_t) + (size_t)t->nchild * sizeof(CExt) + 1024;
    void *p = nullptr;
    if ((err = dev_malloc_async(&p, bytes, s)) != cudaSuccess) return cuda_fail(err, "cudaMallocAsync (extents)");
    t->ext_arena = p;
    t->next_s = static_cast<uint32_t *>(p);
    t->next_l = t->next_s + 3 * m;
    t->cext = reinterpret_cast<CExt *>(reinterpret_cast<char *>(p) +
                                       (((size_t)m * 6 * sizeof(uint32_t) + 255) & ~(size_t)255));
    return OG_OK;
}

// The cell origin of every node: the top L bits of the coordinates of its
// first particle at the build's positions (its box's origin for a root).
// Only the node extents read them, so they are made when extents are first
// needed, before a refit moves the particles.
__global__ void k_cell_origin(int64_t m, int64_t B, const uint8_t *__restrict__ nlev,
                              const uint32_t *__restrict__ nbeg, const uint32_t *__restrict__ px,
                              const uint32_t *__restrict__ py, const uint32_t *__restrict__ pz, uint32_t *norg) {
    pdl_wait();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    if (j < B) {
        norg[3 * j + 0] = norg[3 * j + 1] = norg[3 * j + 2] = 0u;
        return;
    }
    const int L = nlev[j];
    const uint32_t mask = L == 0 ? 0u : ~(uint32_t)((1ull << (32 - L)) - 1ull);
    const uint32_t q = nbeg[j];
    norg[3 * j + 0] = px[q] & mask;
    norg[3 * j + 1] = py[q] & mask;
    norg[3 * j + 2] = pz[q] & mask;
}

static void ensure_origins(og_tree *t) {
    if (t->have_norg) return;
    launch_pdl(k_cell_origin, nblk(t->nnodes), kT, 0, t->ctx->stream, t->nnodes, t->nseg, t->nlev, t->nbeg,
               t->px, t->py, t->pz, t->norg);
    t->have_norg = true;
}

og_status cell_extents(og_tree *t) {
    og_status st = alloc_extents(t);
    if (st) return st;
    ensure_origins(t);
    cudaStream_t s = t->ctx->stream;
    launch_pdl(k_cell_ext, nblk(t->nnodes), kT, 0, s, t->nnodes, t->nlev, t->norg, t->next_s, t->next_l);
    launch_pdl(k_ext_records, nblk(t->nchild), kT, 0, s, t->n, t->nchild, t->child, t->next_s, t->next_l,
                                                 t->cext);
    return OG_OK;
}

// grid of a grid-stride kernel over at most `bound` items
static unsigned stride_grid(int64_t bound) {
    const int64_t b = (bound + kT - 1) / kT;
    return (unsigned)(b < 1 ? 1 : b > 4096 ? 4096 : b);
}

og_status refit_tree(og_tree *t, const double *d_pos) {
    cudaStream_t s = t->ctx->stream;
    const int64_t n = t->n, B = t->nseg;
    cudaError_t err;
    if (!t->cext) {
        // extents live in their own allocation, made on the first refit
        og_status st = alloc_extents(t);
        if (st) return st;
    }
    ensure_origins(t);   // from the build's positions, before k_repos moves them
    const size_t mom_bytes = moments_scratch_bytes(n);
    size_t sb = (size_t)n * (16 + 8 + 4 + 4) + 4096 + mom_bytes + 4 * (kLevels + 3) * sizeof(uint32_t) + 256;
    void *scratch = nullptr;
    if ((err = dev_malloc_async(&scratch, sb, s)) != cudaSuccess) return cuda_fail(err, "cudaMallocAsync (refit)");
    Bump W(scratch, sb);
    uint4 *q4 = W.take<uint4>(n);
    uint64_t *keys = W.take<uint64_t>(n);
    uint32_t *idx = W.take<uint32_t>(n);
    uint32_t *pseg = W.take<uint32_t>(n);
    uint32_t *lcount = W.take<uint32_t>(4 * (kLevels + 3));
    void *mom_scratch = W.take<char>((int64_t)mom_bytes);
    og_status st = level_lists(t, lcount);
    if (st) {
        cudaFreeAsync(scratch, s);
        return st;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (B > 1) {
        launch_pdl(k_fill_seg, nblk(n), kT, 0, s, n, B, t->seg_off, pseg);
    }
    launch_pdl(k_quantize_keys, nblk(n), kT, 0, s, d_pos, n, B > 1 ? pseg : nullptr, t->geom, q4,
                                           keys, nullptr, idx, nullptr, nullptr, nullptr, nullptr, (int64_t)0,
                                           t->ctx->d_status);
    launch_pdl(k_repos, nblk(n), kT, 0, s, n, t->perm, (const uint4 *)q4, t->px, t->py, t->pz);
    node_moments(t, nullptr, t->nnodes, mom_scratch, s);
    extents_bottom_up(t, t->next_s, t->next_l);
    launch_pdl(k_group_fin, stride_grid(t->ngroups), kT, 0, s, n, nullptr, t->ngroups, t->gbeg, t->gend, t->px,
                                                       t->py, t->pz, t->sseg, t->gbox, t->gseg);
    launch_pdl(k_records, stride_grid(t->nchild), kT, 0, s, n, nullptr, t->nchild, t->nchild, t->child, t->px,
                                                    t->py, t->pz, t->pm32, t->pm64, t->nlev, t->ncbeg,
                                                    t->nccnt, t->nmom, t->ncom, t->crec, t->ctx->d_status);
    launch_pdl(k_ext_records, nblk(t->nchild), kT, 0, s, n, t->nchild, t->child, t->next_s, t->next_l,
                                                 t->cext);
    cudaEventRecord(e1, s);
    cudaFreeAsync(scratch, s);
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(err, "refit");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    t->ms_refit = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->refit = true;
    return OG_OK;
}

og_status build_tree(og_tree *t, const double *d_pos, const double *d_mass) {
    cudaStream_t s = t->ctx->stream;
    const int64_t n = t->n;
    const int64_t B = t->nseg;
    cudaError_t err;

    // ---- persistent arrays
    size_t tb = tree_bytes(n, B);
    if ((err = dev_malloc_async(&t->arena, tb, s)) != cudaSuccess) {
        t->arena = nullptr;
        return err == cudaErrorMemoryAllocation ? (set_error("device allocation of %zu bytes failed", tb), OG_ERR_OOM)
                                                : cuda_fail(err, "cudaMallocAsync");
    }
    t->arena_bytes = tb;
    Bump A(t->arena, tb);
    const int64_t mcap = n + B, ccap = n + mcap;
    t->skey = A.take<uint64_t>(n);
    t->perm = A.take<uint32_t>(n);
    t->inv = A.take<uint32_t>(n);
    t->px = A.take<uint32_t>(n);
    t->py = A.take<uint32_t>(n);
    t->pz = A.take<uint32_t>(n);
    t->pm32 = A.take<float>(n);
    t->pm64 = A.take<double>(n);
    t->sseg = A.take<uint32_t>(n);
    t->nlev = A.take<uint8_t>(mcap);
    t->nbeg = A.take<uint32_t>(mcap);
    t->nend = A.take<uint32_t>(mcap);
    t->ncbeg = A.take<uint32_t>(mcap);
    t->nccnt = A.take<uint32_t>(mcap);
    t->npos = A.take<uint32_t>(mcap);
    t->npar = A.take<int32_t>(mcap);
    t->nnext = A.take<int32_t>(mcap);
    t->nsib = A.take<int32_t>(mcap);
    t->nmom = A.take<NodeMom>(mcap);
    t->ncom = A.take<uint32_t>(3 * mcap);
    t->pnext = A.take<int32_t>(n);
    t->owner = A.take<uint32_t>(n);
    t->child = A.take<uint32_t>(ccap);
    t->crec = A.take<CRec>(ccap);
    t->gbeg = A.take<uint32_t>(n);
    t->gend = A.take<uint32_t>(n);
    t->gbox = A.take<uint32_t>(6 * n);
    t->gcost = A.take<uint32_t>(n);
    t->gorder = A.take<uint32_t>(n);
    t->gseg = A.take<uint32_t>(n);
    t->a_sorted = A.take<float>(3 * n);
    t->a_old_sorted = A.take<float>(3 * n);
    t->npp_sorted = A.take<uint32_t>(n);
    t->npn_sorted = A.take<uint32_t>(n);
    t->seg_off = A.take<uint32_t>(B + 1);
    t->geom = A.take<SegGeom>(B);
    t->segp = A.take<WalkParams>(2 * B);
    t->norg = A.take<uint32_t>(3 * mcap);
    t->nocc = A.take<uint32_t>(mcap);
    t->lnodes = A.take<uint32_t>(mcap);
    t->mbits = A.take<int>(2);
    if (A.off > tb) { set_error("internal: arena overflow"); return OG_ERR_STATE; }

    // ---- box table
    {
        // the host copies live in the tree, which outlives the asynchronous
        // copies, so the stream need not be drained here
        std::vector<SegGeom> &hg = t->h_geom;
        hg.assign((size_t)B, SegGeom{});
        for (int64_t b = 0; b < B; ++b) {
            int e2 = 0;
            hg[b].box = t->seg_prm[b].box;
            hg[b].inv_box = 1.0 / t->seg_prm[b].box;
            hg[b].pow2 = std::frexp(t->seg_prm[b].box, &e2) == 0.5 ? 1 : 0;
            hg[b].shift = 33 - e2;   // box = 2^(e2 - 1): x / box * 2^32 = x * 2^(33 - e2)
        }
        cudaMemcpyAsync(t->seg_off, t->h_seg_off.data(), (B + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(t->geom, hg.data(), B * sizeof(SegGeom), cudaMemcpyHostToDevice, s);
    }

    // ---- scratch
    size_t sb_bytes = 0;
    {
        auto add = [&](size_t sz, int64_t cnt) { sb_bytes += ((size_t)(cnt > 0 ? cnt : 1) * sz + 255) & ~(size_t)255; };
        add(16, n);                                             // q4
        add(8, n); add(4, n); add(8, n); add(4, n); add(8, n); add(4, n);  // keys, idx, alt, key copy, pseg
        add(1, n); add(4, n); add(4, n); add(4, n); add(4, n); add(4, n);  // lv sb se first nid sid
        add(4, 4 * kNT * ((n + kSplitTile - 1) / kSplitTile));  // split tile summaries
        add(8, (int64_t)scan_look_words(n + B) + 2);            // scans' look words, counters
        add(4, n + B);                  // nnc
        add(4, n); add(4, n); add(4, n); add(4, n);  // fp rs gs unit
        sb_bytes += radix_sort_scratch_bytes(n) + scan_scratch_bytes(2 * n + B + 8) +
                    moments_scratch_bytes(n) + 4096;
    }
    void *scratch = nullptr;
    if ((err = dev_malloc_async(&scratch, sb_bytes, s)) != cudaSuccess)
        return err == cudaErrorMemoryAllocation ? (set_error("device allocation of %zu bytes failed", sb_bytes), OG_ERR_OOM)
                                                : cuda_fail(err, "cudaMallocAsync");
    Bump W(scratch, sb_bytes);
    uint4 *q4 = W.take<uint4>(n);
    uint64_t *keys = W.take<uint64_t>(n);
    uint32_t *idx = W.take<uint32_t>(n);
    uint64_t *keys_alt = W.take<uint64_t>(n);
    uint32_t *idx_alt = W.take<uint32_t>(n);
    uint64_t *key0 = W.take<uint64_t>(n);
    uint32_t *pseg = W.take<uint32_t>(n);
    uint8_t *lv = W.take<uint8_t>(n);
    uint32_t *sbeg = W.take<uint32_t>(n), *send = W.take<uint32_t>(n);
    uint32_t *first = W.take<uint32_t>(n), *nid = W.take<uint32_t>(n), *sid = W.take<uint32_t>(n);
    int *tsum = W.take<int>(4 * kNT * ((n + kSplitTile - 1) / kSplitTile));
    // the four one-kernel scans of the build share these look words (tags 1-4);
    // their tile counters are the last two words (four 32-bit counters)
    const int64_t nlook_w = (int64_t)scan_look_words(n + B);
    unsigned long long *scan_look = W.take<unsigned long long>(nlook_w + 2);
    const int64_t nlook = nlook_w + 2;
    uint32_t *scan_ctr = reinterpret_cast<uint32_t *>(scan_look + nlook_w);
    uint32_t *occ = t->nocc, *nnc = W.take<uint32_t>(n + B);
    uint32_t *fp = W.take<uint32_t>(n), *rs = W.take<uint32_t>(n), *gs = W.take<uint32_t>(n);
    // a split's previous split in its node: needed only until k_node_init,
    // long before the groups' first use of fp
    uint32_t *prevle = fp;
    uint32_t *unit = W.take<uint32_t>(n);
    void *sort_scratch = W.take<char>((int64_t)radix_sort_scratch_bytes(n));
    void *scan_scratch = W.take<char>((int64_t)scan_scratch_bytes(2 * n + B + 8));
    void *mom_scratch = W.take<char>((int64_t)moments_scratch_bytes(n));
    uint32_t *d_tot = W.take<uint32_t>(4);
    uint32_t *status = t->ctx->d_status;

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);

    // a1, a2
    if (B > 1) {
        launch_pdl(k_fill_seg, nblk(n), kT, 0, s, n, B, t->seg_off, pseg);
    }
    // the masses are checked where they are first read (k_permute), so that a
    // host copy of them can still be in flight here
    // one box: the keys and the permutation are sorted in place in the tree
    if (B == 1) {
        keys = t->skey;
        idx = t->perm;
    }
    launch_pdl(k_quantize_keys, nblk(n), kT, 0, s, d_pos, n, B > 1 ? pseg : nullptr, t->geom, q4,
                                           keys, B > 1 ? key0 : nullptr, idx, B > 1 ? nullptr : t->sseg,
                                           d_tot, t->mbits, scan_look, nlook, status);
    // a3: by key, then (several boxes) stably by box
    bool in_alt = false;
    radix_sort_pairs(keys, idx, keys_alt, idx_alt, n, 63, sort_scratch, s, &in_alt, status);
    if (B > 1) {
        uint32_t *perm1 = in_alt ? idx_alt : idx;
        uint64_t *segkey = in_alt ? keys : keys_alt;      // the free key buffer
        uint64_t *segkey_alt = in_alt ? keys_alt : keys;
        uint32_t *perm1_alt = in_alt ? idx : idx_alt;
        launch_pdl(k_seg_keys, nblk(n), kT, 0, s, n, perm1, pseg, segkey);
        int bits = 1;
        while ((1ll << bits) < B) ++bits;
        bool alt2 = false;
        radix_sort_pairs(segkey, perm1, segkey_alt, perm1_alt, n, bits, sort_scratch, s, &alt2, status);
        const uint32_t *perm_src = alt2 ? perm1_alt : perm1;
        cudaMemcpyAsync(t->perm, perm_src, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        launch_pdl(k_gather_keys, nblk(n), kT, 0, s, n, t->perm, key0, pseg, t->skey, t->sseg);
    } else if (in_alt) {
        // an odd number of passes left the result in the other buffers
        cudaMemcpyAsync(t->skey, keys_alt, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(t->perm, idx_alt, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
    if (t->mass_ready) cudaStreamWaitEvent(s, t->mass_ready, 0);
    launch_pdl(k_permute, nblk(n), kT, 0, s, n, t->perm, (const uint4 *)q4, d_mass, t->px, t->py, t->pz, t->pm32,
                                     t->pm64, t->inv, t->mbits, status);
    // a4: nodes from splits.  The node count stays on the device (d_tot[0]
    // counts the first splits, m = B + that): the kernels up to the groups
    // read it there and are sized for the most nodes a tree can have, so the
    // host does not wait for it.
    uint32_t h_tot[4] = {0, 0, 0, 0};
    int64_t nsplit = n - 1;
    if (nsplit > 0) {
        const int64_t ntiles = (nsplit + kSplitTile - 1) / kSplitTile;
        int *tlast = tsum, *tfirst = tsum + ntiles * kNT;
        int *clast = tsum + 2 * ntiles * kNT, *cfirst = tsum + 3 * ntiles * kNT;
        launch_pdl(k_split_tiles, dim3((unsigned)ntiles), kSplitTile, 0, s, t->skey, t->sseg, nsplit, lv, tlast,
                   tfirst);
        launch_pdl(k_split_carry, dim3(kNT), kSplitTile, 0, s, ntiles, (const int *)tlast, (const int *)tfirst,
                   clast, cfirst);
        launch_pdl(k_split_ranges, dim3((unsigned)ntiles), kSplitTile, 0, s, (const uint8_t *)lv, nsplit,
                   (const int *)clast, (const int *)cfirst, sbeg, send, first, prevle);
        scan_exclusive_u32_look(first, nid, nsplit, d_tot, scan_look, scan_ctr + 0, 1, status, scan_scratch, s);
    }
    const uint32_t *nsp = d_tot;
    // (mcap = n + B covers the splits and the roots too.)  Child counts beyond
    // the last node stay 0, so the scan over mcap entries gives the nodes'
    // child offsets and, as its total, the child entries.
    launch_pdl(k_node_init, nblk(mcap), kT, 0, s, n, B, t->seg_off, first, nid, lv, sbeg, send, prevle,
               t->sseg, t->nlev, t->nbeg, t->nend, sid, mcap, occ, nnc, t->nccnt,
               status);
    launch_pdl(k_link, nblk(n + mcap), kT, 0, s, n, nsp, B, t->skey, lv, sid, t->sseg, t->nlev, t->nbeg,
                                         t->nend, t->npar, t->owner, occ, nnc, status);
    launch_pdl(k_ccnt, nblk(mcap), kT, 0, s, nsp, B, t->nlev, t->nbeg, t->nend, occ, t->nccnt);
    scan_exclusive_u32_look(t->nccnt, t->ncbeg, mcap, d_tot + 1, scan_look, scan_ctr + 1, 2, status, scan_scratch, s);
    launch_pdl(k_place, nblk(n + mcap), kT, 0, s, n, nsp, B, t->skey, t->nlev, t->nbeg, t->ncbeg, occ,
                                          t->npar, t->owner, t->child, t->npos, status);
    launch_pdl(k_threading, nblk(ccap), kT, 0, s, n, nsp, B, t->child, t->ncbeg, t->nccnt, t->npar,
                                          t->npos, t->owner, t->nnext, t->nsib, t->pnext, status);
    // a5: exact moments and centres of mass of every node (in units fixed by
    // the masses' set-bit span, which k_permute gathered)
    node_moments(t, nsp, mcap, mom_scratch, s);
    // a6: groups (one group size for the whole forest)
    const int G = t->prm.group_max;
    launch_pdl(k_frontier, nblk(n), kT, 0, s, n, B, G, t->owner, t->npar, t->nbeg, t->nend, fp, unit, rs);
    scan_inclusive_max_u32_look(rs, rs, n, scan_look, scan_ctr + 2, 3, status, scan_scratch, s);
    launch_pdl(k_groupmark, nblk(n), kT, 0, s, n, G, rs, fp, unit, t->nbeg, t->nend, gs);
    // group starts, compacted into gbeg; their count to d_tot[2]
    scan_compact_u32_look(gs, t->gbeg, n, d_tot + 2, scan_look, scan_ctr + 3, 4, status, scan_scratch, s);
    // group count (d_tot[2]) and child count (d_tot[1]) from the device
    launch_pdl(k_group_fin, stride_grid(n), kT, 0, s, n, d_tot + 2, 0, t->gbeg, t->gend, t->px, t->py, t->pz,
                                              t->sseg, t->gbox, t->gseg);
    launch_pdl(k_records, stride_grid(ccap), kT, 0, s, n, d_tot + 1, 0, ccap, t->child, t->px, t->py, t->pz,
                                               t->pm32, t->pm64, t->nlev, t->ncbeg, t->nccnt, t->nmom,
                                               t->ncom, t->crec, status);
    cudaEventRecord(e1, s);
    // the counts and the status word, read once the build is complete (its
    // only host synchronisation)
    uint32_t *hc = pinned_counts(t->ctx), *hs = pinned_status(t->ctx);
    cudaMemcpyAsync(hc, d_tot, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hs, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(scratch, s);
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(err, "build");
    for (int k = 0; k < 3; ++k) h_tot[k] = hc[k];
    t->build_status = *hs;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    t->ms_build = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((err = cudaGetLastError()) != cudaSuccess) return cuda_fail(err, "build launch");
    const int64_t m = B + (int64_t)h_tot[0];
    if (m > mcap) {
        set_error("internal: node count %lld above its bound %lld", (long long)m, (long long)mcap);
        return OG_ERR_STATE;
    }
    t->nnodes = m;
    const int64_t nchild = n + (m - B);
    t->nchild = nchild;
    if ((int64_t)h_tot[1] != nchild) {
        set_error("internal: child count %u != %lld", h_tot[1], (long long)nchild);
        return OG_ERR_STATE;
    }
    t->ngroups = h_tot[2];
    return OG_OK;
}

}  // namespace og
