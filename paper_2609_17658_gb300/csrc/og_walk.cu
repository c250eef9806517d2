// og_walk.cu -- group-wise tree walk and force evaluation (Sect. 4.1.2, 4.1.3, 4.2).
//
// The paper walks the tree once per target particle with a threaded
// (nextnode / sibling) loop and, on GPUs, processes neighbours in chunks of
// 32.  Here one warp walks the tree once for a whole group of up to 32
// spatially close targets and shares the resulting interaction list:
//
//   list building   the warp keeps a stack of child-array ranges of opened
//                   nodes in shared memory.  Each round the 32 lanes take the
//                   next 64 child records (32-byte records, coalesced loads;
//                   two independent records per lane), and each lane
//                   classifies its records against the group's integer
//                   bounding box:
//                     particle -> PP entry unless beyond the prune distance;
//                     node     -> pruned, opened (range pushed), or PN entry.
//                   Prune and boundary tests are exact integer geometry.  The
//                   Barnes-Hut / relative test is decided in FP32 when the
//                   FP32 value is farther from the threshold than its proven
//                   error bound, and otherwise by the exact FP64 expression
//                   (fixed operation order, no fused operations), so every
//                   decision equals the FP64 decision of the oracle.
//   evaluation      entries (x, y, z, m) go to one of two shared-memory chunks:
//                   "far" entries (integer distance from the group box >= h,
//                   so no target can need the softened kernel) and "near"
//                   entries.  A full chunk is evaluated by every lane for its
//                   target: exact int32 minimum-image separation, converted to
//                   FP32, r^2 by FMA, cutoff, rsqrt, erfc split factor, spline
//                   softening for near entries only, FP32 accumulation over the
//                   chunk, then a compensated (Kahan) add into the totals.
//                   A group of g <= 16 targets replicates each target on
//                   32 / P lanes (P the next power of two >= g) that split the
//                   chunk's entries; the replicas' totals are added in a fixed
//                   order at the end.
//
// Work distribution: persistent blocks; warps take groups from a global
// atomic counter, in decreasing order of the previous pass's list length
// when that is known (longest first shortens the tail of the launch).
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kMaxWarps = 8;       // warps per block: 1..kMaxWarps, chosen at launch
constexpr int kStackCap = 768;     // ranges per warp stack
constexpr int kNearChunk = 64;     // near entries per shared chunk (>= 64: see kMinChunk)
// The far chunk holds `chunk` entries (WalkArgs::chunk, chosen at launch,
// kMinChunk..kMaxChunk): a round adds at most 64 entries to either chunk, so
// a flushed chunk always has room for the next round.
constexpr int kMinChunk = 64, kMaxChunk = 1024;

// shared memory of one warp: its stack, near chunk and far chunk
__host__ __device__ constexpr size_t warp_smem(int chunk) {
    return kStackCap * sizeof(uint2) + ((size_t)chunk + kNearChunk) * sizeof(uint4);
}
constexpr size_t kMaxBlockSmem = kMaxWarps * warp_smem(kMaxChunk);
static_assert(kMaxBlockSmem <= 227 * 1024, "walk block exceeds the shared memory of an SM");

// Abramowitz & Stegun 7.1.26: erfc(x) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
// t = 1 / (1 + p x), |error| <= 1.5e-7 for x >= 0.
constexpr float kAsP = 0.3275911f;
constexpr float kAs1 = 0.254829592f, kAs2 = -0.284496736f, kAs3 = 1.421413741f;
constexpr float kAs4 = -1.453152027f, kAs5 = 1.061405429f;
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

// relative margin of the FP32 opening filter (the FP32 evaluation errs by
// less than 2^-20; inside this band the FP64 expression decides)
constexpr float kFilterHi = 1.0f + 1.0f / 65536.0f;
constexpr float kFilterLo = 1.0f - 1.0f / 65536.0f;

// One tree as the walk sees it (a forest counts as one tree).
struct TreeView {
    int64_t n, ngroups;
    const uint32_t *gbeg, *gend, *gbox;
    const uint32_t *gorder;       // processing order of the groups, or null (key order)
    uint32_t *gcost;              // out: list length per group
    const CRec *crec;
    const CExt *cext;             // node extents after a refit (kRefit), else unused
    int64_t nchild, max_rounds;
    const uint32_t *gseg;         // box of each group
    const uint32_t *ncbeg, *nccnt;  // child range of each node (the roots are nodes 0..B-1)
    const WalkParams *segp;       // per-box parameters
    const uint32_t *px, *py, *pz;
    const float *a_old;           // [3][n] sorted, relative criterion only
    float *acc;                   // [3][n] sorted, out
    float *pot;                   // [n] sorted, out (potential launches only)
    uint32_t *npp, *npn;          // [n] sorted, out
    int has_cost;                 // gcost holds the list lengths of a previous pass
};

struct WalkArgs {
    TreeView tree0;               // the tree of a single-tree launch
    const TreeView *trees;        // several trees: descriptors in device memory
    const uint64_t *goff;         // several trees: first item of each tree, plus the total
    const uint32_t *items;        // several trees: item order (longest list first), or null
    int64_t ntrees, nitems;
    uint32_t *lists;              // debug dump: (group, child slot) pairs
    unsigned long long *list_cursor;
    int64_t list_cap;
    unsigned long long *work;     // item counter
    int warps, chunk;             // launch shape: warps per block, far-chunk entries
    int one_seg;                  // a single tree of one box: its parameters are p0
    WalkParams p0;                // the box's parameters, in the launch's own argument space
    unsigned long long *inter;    // interactions evaluated
    unsigned long long *tree_inter;  // several trees: interactions per tree, or null
    uint32_t *status;
};

// multi-function-unit approximations (PTX .approx with flush-to-zero); the
// operands here are never subnormal: r^2 >= 1 in grid units, see eval_near
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Intervals on the circle of 2^32 grid units are [lo, hi] with length
// hi - lo (mod 2^32); a drifted interval may wrap through 0.
// point c to the interval [lo, lo + len]
__device__ __forceinline__ uint32_t point_gap(uint32_t c, uint32_t lo, uint32_t len) {
    const uint32_t d = c - lo;
    if (d <= len) return 0u;
    const uint32_t fwd = d - len, back = 0u - d;
    return fwd < back ? fwd : back;
}

// interval [alo, alo + la] to interval [blo, blo + lb]
__device__ __forceinline__ uint32_t box_gap(uint32_t alo, uint32_t la, uint32_t blo, uint32_t lb) {
    if (blo - alo <= la || alo - blo <= lb) return 0u;
    const uint32_t a = blo - (alo + la), b = alo - (blo + lb);
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long sq64(uint32_t g) {
    return (unsigned long long)g * (unsigned long long)g;
}

// Near-chunk evaluation for one target per lane (entries closer than h to
// the group box: the softened kernel may apply).  Entries e = rep, rep + R,
// ... are this lane's share.  r^2 is guarded from below by 1 (a nonzero integer
// separation has r^2 >= 1 in grid units); a zero separation then contributes
// f * 0 = 0 exactly, the self term included.
// kPot: also the short-range potential sum of m erfc(r / 2 r_s) psi(r), psi the
// potential kernel of the spline (1/r beyond h); the self term (r = 0) is left
// out explicitly, it has no force to vanish with.
template <bool kSplit, bool kPot = false>
__device__ __forceinline__ void eval_near(const uint4 *ch, int cnt, int rep, int R, uint32_t xi,
                                          uint32_t yi, uint32_t zi, const WalkParams &p,
                                          float &ax, float &ay, float &az, float &ap) {
    const float rc2 = p.rc2, kexp = p.kexp;
    // u = r / (2 r_s) only enters as p u and (2 / sqrt(pi)) u
    const float c_pr = kAsP * p.inv_2rs, c_tspr = kTwoOverSqrtPi * p.inv_2rs;
    const float h = p.h, inv_h = p.inv_h;
    const float hinv3 = inv_h * inv_h * inv_h;
#pragma unroll 2
    for (int e = rep; e < cnt; e += R) {
        const uint4 s = ch[e];
        const float fx = (float)(int)(s.x - xi);
        const float fy = (float)(int)(s.y - yi);
        const float fz = (float)(int)(s.z - zi);
        const float r2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, __fmul_rn(fz, fz)));
        float m = __uint_as_float(s.w);
        if (kSplit) m = (r2 < rc2) ? m : 0.0f;
        const float r2c = fmaxf(r2, 1.0f);
        const float rinv = rsqrt_ftz(r2c);
        float mS = m;
        const float r = r2c * rinv;
        float erfcv = 1.0f;
        if (kSplit) {
            const float t = rcp_ftz(fmaf(c_pr, r, 1.0f));
            const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, kAs5, kAs4), kAs3), kAs2), kAs1);
            const float ex = ex2_ftz(r2c * kexp);
            mS = m * (ex * fmaf(c_tspr, r, poly));
            if (kPot) erfcv = ex * poly;
        }
        if (kPot) {
            float psi = rinv;
            {
                const float u = r * inv_h;
                const float u2 = u * u;
                const float pin = fmaf(u2, fmaf(u2, fmaf(-32.0f / 5.0f, u, 48.0f / 5.0f), -16.0f / 3.0f),
                                       14.0f / 5.0f);
                const float pout = fmaf(u2, fmaf(u, fmaf(u, fmaf(32.0f / 15.0f, u, -48.0f / 5.0f), 16.0f),
                                                 -32.0f / 3.0f),
                                        16.0f / 5.0f) -
                                   (1.0f / 15.0f) * rcp_ftz(u);
                psi = (r < h) ? inv_h * ((u < 0.5f) ? pin : pout) : psi;
            }
            ap = fmaf((r2 > 0.0f ? m : 0.0f) * erfcv, psi, ap);
        }
        float g = rinv * rinv * rinv;
        {
            // cubic-spline softened kernel inside h (Monaghan 1985 form)
            const float u = r * inv_h;
            const float u2 = u * u;
            const float gin = hinv3 * fmaf(u2, fmaf(32.0f, u, -192.0f / 5.0f), 32.0f / 3.0f);
            const float gout = hinv3 * (fmaf(u, fmaf(u, fmaf(u, -32.0f / 3.0f, 192.0f / 5.0f), -48.0f),
                                             64.0f / 3.0f) -
                                        (1.0f / 15.0f) * rcp_ftz(u2 * u));
            g = (r < h) ? ((u < 0.5f) ? gin : gout) : g;
        }
        const float f = mS * g;
        ax = fmaf(f, fx, ax);
        ay = fmaf(f, fy, ay);
        az = fmaf(f, fz, az);
    }
}

// Far entries: every target of the group is at least h away (the entry lies
// outside the group box by more than h, and by at least one grid unit), so
// no softening applies and r^2 >= 1 needs no guard.  Two entries of this
// lane's share, e and e + R, go through the arithmetic together as FP32
// pairs (the f32x2 multiply and fused multiply-add of sm_100 and later:
// each half is the same IEEE operation as the scalar one, so the cutoff
// decision is unchanged); an odd last entry goes alone.
template <bool kSplit, bool kPot = false, int kUnroll = 2>
__device__ __forceinline__ void eval_far(const uint4 *ch, int cnt, int rep, int R, uint32_t xi,
                                         uint32_t yi, uint32_t zi, const WalkParams &p,
                                         float &ax, float &ay, float &az, float &ap) {
    const float rc2 = p.rc2;
    const float2 c_kexp = make_float2(p.kexp, p.kexp);
    const float2 c_one = make_float2(1.0f, 1.0f);
    const float2 c5 = make_float2(kAs5, kAs5), c4 = make_float2(kAs4, kAs4);
    const float2 c3 = make_float2(kAs3, kAs3), c2 = make_float2(kAs2, kAs2);
    const float2 c1 = make_float2(kAs1, kAs1);
    // u = r / (2 r_s) only enters as p u and (2 / sqrt(pi)) u: 1 / (2 r_s) folds into both
    const float2 c_pr = make_float2(kAsP * p.inv_2rs, kAsP * p.inv_2rs);
    const float2 c_tspr = make_float2(kTwoOverSqrtPi * p.inv_2rs, kTwoOverSqrtPi * p.inv_2rs);
    float2 sx = make_float2(0.f, 0.f), sy = sx, sz = sx, sp = sx;
    int e = rep;
#pragma unroll kUnroll
    for (; e + R < cnt; e += 2 * R) {
        const uint4 s0 = ch[e], s1 = ch[e + R];
        const float2 fx = make_float2((float)(int)(s0.x - xi), (float)(int)(s1.x - xi));
        const float2 fy = make_float2((float)(int)(s0.y - yi), (float)(int)(s1.y - yi));
        const float2 fz = make_float2((float)(int)(s0.z - zi), (float)(int)(s1.z - zi));
        const float2 r2 = __ffma2_rn(fx, fx, __ffma2_rn(fy, fy, __fmul2_rn(fz, fz)));
        float2 m = make_float2(__uint_as_float(s0.w), __uint_as_float(s1.w));
        if (kSplit) {
            m.x = (r2.x < rc2) ? m.x : 0.0f;
            m.y = (r2.y < rc2) ? m.y : 0.0f;
        }
        const float2 rinv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
        float2 f;
        if (kSplit) {
            // S(r) r^-3 = (erfc(u) + (2 / sqrt(pi)) u exp(-u^2)) r^-3, with the
            // second term's r r^-1 taken as 1: (poly rinv + c) exp(-u^2) rinv^2
            const float2 r = __fmul2_rn(r2, rinv);
            const float2 den = __ffma2_rn(c_pr, r, c_one);
            const float2 t = make_float2(rcp_ftz(den.x), rcp_ftz(den.y));
            float2 q = __ffma2_rn(t, c5, c4);
            q = __ffma2_rn(t, q, c3);
            q = __ffma2_rn(t, q, c2);
            q = __ffma2_rn(t, q, c1);
            const float2 poly = __fmul2_rn(t, q);
            const float2 arg = __fmul2_rn(r2, c_kexp);
            const float2 ex = make_float2(ex2_ftz(arg.x), ex2_ftz(arg.y));
            const float2 mex = __fmul2_rn(m, ex);
            if (kPot) sp = __ffma2_rn(__fmul2_rn(mex, poly), rinv, sp);
            f = __fmul2_rn(mex, __fmul2_rn(__ffma2_rn(poly, rinv, c_tspr), __fmul2_rn(rinv, rinv)));
        } else {
            if (kPot) sp = __ffma2_rn(m, rinv, sp);
            f = __fmul2_rn(m, __fmul2_rn(rinv, __fmul2_rn(rinv, rinv)));
        }
        sx = __ffma2_rn(f, fx, sx);
        sy = __ffma2_rn(f, fy, sy);
        sz = __ffma2_rn(f, fz, sz);
    }
    float tx = __fadd_rn(sx.x, sx.y), ty = __fadd_rn(sy.x, sy.y), tz = __fadd_rn(sz.x, sz.y);
    float tp = kPot ? __fadd_rn(sp.x, sp.y) : 0.0f;
    if (e < cnt) {
        const uint4 s = ch[e];
        const float fx = (float)(int)(s.x - xi);
        const float fy = (float)(int)(s.y - yi);
        const float fz = (float)(int)(s.z - zi);
        const float r2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, __fmul_rn(fz, fz)));
        float m = __uint_as_float(s.w);
        if (kSplit) m = (r2 < rc2) ? m : 0.0f;
        const float rinv = rsqrt_ftz(r2);
        float f;
        if (kSplit) {
            const float r = r2 * rinv;
            const float t = rcp_ftz(fmaf(c_pr.x, r, 1.0f));
            const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, kAs5, kAs4), kAs3), kAs2), kAs1);
            const float ex = ex2_ftz(r2 * p.kexp);
            const float mex = m * ex;
            if (kPot) tp = fmaf(mex * poly, rinv, tp);
            f = mex * (fmaf(poly, rinv, c_tspr.x) * (rinv * rinv));
        } else {
            if (kPot) tp = fmaf(m, rinv, tp);
            f = m * (rinv * (rinv * rinv));
        }
        tx = fmaf(f, fx, tx);
        ty = fmaf(f, fy, ty);
        tz = fmaf(f, fz, tz);
    }
    ax = tx;
    ay = ty;
    az = tz;
    if (kPot) ap = tp;
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v) {
    const float y = __fsub_rn(v, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

struct Acc {
    float sx = 0.f, sy = 0.f, sz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
    __device__ __forceinline__ void add(float tx, float ty, float tz) {
        kahan_add(sx, kx, tx);
        kahan_add(sy, ky, ty);
        kahan_add(sz, kz, tz);
    }
};

// The squared distance of the gaps (gx, gy, gz) in single precision: each
// gap rounded once, then fma(fx, fx, fma(fy, fy, fz * fz)).  Its relative
// error is below 5 * 2^-24.
__device__ __forceinline__ float dist2f(uint32_t gx, uint32_t gy, uint32_t gz) {
    const float fx = (float)gx, fy = (float)gy, fz = (float)gz;
    return fmaf(fx, fx, fmaf(fy, fy, fz * fz));
}

// Barnes-Hut: open iff l2 > th2 * d2 with d2 = (dx*dx + dy*dy) + dz*dz in FP64.
// The FP32 value d2f decides when it is farther from the threshold than its
// error bound; inside that band the FP64 expression does.
__device__ __forceinline__ bool open_bh(uint32_t gx, uint32_t gy, uint32_t gz, float d2f, float l2f,
                                        double l2, const WalkParams &p) {
    const float q = p.th2f * d2f;
    if (l2f > q * kFilterHi) return true;
    if (l2f < q * kFilterLo) return false;
    const double dx = (double)gx, dy = (double)gy, dz = (double)gz;
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return l2 > __dmul_rn(p.th2, d2);
}

// relative: open iff (G M) l2 > arel (d2 d2), arel = (alpha a_min) s^2, in FP64.
__device__ __forceinline__ bool open_rel(uint32_t gx, uint32_t gy, uint32_t gz, float d2f, float l2f,
                                         double l2, float Mf, double M, float arelf, double arel,
                                         const WalkParams &p) {
    const float lhs = (p.Gf * Mf) * l2f;
    const float rhs = (arelf * d2f) * d2f;
    const bool normal = lhs >= 1e-30f && lhs <= 1e30f && rhs >= 1e-30f && rhs <= 1e30f;
    if (normal) {
        if (lhs > rhs * kFilterHi) return true;
        if (lhs < rhs * kFilterLo) return false;
    }
    const double dx = (double)gx, dy = (double)gy, dz = (double)gz;
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return __dmul_rn(__dmul_rn(p.G, M), l2) > __dmul_rn(arel, __dmul_rn(d2, d2));
}

// Gap between a node's cell and the group box on one axis, from the cell's
// centre c (cell [c - s2, c + s2 - 1], s2 = half the side).  d = c - lo on
// the circle; outside the box the centre is fwd = d - len past its far end or
// back = -d before its near end.  The centre's own gap is dc = min(fwd, back)
// (0 inside); the cell's gap is dc - s2 when the box lies before the cell
// (fwd side) and dc - s2 + 1 when it lies after it (back side, the cell ends
// at c + s2 - 1), and 0 when that is not positive (they meet).  Equal to the
// interval gap of the cell and the box, exactly.
__device__ __forceinline__ void cell_gap(uint32_t c, uint32_t lo, uint32_t len, uint32_t s2,
                                         uint32_t &dc, uint32_t &cg) {
    const uint32_t d = c - lo;
    const uint32_t fwd = d - len, back = 0u - d;
    const bool inside = d <= len;
    const bool onback = back < fwd;
    dc = inside ? 0u : (onback ? back : fwd);
    const int e = (int)(dc - s2 + (onback ? 1u : 0u));
    cg = e > 0 ? (uint32_t)e : 0u;
}

// Registers: at most 96 per thread (64 KB / (96 x 128) gives 5 blocks of 4
// warps per SM, as many as their shared memory allows), 128 with the
// potential output; a block of kMaxWarps warps fits either way.
// One child record against the group box: PP / PN entry, opened node (its
// child range to push), or nothing (pruned, or no record in this slot).
struct Cls {
    bool emit, open, isnode, near;
    uint4 ent;
    uint32_t push_ref, push_cnt;
};

template <int kOpen, bool kSplit, bool kRefit>
__device__ __forceinline__ Cls classify(const TreeView &T, uint32_t ci, bool has, const uint32_t *lo,
                                        const uint32_t *gl, const WalkParams &p, float arelf,
                                        double arel) {
    bool emit = false, open = false, isnode = false, near = false;
    uint4 ent = make_uint4(0u, 0u, 0u, 0u);
    uint32_t push_ref = 0u, push_cnt = 0u;
    if (has && ci < T.nchild) {
        const CRec r = T.crec[ci];
        ent = make_uint4(r.x, r.y, r.z, __float_as_uint(r.m));
        isnode = (r.info >> 31) != 0u;
        // gaps of the particle, or of the node's centre of mass, to the group box
        const uint32_t gx = point_gap(r.x, lo[0], gl[0]);
        const uint32_t gy = point_gap(r.y, lo[1], gl[1]);
        const uint32_t gz = point_gap(r.z, lo[2], gl[2]);
        if (!isnode) {
            const unsigned long long pg2 = sq64(gx) + sq64(gy) + sq64(gz);
            near = pg2 < p.hnear2;
            emit = !kSplit || pg2 <= p.rprune;
        } else {
            bool pruned = false, bnear;
            float l2f;
            double l2;
            if (kRefit) {
                // the node's extent: its cell joined with its drifted members
                const CExt e = T.cext[ci];
                const unsigned long long ell =
                    (unsigned long long)max(e.lx, max(e.ly, e.lz)) + 1ull;
                l2 = (double)ell * (double)ell;
                l2f = (float)l2;
                if (kSplit) {
                    const unsigned long long g2 = sq64(box_gap(lo[0], gl[0], e.sx, e.lx)) +
                                                  sq64(box_gap(lo[1], gl[1], e.sy, e.ly)) +
                                                  sq64(box_gap(lo[2], gl[2], e.sz, e.lz));
                    pruned = g2 > p.rprune;
                }
                // boundary check: the box meets the cube of side 1.2 ell
                // centred on the extent: 10 g <= 6 ell, i.e. g <= floor(3 ell / 5)
                // (ell <= 2^32, so the limit fits in 32 bits)
                const uint32_t blim = (uint32_t)((3ull * ell) / 5ull);
                bnear = point_gap(e.sx + (uint32_t)(((unsigned long long)e.lx + 1ull) >> 1), lo[0], gl[0]) <= blim &&
                        point_gap(e.sy + (uint32_t)(((unsigned long long)e.ly + 1ull) >> 1), lo[1], gl[1]) <= blim &&
                        point_gap(e.sz + (uint32_t)(((unsigned long long)e.lz + 1ull) >> 1), lo[2], gl[2]) <= blim;
            } else {
                // the node's cell, from its level and centre of mass: half side
                // s2 = 2^(31 - lev), centre = (COM with the low 32 - lev bits
                // cleared) + s2
                const uint32_t lev = (r.info >> 26) & 31u;
                const uint32_t s2 = 0x80000000u >> lev;
                const uint32_t keep = ~(2u * s2 - 1u);
                l2f = __uint_as_float((uint32_t)(127 + 64 - 2 * lev) << 23);
                l2 = __longlong_as_double((long long)(1023 + 64 - 2 * lev) << 52);
                uint32_t dcx, dcy, dcz, cgx, cgy, cgz;
                cell_gap((r.x & keep) | s2, lo[0], gl[0], s2, dcx, cgx);
                cell_gap((r.y & keep) | s2, lo[1], gl[1], s2, dcy, cgy);
                cell_gap((r.z & keep) | s2, lo[2], gl[2], s2, dcz, cgz);
                if (kSplit) pruned = sq64(cgx) + sq64(cgy) + sq64(cgz) > p.rprune;
                // boundary check: the box meets the cell enlarged to 0.6 side,
                // 10 dc <= 6 side, i.e. dc <= floor(6 s2 / 5) = s2 + floor(s2 / 5)
                const uint32_t blim = s2 + (__umulhi(s2, 0xCCCCCCCDu) >> 2);
                bnear = dcx <= blim && dcy <= blim && dcz <= blim;
            }
            if (!pruned) {
                const float d2f = dist2f(gx, gy, gz);
                if (bnear) {
                    open = true;
                } else {
                    if (kOpen == OG_OPEN_BH) open = open_bh(gx, gy, gz, d2f, l2f, l2, p);
                    else open = open_rel(gx, gy, gz, d2f, l2f, l2, r.m, r.M, arelf, arel, p);
                }
                emit = !open;
                // conservative: in single precision with a margin above its error
                near = !(d2f >= p.hnear2f);
                push_ref = r.ref;
                push_cnt = r.info & 0x3ffffffu;
            }
        }
    }
    return Cls{emit, open, isnode, near, ent, push_ref, push_cnt};
}

// kOneSeg: a single tree of one box, whose parameters come from the launch
// argument (constant operands) instead of a per-box record in global memory.
template <int kOpen, bool kSplit, bool kDump, bool kRefit, bool kMulti, bool kPot = false,
          bool kOneSeg = false>
__global__ void __maxnreg__(kPot ? 128 : 96) k_walk(WalkArgs a);

template <int kOpen, bool kSplit, bool kDump, bool kRefit, bool kMulti, bool kPot, bool kOneSeg>
__global__ void __maxnreg__(kPot ? 128 : 96) k_walk(WalkArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: per warp, its stack, near chunk and far chunk (warp_smem bytes);
    // blockDim.x = 32 * a.warps and the launch sizes smem to match
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int chunk = a.chunk;
    // far-entry pairs in flight per lane: 4 in the Barnes-Hut kernels and in
    // the one-box kernels (their parameters are constant operands), 2 where
    // the relative test's extra registers would spill
    constexpr int kFarUnroll = (kOpen == OG_OPEN_BH || kOneSeg) ? 4 : 2;
    unsigned char *wbase = smem + (size_t)warp * warp_smem(chunk);
    uint2 *stk = reinterpret_cast<uint2 *>(wbase);
    uint4 *chn = reinterpret_cast<uint4 *>(wbase + kStackCap * sizeof(uint2));
    uint4 *chf = chn + kNearChunk;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;

    while (true) {
        unsigned long long gq = 0;
        if (lane == 0) gq = atomicAdd(a.work, 1ull);
        gq = __shfl_sync(FULL, gq, 0);
        int64_t g;
        int64_t ti = 0;
        if (kMulti) {
            if (gq >= (unsigned long long)a.nitems) break;
            const uint64_t item = a.items ? a.items[gq] : gq;
            int64_t lo_t = 0, hi_t = a.ntrees;  // goff[lo_t] <= item < goff[hi_t]
            while (hi_t - lo_t > 1) {
                const int64_t mid = (lo_t + hi_t) >> 1;
                if (a.goff[mid] <= item) lo_t = mid; else hi_t = mid;
            }
            ti = lo_t;
            g = (int64_t)(item - a.goff[ti]);
        } else {
            if (gq >= (unsigned long long)a.tree0.ngroups) break;
            g = a.tree0.gorder ? (int64_t)a.tree0.gorder[gq] : (int64_t)gq;
        }
        const TreeView &T = kMulti ? a.trees[ti] : a.tree0;
        const uint32_t seg = kOneSeg ? 0u : T.gseg[g];
        const WalkParams &p = kOneSeg ? a.p0 : T.segp[seg];
        const uint32_t gb = T.gbeg[g], ge = T.gend[g];
        const uint32_t gsize = ge - gb;
        uint32_t lo[3], gl[3];  // the group box: [lo, lo + gl] per axis
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = T.gbox[6 * g + k];
            gl[k] = T.gbox[6 * g + 3 + k] - lo[k];
        }
        // lane -> (target, replica): P lanes per replica, R = 32 / P replicas
        const int P = gsize > 16u ? 32 : gsize > 8u ? 16 : gsize > 4u ? 8 : gsize > 2u ? 4 : gsize > 1u ? 2 : 1;
        const int R = 32 / P;
        const int tl = lane & (P - 1), rep = lane / P;
        const uint32_t i = gb + tl;
        const bool active = (uint32_t)tl < gsize;
        const uint32_t xi = active ? T.px[i] : 0u;
        const uint32_t yi = active ? T.py[i] : 0u;
        const uint32_t zi = active ? T.pz[i] : 0u;
        // relative criterion: arel = (alpha * a_min) * s^2, a_min = min over the group
        // of |a_old| in FP64 of the single-precision components
        double arel = 0.0;
        float arelf = 0.0f;
        if (kOpen == OG_OPEN_REL) {
            double an = __longlong_as_double(0x7ff0000000000000ll);  // +inf
            if (active) {
                double ax0 = T.a_old[i], ay0 = T.a_old[T.n + i], az0 = T.a_old[2 * T.n + i];
                an = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ax0, ax0), __dmul_rn(ay0, ay0)),
                                          __dmul_rn(az0, az0)));
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) an = fmin(an, __shfl_xor_sync(FULL, an, d));
            arel = __dmul_rn(__dmul_rn(p.alpha, an), p.s2);
            arelf = __double2float_rn(arel);
        }

        if (lane == 0) stk[0] = make_uint2(T.ncbeg[seg], T.nccnt[seg]);
        __syncwarp();
        int sp = 1, cf = 0, cn = 0;
        int64_t rounds = 0;
        uint32_t cnt_pp = 0, cnt_pn = 0;
        Acc acc;
        float psum = 0.f, pcomp = 0.f;   // potential total (kPot), compensated
        bool overflow = false;

        // the last pass of this loop finds the stack empty: an empty round whose
        // flush evaluates what the chunks still hold (one evaluation site)
        while (true) {
            const bool done = sp == 0;
            // every round consumes at least one child record and a record is
            // visited at most once per walk: more rounds than records is a bug
            if (++rounds > T.max_rounds) {
                overflow = true;
                if (lane == 0) atomicOr(a.status, ST_INTERNAL);
                break;
            }
            // a round takes up to 64 child records from the top ranges of the
            // stack: slot l and slot l + 32 go to lane l
            const int nr = sp < 32 ? sp : 32;
            uint2 Rg = make_uint2(0u, 0u);
            if (lane < nr) Rg = stk[sp - 1 - lane];
            const uint32_t cnt = Rg.y;
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t o = __shfl_up_sync(FULL, incl, d);
                if (lane >= d) incl += o;
            }
            const uint32_t excl = incl - cnt;
            const unsigned fullm = __ballot_sync(FULL, lane < nr && incl <= 64u);
            const int nfull = __popc(fullm);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const int ntake = total < 64u ? (int)total : 64;
            // first slot of every range that starts in this round, slots 0..31 and 32..63
            const unsigned slo = __reduce_or_sync(FULL, (lane < nr && excl < 32u) ? (1u << excl) : 0u);
            const unsigned shi = __reduce_or_sync(
                FULL, (lane < nr && excl >= 32u && excl < 64u) ? (1u << (excl - 32u)) : 0u);
            __syncwarp();
            const int sp_new = sp - nfull;
            if (lane == nfull && lane < nr && excl < 64u) {
                const uint32_t used = 64u - excl;
                stk[sp - 1 - nfull] = make_uint2(Rg.x + used, Rg.y - used);
            }
            // this lane's two child slots: the range of a slot is the last one
            // starting at or before it
            const unsigned upm = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
            const int rj0 = __popc(slo & upm) - 1;
            const int rj1 = __popc(slo) + __popc(shi & upm) - 1;
            const int rs0 = rj0 < 0 ? 0 : rj0, rs1 = rj1 < 0 ? 0 : (rj1 > 31 ? 31 : rj1);
            const uint32_t rcb0 = __shfl_sync(FULL, Rg.x, rs0), rex0 = __shfl_sync(FULL, excl, rs0);
            const uint32_t rcb1 = __shfl_sync(FULL, Rg.x, rs1), rex1 = __shfl_sync(FULL, excl, rs1);
            const uint32_t ci0 = rcb0 + ((uint32_t)lane - rex0);
            const uint32_t ci1 = rcb1 + ((uint32_t)lane + 32u - rex1);
            const Cls c0 = classify<kOpen, kSplit, kRefit>(T, ci0, lane < ntake, lo, gl, p, arelf, arel);
            const Cls c1 = classify<kOpen, kSplit, kRefit>(T, ci1, lane + 32 < ntake, lo, gl, p, arelf, arel);
            // push opened ranges
            const unsigned bo0 = __ballot_sync(FULL, c0.open), bo1 = __ballot_sync(FULL, c1.open);
            const int np0 = __popc(bo0), npush = np0 + __popc(bo1);
            if (sp_new + npush > kStackCap) {
                overflow = true;
                break;
            }
            // a node always has children; a zero count would stall the walk
            if (c0.open) {
                stk[sp_new + __popc(bo0 & lt)] = make_uint2(c0.push_ref, c0.push_cnt > 0u ? c0.push_cnt : 1u);
                if (c0.push_cnt == 0u || (uint64_t)c0.push_ref + c0.push_cnt > (uint64_t)T.nchild)
                    atomicOr(a.status, ST_INTERNAL);
            }
            if (c1.open) {
                stk[sp_new + np0 + __popc(bo1 & lt)] =
                    make_uint2(c1.push_ref, c1.push_cnt > 0u ? c1.push_cnt : 1u);
                if (c1.push_cnt == 0u || (uint64_t)c1.push_ref + c1.push_cnt > (uint64_t)T.nchild)
                    atomicOr(a.status, ST_INTERNAL);
            }
            sp = sp_new + npush;
            // append entries to the far / near chunks (at most 64 each per round)
            const unsigned be0 = __ballot_sync(FULL, c0.emit), be1 = __ballot_sync(FULL, c1.emit);
            const unsigned bn0 = __ballot_sync(FULL, c0.isnode), bn1 = __ballot_sync(FULL, c1.isnode);
            const unsigned bq0 = __ballot_sync(FULL, c0.emit && c0.near);
            const unsigned bq1 = __ballot_sync(FULL, c1.emit && c1.near);
            const unsigned bf0 = be0 & ~bq0, bf1 = be1 & ~bq1;
            cnt_pn += __popc(be0 & bn0) + __popc(be1 & bn1);
            cnt_pp += __popc(be0 & ~bn0) + __popc(be1 & ~bn1);
            const int nf0 = __popc(bf0), nfar = nf0 + __popc(bf1);
            const int nq0 = __popc(bq0), nnear = nq0 + __popc(bq1);
            // a full chunk (or the walk's end) is evaluated before the round's
            // entries are appended; flushes are rare, so they are hinted off
            // the round's main path (the near chunk first: this layout measured
            // fastest, and the order of the chunk totals is free)
            if (__builtin_expect(done || cn + nnear > kNearChunk, 0)) {
                __syncwarp();
                float tx = 0.f, ty = 0.f, tz = 0.f, tp = 0.f;
                eval_near<kSplit, kPot>(chn, cn, rep, R, xi, yi, zi, p, tx, ty, tz, tp);
                acc.add(tx, ty, tz);
                if (kPot) kahan_add(psum, pcomp, tp);
                cn = 0;
                __syncwarp();
            }
            if (__builtin_expect(done || cf + nfar > chunk, 0)) {
                __syncwarp();
                float tx = 0.f, ty = 0.f, tz = 0.f, tp = 0.f;
                eval_far<kSplit, kPot, kFarUnroll>(chf, cf, rep, R, xi, yi, zi, p, tx, ty, tz, tp);
                acc.add(tx, ty, tz);
                if (kPot) kahan_add(psum, pcomp, tp);
                cf = 0;
                __syncwarp();
            }
            if (c0.emit) {
                if (c0.near) chn[cn + __popc(bq0 & lt)] = c0.ent;
                else chf[cf + __popc(bf0 & lt)] = c0.ent;
            }
            if (c1.emit) {
                if (c1.near) chn[cn + nq0 + __popc(bq1 & lt)] = c1.ent;
                else chf[cf + nf0 + __popc(bf1 & lt)] = c1.ent;
            }
            if (kDump && (nfar + nnear) > 0) {
                const int nem = nfar + nnear;
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.list_cursor, (unsigned long long)nem);
                base = __shfl_sync(FULL, base, 0);
                const unsigned long long pos0 = base + __popc(be0 & lt);
                const unsigned long long pos1 = base + __popc(be0) + __popc(be1 & lt);
                if (c0.emit) {
                    if (pos0 < (unsigned long long)a.list_cap) {
                        a.lists[2 * pos0] = (uint32_t)g;
                        a.lists[2 * pos0 + 1] = ci0;
                    } else {
                        atomicOr(a.status, ST_LIST_OVF);
                    }
                }
                if (c1.emit) {
                    if (pos1 < (unsigned long long)a.list_cap) {
                        a.lists[2 * pos1] = (uint32_t)g;
                        a.lists[2 * pos1 + 1] = ci1;
                    } else {
                        atomicOr(a.status, ST_LIST_OVF);
                    }
                }
            }
            cf += nfar;
            cn += nnear;
            __syncwarp();
            if (done) break;
        }
        if (overflow) {
            if (lane == 0) atomicOr(a.status, ST_STACK_OVF);
            __syncwarp();
            continue;
        }
        __syncwarp();
        float vx = __fsub_rn(acc.sx, acc.kx), vy = __fsub_rn(acc.sy, acc.ky),
              vz = __fsub_rn(acc.sz, acc.kz);
        float vp = kPot ? __fsub_rn(psum, pcomp) : 0.f;
        // replicas of a target: fixed-order pairwise sums
        for (int o = P; o < 32; o <<= 1) {
            vx = __fadd_rn(vx, __shfl_xor_sync(FULL, vx, o));
            vy = __fadd_rn(vy, __shfl_xor_sync(FULL, vy, o));
            vz = __fadd_rn(vz, __shfl_xor_sync(FULL, vz, o));
            if (kPot) vp = __fadd_rn(vp, __shfl_xor_sync(FULL, vp, o));
        }
        if (active && rep == 0) {
            T.acc[i] = vx * p.out_scale;
            T.acc[T.n + i] = vy * p.out_scale;
            T.acc[2 * T.n + i] = vz * p.out_scale;
            T.npp[i] = cnt_pp - 1u;
            T.npn[i] = cnt_pn;
            if (kPot) T.pot[i] = -vp * p.pot_scale;
        }
        if (lane == 0) {
            T.gcost[g] = cnt_pp + cnt_pn;
            const unsigned long long ni = (unsigned long long)gsize * (unsigned long long)(cnt_pp - 1u + cnt_pn);
            atomicAdd(a.inter, ni);
            if (kMulti && a.tree_inter) atomicAdd(a.tree_inter + ti, ni);
        }
    }
}

template <int kOpen, bool kSplit, bool kDump, bool kRefit, bool kMulti, bool kPot = false,
          bool kOneSeg = false>
void launch_walk_t(const WalkArgs &a, int64_t nitems, cudaStream_t s, int sms) {
    const size_t smem = (size_t)a.warps * warp_smem(a.chunk);
    auto kern = k_walk<kOpen, kSplit, kDump, kRefit, kMulti, kPot, kOneSeg>;
    // resident blocks per SM of each launch shape, queried once per shape
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> per_sm_of;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = per_sm_of.find({a.warps, a.chunk});
        if (it != per_sm_of.end()) {
            per_sm = it->second;
        } else {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxBlockSmem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, a.warps * 32, smem);
            if (per_sm < 1) per_sm = 1;
            per_sm_of[{a.warps, a.chunk}] = per_sm;
        }
    }
    int64_t want = (nitems + a.warps - 1) / a.warps;
    int64_t grid = (int64_t)sms * per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, a.warps * 32, smem, s>>>(a); note_launch();
}

template <int kOpen, bool kSplit>
void launch_walk(const WalkArgs &a, bool dump, bool refit, bool multi, bool pot, int64_t nitems,
                 cudaStream_t s, int sms) {
    if (pot) {
        // the potential is computed on single trees without list dumps
        if (refit) launch_walk_t<kOpen, kSplit, false, true, false, true>(a, nitems, s, sms);
        else launch_walk_t<kOpen, kSplit, false, false, false, true>(a, nitems, s, sms);
    } else if (multi) {
        if (refit) launch_walk_t<kOpen, kSplit, false, true, true>(a, nitems, s, sms);
        else launch_walk_t<kOpen, kSplit, false, false, true>(a, nitems, s, sms);
    } else if (dump) {
        if (refit) launch_walk_t<kOpen, kSplit, true, true, false>(a, nitems, s, sms);
        else launch_walk_t<kOpen, kSplit, true, false, false>(a, nitems, s, sms);
    } else if (a.one_seg) {
        if (refit) launch_walk_t<kOpen, kSplit, false, true, false, false, true>(a, nitems, s, sms);
        else launch_walk_t<kOpen, kSplit, false, false, false, false, true>(a, nitems, s, sms);
    } else {
        if (refit) launch_walk_t<kOpen, kSplit, false, true, false>(a, nitems, s, sms);
        else launch_walk_t<kOpen, kSplit, false, false, false>(a, nitems, s, sms);
    }
}

__global__ void k_cost_keys(int64_t ng, const uint32_t *__restrict__ gcost, uint64_t *keys,
                            uint32_t *vals) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    // longest list first in coarse classes, a quarter octave of list length
    // each (the exponent and the next two bits of cost + 1), key order within
    // a class: the long groups still start first, and groups walked together
    // stay close in space, so more of their tree records are still in L2
    const uint32_t c = gcost[g] + 1u;
    const uint32_t e = 31u - __clz(c);
    const uint32_t code = (e << 2) | (e >= 2u ? ((c >> (e - 2u)) & 3u) : 0u);
    keys[g] = (uint64_t)(255u - code);
    vals[g] = (uint32_t)g;
}

// several trees: sort keys of every (tree, group) item, longest list first
__global__ void k_item_keys(int64_t nitems, int64_t ntrees, const uint64_t *__restrict__ goff,
                            const TreeView *__restrict__ trees, uint64_t *keys, uint32_t *vals) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nitems) return;
    int64_t lo = 0, hi = ntrees;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (goff[mid] <= (uint64_t)q) lo = mid; else hi = mid;
    }
    const TreeView &T = trees[lo];
    const uint32_t cost = T.has_cost ? T.gcost[q - goff[lo]] : 0u;
    // the classes of k_cost_keys: longest first, tree and key order within
    const uint32_t c = cost + 1u;
    const uint32_t e = 31u - __clz(c);
    const uint32_t code = (e << 2) | (e >= 2u ? ((c >> (e - 2u)) & 3u) : 0u);
    keys[q] = (uint64_t)(255u - code);
    vals[q] = (uint32_t)q;
}

template <int kOpen>
void dispatch(const WalkArgs &a, bool split, bool dump, bool refit, bool multi, bool pot,
              int64_t nitems, cudaStream_t s, int sms) {
    if (split) launch_walk<kOpen, true>(a, dump, refit, multi, pot, nitems, s, sms);
    else launch_walk<kOpen, false>(a, dump, refit, multi, pot, nitems, s, sms);
}

void launch(const WalkArgs &a, int opening, bool split, bool dump, bool refit, bool multi,
            int64_t nitems, cudaStream_t s, bool pot = false) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (opening == OG_OPEN_BH) dispatch<OG_OPEN_BH>(a, split, dump, refit, multi, pot, nitems, s, sms);
    else dispatch<OG_OPEN_REL>(a, split, dump, refit, multi, pot, nitems, s, sms);
}

// Per-box parameters of a pass (uploaded) and the tree's view.  The first
// pass of the relative criterion is Barnes-Hut with theta_first_pass.
og_status prepare_view(og_tree *t, int opening, bool first_pass, const float *a_old_sorted,
                       float *acc_sorted, TreeView *v, WalkParams *wp0) {
    cudaStream_t s = t->ctx->stream;
    const int64_t B = t->nseg;
    t->h_wp.resize((size_t)B);
    for (int64_t b = 0; b < B; ++b) {
        const og_params &q = t->seg_prm[b];
        t->h_wp[b] = make_walk_params(q, opening, first_pass ? q.theta_first_pass : q.theta);
        if (first_pass) t->h_wp[b].dump = false;
        // FP64 output: the last pass stores the unscaled sums, scaled in FP64 later
        if (!first_pass && t->unscaled_out) t->h_wp[b].out_scale = 1.0f;
    }
    *wp0 = t->h_wp[0];
    WalkParams *dp = t->segp + (first_pass ? 0 : B);
    cudaError_t err = cudaMemcpyAsync(dp, t->h_wp.data(), B * sizeof(WalkParams), cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return cuda_fail(err, "walk setup");
    TreeView &w = *v;
    w = TreeView{};
    w.n = t->n;
    w.ngroups = t->ngroups;
    w.gbeg = t->gbeg;
    w.gend = t->gend;
    w.gbox = t->gbox;
    w.gcost = t->gcost;
    w.gorder = nullptr;
    w.crec = t->crec;
    w.cext = t->cext;
    w.nchild = t->nchild;
    w.max_rounds = t->nchild + 2;
    w.gseg = t->gseg;
    w.ncbeg = t->ncbeg;
    w.nccnt = t->nccnt;
    w.segp = dp;
    w.px = t->px;
    w.py = t->py;
    w.pz = t->pz;
    w.a_old = a_old_sorted;
    w.acc = acc_sorted;
    w.npp = t->npp_sorted;
    w.npn = t->npn_sorted;
    w.has_cost = t->have_cost ? 1 : 0;
    return OG_OK;
}

void fill_common(WalkArgs &a, og_ctx *c, og_tree *t) {
    // a tree's launch shape (zero fields take the defaults)
    a.warps = t && t->prm.walk_warps > 0 ? t->prm.walk_warps : kDefaultWalkWarps;
    a.chunk = t && t->prm.walk_chunk > 0 ? t->prm.walk_chunk : kDefaultWalkChunk;
    a.lists = t ? t->lists : nullptr;
    a.list_cap = t ? t->list_cap : 0;
    a.work = c->d_counters;
    a.inter = c->d_counters + 1;
    a.list_cursor = c->d_counters + 2;
    a.status = c->d_status;
}

}  // namespace

WalkParams make_walk_params(const og_params &p, int opening, double theta) {
    WalkParams w{};
    const double two32 = 4294967296.0;
    w.opening = opening;
    w.split = p.r_s > 0.0;
    w.dump = (p.flags & OG_DEBUG_DUMP_LISTS) != 0;
    w.th2 = theta * theta;
    w.th2f = (float)w.th2;
    w.G = p.G;
    w.Gf = (float)p.G;
    const double s = p.box / two32;
    w.s2 = s * s;
    w.alpha = p.alpha;
    if (w.split) {
        const double rcg = (p.rcut_over_rs * p.r_s) / p.box * two32;
        const double rsg = p.r_s / p.box * two32;
        w.rc2 = (float)(rcg * rcg);
        w.rprune = (unsigned long long)(rcg * rcg * (1.0 + 1.0 / 1024.0));
        w.inv_2rs = (float)(1.0 / (2.0 * rsg));
        // exp(-r^2 / (4 r_s^2)) = 2^(r^2 * kexp)
        w.kexp = (float)(-1.4426950408889634 / (4.0 * rsg * rsg));
    } else {
        w.rc2 = __builtin_huge_valf();
        w.rprune = ~0ull;
        w.inv_2rs = 0.0f;
        w.kexp = 0.0f;
    }
    const double hg = 2.8 * p.eps / p.box * two32;
    w.h = (float)hg;
    w.inv_h = hg > 0.0 ? (float)(1.0 / hg) : 0.0f;
    // an entry is "near" when its integer distance to the group box is below
    // h (with a generous rounding margin); only near entries may need
    // softening.  An entry inside the group box (a member itself) is always
    // near, so a far entry is at r^2 >= 1 from every target.
    const double hn = hg * (1.0 + 1.0 / 256.0) + 2.0;
    w.hnear2 = hg > 0.0 ? (unsigned long long)(hn * hn) : 1ull;
    // the single-precision square of an integer distance errs by less than
    // 5 * 2^-24 relative, so d2f >= hnear2f implies an exact square >= hnear2
    w.hnear2f = nextafterf((float)((double)w.hnear2 * (1.0 + 1.0 / (1 << 20))), __builtin_huge_valf());
    w.out_scale = (float)(p.G * (two32 / p.box) * (two32 / p.box));
    w.pot_scale = (float)(p.G * (two32 / p.box));
    return w;
}

static og_status finish_pass(og_ctx *c, cudaEvent_t e0, cudaEvent_t e1, float *ms_out,
                             unsigned long long h[3]) {
    cudaStream_t s = c->stream;
    cudaMemcpyAsync(h, c->d_counters, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaError_t err = cudaStreamSynchronize(s);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "walk");
    if ((err = cudaGetLastError()) != cudaSuccess) return cuda_fail(err, "walk launch");
    if (ms_out) *ms_out = ms;
    return OG_OK;
}

// Replace the debug list buffer by one of at least `need` entries and clear
// the overflow bit the short buffer left in the status word.
static og_status grow_lists(og_tree *t, int64_t need) {
    cudaStream_t s = t->ctx->stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "list buffer");
    cudaFree(t->lists);
    t->lists = nullptr;
    t->list_cap = 0;
    const int64_t cap = need + need / 8 + 1024;
    if ((e = cudaMalloc(&t->lists, (size_t)cap * 2 * sizeof(uint32_t))) != cudaSuccess) {
        t->lists = nullptr;
        return cuda_fail(e, "cudaMalloc (lists)");
    }
    t->list_cap = cap;
    uint32_t st = 0;
    if ((e = cudaMemcpy(&st, t->ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    st &= ~(uint32_t)ST_LIST_OVF;
    if ((e = cudaMemcpy(t->ctx->d_status, &st, sizeof(st), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "status write");
    return OG_OK;
}

og_status finish_deferred(og_tree *t, float *ms_walk) {
    og_status st = OG_OK;
    for (int k = 0; k < t->npend; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, t->pend_e0[k], t->pend_e1[k]) == cudaSuccess && ms_walk)
            *ms_walk += ms;
        cudaEventDestroy(t->pend_e0[k]);
        cudaEventDestroy(t->pend_e1[k]);
        t->pend_e0[k] = t->pend_e1[k] = nullptr;
        const unsigned long long *h = pinned_counters(t->ctx, k);
        t->interactions_last = (int64_t)h[1];
        t->interactions += (int64_t)h[1];
    }
    t->npend = 0;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) st = cuda_fail(err, "walk launch");
    return st;
}

og_status walk_pass(og_tree *t, int opening, bool first_pass, const float *a_old_sorted,
                    float *acc_sorted, float *ms_out, bool use_order, const uint32_t *subset,
                    int64_t nsubset, float *pot_sorted, bool defer) {
    cudaStream_t s = t->ctx->stream;
    WalkArgs a{};
    WalkParams wp;
    og_status st = prepare_view(t, opening, first_pass, a_old_sorted, acc_sorted, &a.tree0, &wp);
    if (st) return st;
    fill_common(a, t->ctx, t);
    a.one_seg = t->nseg == 1 ? 1 : 0;
    a.p0 = t->h_wp[0];
    cudaError_t err;
    void *sort_tmp = nullptr;
    if (subset) {
        // only these groups, in this order (the walk takes them from gorder)
        a.tree0.gorder = subset;
        a.tree0.ngroups = nsubset;
    } else if (use_order && t->have_cost && t->ngroups > 1) {
        // longest list first, from the costs of the previous pass on this tree
        const int64_t ng = t->ngroups;
        size_t bytes = (size_t)ng * 24 + radix_sort_scratch_bytes(ng) + 1024;
        if ((err = dev_malloc_async(&sort_tmp, bytes, s)) != cudaSuccess)
            return cuda_fail(err, "cudaMallocAsync (group order)");
        char *q = static_cast<char *>(sort_tmp);
        uint64_t *k0 = reinterpret_cast<uint64_t *>(q);
        uint64_t *k1 = k0 + ng;
        uint32_t *v0 = reinterpret_cast<uint32_t *>(k1 + ng);
        uint32_t *v1 = v0 + ng;
        void *scr = v1 + ng + 64;
        k_cost_keys<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(ng, t->gcost, k0, v0); note_launch();
        bool alt = false;
        radix_sort_pairs(k0, v0, k1, v1, ng, 8, scr, s, &alt, t->ctx->d_status);
        cudaMemcpyAsync(t->gorder, alt ? v1 : v0, ng * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        a.tree0.gorder = t->gorder;
    }
    if (defer && !wp.dump && t->npend < 2) {
        // no host synchronisation: the counters go to a page-locked slot and
        // the times to events, both read by finish_deferred
        const int k = t->npend;
        cudaMemsetAsync(t->ctx->d_counters, 0, 3 * sizeof(unsigned long long), s);
        cudaEventCreate(&t->pend_e0[k]);
        cudaEventCreate(&t->pend_e1[k]);
        cudaEventRecord(t->pend_e0[k], s);
        a.tree0.pot = pot_sorted;
        launch(a, opening, wp.split, false, t->refit, false, a.tree0.ngroups, s, pot_sorted != nullptr);
        cudaEventRecord(t->pend_e1[k], s);
        cudaMemcpyAsync(pinned_counters(t->ctx, k), t->ctx->d_counters, 3 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s);
        t->npend = k + 1;
        if (sort_tmp) cudaFreeAsync(sort_tmp, s);
        // the next pass may take this one's list lengths: stream order makes them ready
        t->have_cost = true;
        if (ms_out) *ms_out = 0.0f;
        return OG_OK;
    }
    unsigned long long h[3] = {0, 0, 0};
    for (int attempt = 0; attempt < 2; ++attempt) {
        cudaMemsetAsync(t->ctx->d_counters, 0, 3 * sizeof(unsigned long long), s);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
        a.tree0.pot = pot_sorted;
        launch(a, opening, wp.split, wp.dump && !pot_sorted, t->refit, false, a.tree0.ngroups, s,
               pot_sorted != nullptr);
        cudaEventRecord(e1, s);
        st = finish_pass(t->ctx, e0, e1, ms_out, h);
        if (st) break;
        if (!wp.dump || h[2] <= (unsigned long long)t->list_cap) break;
        // debug lists only: the pass counted every entry it could not keep;
        // give the buffer that size and walk again (the pass is deterministic)
        st = grow_lists(t, (int64_t)h[2]);
        if (st) break;
        a.lists = t->lists;
        a.list_cap = t->list_cap;
    }
    if (sort_tmp) cudaFreeAsync(sort_tmp, s);
    if (st) return st;
    t->have_cost = true;
    t->interactions_last = (int64_t)h[1];
    t->interactions += (int64_t)h[1];
    if (wp.dump) t->list_len = (int64_t)(h[2] < (unsigned long long)t->list_cap ? h[2] : t->list_cap);
    return OG_OK;
}

og_status walk_multi(og_ctx *c, og_tree *const *trees, int64_t ntrees, int opening,
                     const float *const *a_old_sorted, float *const *acc_sorted, float *ms_out,
                     int64_t *interactions, int64_t *tree_interactions) {
    cudaStream_t s = c->stream;
    if (ntrees < 1) return OG_OK;
    std::vector<TreeView> hv((size_t)ntrees);
    std::vector<uint64_t> hoff((size_t)ntrees + 1);
    bool split = false, refit = false;
    uint64_t total = 0;
    for (int64_t k = 0; k < ntrees; ++k) {
        WalkParams wp;
        og_status st = prepare_view(trees[k], opening, false, a_old_sorted ? a_old_sorted[k] : nullptr,
                                    acc_sorted[k], &hv[k], &wp);
        if (st) return st;
        if (k == 0) split = wp.split;
        else if (wp.split != split) {
            set_error("walk over several trees: split on/off must agree");
            return OG_ERR_ARG;
        }
        refit = refit || trees[k]->refit;
        hoff[k] = total;
        total += (uint64_t)trees[k]->ngroups;
    }
    hoff[ntrees] = total;
    if (refit) {
        // one instantiation for all trees: built trees read their cells as extents
        for (int64_t k = 0; k < ntrees; ++k) {
            if (!trees[k]->cext) {
                og_status st = cell_extents(trees[k]);
                if (st) return st;
            }
            hv[k].cext = trees[k]->cext;
        }
    }
    const int64_t nitems = (int64_t)total;
    size_t bytes = (size_t)ntrees * sizeof(TreeView) + (size_t)(ntrees + 1) * 8 + (size_t)nitems * 24 +
                   radix_sort_scratch_bytes(nitems) + (size_t)ntrees * 8 + 4096;
    void *tmp = nullptr;
    cudaError_t err;
    if ((err = dev_malloc_async(&tmp, bytes, s)) != cudaSuccess) return cuda_fail(err, "cudaMallocAsync (walk items)");
    char *q = static_cast<char *>(tmp);
    TreeView *dv = reinterpret_cast<TreeView *>(q);
    q += ((size_t)ntrees * sizeof(TreeView) + 255) & ~(size_t)255;
    uint64_t *doff = reinterpret_cast<uint64_t *>(q);
    q += ((size_t)(ntrees + 1) * 8 + 255) & ~(size_t)255;
    uint64_t *k0 = reinterpret_cast<uint64_t *>(q);
    uint64_t *k1 = k0 + nitems;
    uint32_t *v0 = reinterpret_cast<uint32_t *>(k1 + nitems);
    uint32_t *v1 = v0 + nitems;
    unsigned long long *tint = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(v1 + nitems) + 255) & ~(uintptr_t)255);
    void *scr = tint + ntrees + 32;
    cudaMemcpyAsync(dv, hv.data(), ntrees * sizeof(TreeView), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(doff, hoff.data(), (ntrees + 1) * 8, cudaMemcpyHostToDevice, s);
    k_item_keys<<<(unsigned)((nitems + 255) / 256), 256, 0, s>>>(nitems, ntrees, doff, dv, k0, v0); note_launch();
    bool alt = false;
    radix_sort_pairs(k0, v0, k1, v1, nitems, 8, scr, s, &alt, c->d_status);
    WalkArgs a{};
    fill_common(a, c, nullptr);
    a.trees = dv;
    a.goff = doff;
    a.items = alt ? v1 : v0;
    a.ntrees = ntrees;
    a.nitems = nitems;
    a.tree_inter = tint;
    cudaMemsetAsync(tint, 0, (size_t)ntrees * sizeof(unsigned long long), s);
    cudaMemsetAsync(c->d_counters, 0, 3 * sizeof(unsigned long long), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    launch(a, opening, split, false, refit, true, nitems, s);
    cudaEventRecord(e1, s);
    std::vector<unsigned long long> hti(tree_interactions ? (size_t)ntrees : 0);
    if (tree_interactions)
        cudaMemcpyAsync(hti.data(), tint, (size_t)ntrees * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(tmp, s);
    unsigned long long h[3] = {0, 0, 0};
    og_status st = finish_pass(c, e0, e1, ms_out, h);
    if (st) return st;
    for (int64_t k = 0; k < ntrees; ++k) trees[k]->have_cost = true;
    if (interactions) *interactions = (int64_t)h[1];
    if (tree_interactions)
        for (int64_t k = 0; k < ntrees; ++k) tree_interactions[k] = (int64_t)hti[(size_t)k];
    return OG_OK;
}

}  // namespace og
