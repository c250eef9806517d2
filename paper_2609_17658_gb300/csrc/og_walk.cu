// og_walk.cu -- group-wise tree walk and force evaluation (Sect. 4.1.2, 4.1.3, 4.2).
//
// The paper walks the tree once per target particle with a threaded
// (nextnode / sibling) loop and, on GPUs, processes neighbours in chunks of
// 32.  Here one warp walks the tree once for a whole group of up to 32
// spatially close targets (one target per lane) and shares the resulting
// interaction list:
//
//   list building   the warp keeps a stack of child-array ranges of opened
//                   nodes in shared memory.  Each round the 32 lanes take the
//                   next 32 child records (32-byte records, coalesced loads),
//                   and each lane classifies its record against the group's
//                   integer bounding box:
//                     particle -> PP entry unless beyond the prune distance;
//                     node     -> pruned, opened (range pushed), or PN entry.
//                   The prune test is exact integer geometry; the boundary
//                   check is an exact integer test; the Barnes-Hut / relative
//                   opening test is FP64 with a fixed operation order and no
//                   fused operations, so the lists equal the oracle's.
//   evaluation      accepted entries (x, y, z, m) are appended to a shared
//                   chunk; when it fills, every lane evaluates the chunk for
//                   its target: exact int32 minimum-image separation, converted
//                   to FP32, r^2 by FMA, cutoff, rsqrt, spline softening inside
//                   h, erfc split factor, FP32 accumulation over the chunk, then
//                   a compensated (Kahan) add of the chunk sum into the totals.
//
// Work distribution: persistent blocks, warps take groups from a global
// atomic counter (groups in clustered regions cost far more than others).
#include "og_internal.h"

namespace og {
namespace {

constexpr int kWarps = 4;          // warps per block
constexpr int kStackCap = 768;     // ranges per warp stack
constexpr int kChunk = 256;        // entries per shared chunk

// Abramowitz & Stegun 7.1.26: erfc(x) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
// t = 1 / (1 + p x), |error| <= 1.5e-7 for x >= 0.
constexpr float kAsP = 0.3275911f;
constexpr float kAs1 = 0.254829592f, kAs2 = -0.284496736f, kAs3 = 1.421413741f;
constexpr float kAs4 = -1.453152027f, kAs5 = 1.061405429f;
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

struct WalkArgs {
    int64_t n, ngroups;
    const uint32_t *gbeg, *gend, *gbox;
    const CRec *crec;
    int64_t nchild, max_rounds;
    uint32_t root_cbeg, root_ccnt;
    const uint32_t *px, *py, *pz;
    const float *a_old;           // [3][n] sorted, relative criterion only
    float *acc;                   // [3][n] sorted, out
    uint32_t *npp, *npn;          // [n] sorted, out
    uint32_t *lists;              // debug dump: (group, child slot) pairs
    unsigned long long *list_cursor;
    int64_t list_cap;
    unsigned long long *work;     // group counter
    unsigned long long *inter;    // interactions evaluated
    uint32_t *status;
    WalkParams p;
};

__device__ __forceinline__ uint32_t point_gap(uint32_t c, uint32_t lo, uint32_t hi) {
    if (c >= lo && c <= hi) return 0u;
    uint32_t a = lo - c, b = c - hi;
    return a < b ? a : b;
}

__device__ __forceinline__ uint32_t box_gap(uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi) {
    if (alo <= bhi && blo <= ahi) return 0u;
    uint32_t a = blo - ahi, b = alo - bhi;
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long sq64(uint32_t g) {
    return (unsigned long long)g * (unsigned long long)g;
}

template <bool kSplit>
__device__ __forceinline__ void eval_chunk(const uint4 *ch, int cnt, uint32_t xi, uint32_t yi,
                                           uint32_t zi, const WalkParams &p, float &ax, float &ay,
                                           float &az) {
    const float rc2 = p.rc2, h = p.h, inv_h = p.inv_h, inv_2rs = p.inv_2rs;
    const float hinv3 = inv_h * inv_h * inv_h;
#pragma unroll 4
    for (int e = 0; e < cnt; ++e) {
        const uint4 s = ch[e];
        const float fx = __int2float_rn((int)(s.x - xi));
        const float fy = __int2float_rn((int)(s.y - yi));
        const float fz = __int2float_rn((int)(s.z - zi));
        const float r2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, __fmul_rn(fz, fz)));
        const bool in = (r2 > 0.0f) && (r2 < rc2);
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        float g = rinv * rinv * rinv;
        if (r < h) {
            const float u = r * inv_h;
            const float u2 = u * u;
            if (u < 0.5f)
                g = hinv3 * (32.0f / 3.0f + u2 * (32.0f * u - 192.0f / 5.0f));
            else
                g = hinv3 * (64.0f / 3.0f - 48.0f * u + 192.0f / 5.0f * u2 -
                             32.0f / 3.0f * u2 * u - (1.0f / 15.0f) / (u2 * u));
        }
        float S = 1.0f;
        if (kSplit) {
            const float us = r * inv_2rs;
            const float t = __fdividef(1.0f, fmaf(kAsP, us, 1.0f));
            const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, kAs5, kAs4), kAs3), kAs2), kAs1);
            const float ex = __expf(-us * us);
            S = ex * fmaf(kTwoOverSqrtPi, us, poly);
        }
        const float f = in ? __uint_as_float(s.w) * g * S : 0.0f;
        ax = fmaf(f, fx, ax);
        ay = fmaf(f, fy, ay);
        az = fmaf(f, fz, az);
    }
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v) {
    const float y = __fsub_rn(v, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

template <int kOpen, bool kSplit, bool kDump>
__global__ void __launch_bounds__(kWarps * 32) k_walk(WalkArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint2 *stk = reinterpret_cast<uint2 *>(smem) + warp * kStackCap;
    uint4 *ch = reinterpret_cast<uint4 *>(smem + kWarps * kStackCap * sizeof(uint2)) + warp * kChunk;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    const WalkParams &p = a.p;

    while (true) {
        unsigned long long gq = 0;
        if (lane == 0) gq = atomicAdd(a.work, 1ull);
        gq = __shfl_sync(FULL, gq, 0);
        if (gq >= (unsigned long long)a.ngroups) break;
        const int64_t g = (int64_t)gq;
        const uint32_t gb = a.gbeg[g], ge = a.gend[g];
        uint32_t lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = a.gbox[6 * g + k];
            hi[k] = a.gbox[6 * g + 3 + k];
        }
        const uint32_t i = gb + lane;
        const bool active = i < ge;
        const uint32_t xi = active ? a.px[i] : 0u;
        const uint32_t yi = active ? a.py[i] : 0u;
        const uint32_t zi = active ? a.pz[i] : 0u;
        // relative criterion: arel = (alpha * a_min) * s^2, a_min = min over the group
        // of |a_old| in FP64 of the single-precision components
        double arel_coef = 0.0;
        if (kOpen == OG_OPEN_REL) {
            double an = __longlong_as_double(0x7ff0000000000000ll);  // +inf
            if (active) {
                double ax0 = a.a_old[i], ay0 = a.a_old[a.n + i], az0 = a.a_old[2 * a.n + i];
                an = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ax0, ax0), __dmul_rn(ay0, ay0)),
                                          __dmul_rn(az0, az0)));
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) an = fmin(an, __shfl_xor_sync(FULL, an, d));
            arel_coef = __dmul_rn(__dmul_rn(p.alpha, an), p.s2);
        }

        if (lane == 0) stk[0] = make_uint2(a.root_cbeg, a.root_ccnt);
        __syncwarp();
        int sp = 1, cc = 0;
        int64_t rounds = 0;
        uint32_t cnt_pp = 0, cnt_pn = 0;
        float sx = 0.f, sy = 0.f, sz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
        bool overflow = false;

        while (sp > 0) {
            // every round consumes at least one child record and a record is
            // visited at most once per walk: more rounds than records is a bug
            if (++rounds > a.max_rounds) {
                overflow = true;
                if (lane == 0) atomicOr(a.status, ST_INTERNAL);
                break;
            }
            const int nr = sp < 32 ? sp : 32;
            uint2 R = make_uint2(0u, 0u);
            if (lane < nr) R = stk[sp - 1 - lane];
            const uint32_t cnt = R.y;
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t o = __shfl_up_sync(FULL, incl, d);
                if (lane >= d) incl += o;
            }
            const uint32_t excl = incl - cnt;
            const unsigned fullm = __ballot_sync(FULL, lane < nr && incl <= 32u);
            const int nfull = __popc(fullm);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const int ntake = total < 32u ? (int)total : 32;
            const unsigned bit = (lane < nr && excl < 32u) ? (1u << excl) : 0u;
            const unsigned smask = __reduce_or_sync(FULL, bit);
            __syncwarp();
            const int sp_new = sp - nfull;
            if (lane == nfull && lane < nr && excl < 32u) {
                const uint32_t used = 32u - excl;
                stk[sp - 1 - nfull] = make_uint2(R.x + used, R.y - used);
            }
            // this lane's child slot
            const unsigned upto = lane == 31 ? smask : (smask & ((2u << lane) - 1u));
            const int rj = __popc(upto) - 1;
            const uint32_t rcb = __shfl_sync(FULL, R.x, rj < 0 ? 0 : rj);
            const uint32_t rex = __shfl_sync(FULL, excl, rj < 0 ? 0 : rj);
            const bool has = lane < ntake;
            const uint32_t ci = rcb + ((uint32_t)lane - rex);

            bool emit = false, open = false, isnode = false;
            CRec r;
            r.x = r.y = r.z = 0u;
            r.m = 0.f;
            r.M = 0.0;
            r.info = 0u;
            r.ref = 0u;
            if (has && ci < a.nchild) {
                r = a.crec[ci];
                isnode = (r.info >> 31) != 0u;
                if (!isnode) {
                    if (!kSplit) {
                        emit = true;
                    } else {
                        unsigned long long g2 = sq64(point_gap(r.x, lo[0], hi[0])) +
                                                sq64(point_gap(r.y, lo[1], hi[1])) +
                                                sq64(point_gap(r.z, lo[2], hi[2]));
                        emit = g2 <= p.rprune;
                    }
                } else {
                    const uint32_t lev = (r.info >> 26) & 31u;
                    const uint32_t side = 1u << (32u - lev);
                    const uint32_t msk = ~(side - 1u);
                    const uint32_t com[3] = {r.x, r.y, r.z};
                    uint32_t org[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) org[k] = com[k] & msk;
                    bool pruned = false;
                    if (kSplit) {
                        unsigned long long g2 = 0;
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            g2 += sq64(box_gap(lo[k], hi[k], org[k], org[k] + (side - 1u)));
                        pruned = g2 > p.rprune;
                    }
                    if (!pruned) {
                        // boundary check: box meets the cell enlarged to 0.6 side
                        bool near = true;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const uint32_t centre = org[k] + (side >> 1);
                            const unsigned long long dc = point_gap(centre, lo[k], hi[k]);
                            if (10ull * dc > 6ull * (unsigned long long)side) near = false;
                        }
                        if (near) {
                            open = true;
                        } else {
                            const double dx = (double)point_gap(com[0], lo[0], hi[0]);
                            const double dy = (double)point_gap(com[1], lo[1], hi[1]);
                            const double dz = (double)point_gap(com[2], lo[2], hi[2]);
                            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                                        __dmul_rn(dz, dz));
                            const double l2 = (double)side * (double)side;
                            if (kOpen == OG_OPEN_BH) {
                                open = l2 > __dmul_rn(p.th2, d2);
                            } else {
                                const double lhs = __dmul_rn(__dmul_rn(p.G, r.M), l2);
                                const double rhs = __dmul_rn(arel_coef, __dmul_rn(d2, d2));
                                open = lhs > rhs;
                            }
                        }
                        emit = !open;
                    }
                }
            }
            // push opened ranges
            const unsigned bo = __ballot_sync(FULL, open);
            const int npush = __popc(bo);
            if (sp_new + npush > kStackCap) {
                overflow = true;
                break;
            }
            if (open) {
                const uint32_t cnt_c = r.info & 0x3ffffffu;
                // a node always has children; a zero count would stall the walk
                stk[sp_new + __popc(bo & lt)] = make_uint2(r.ref, cnt_c > 0u ? cnt_c : 1u);
                if (cnt_c == 0u || (uint64_t)r.ref + cnt_c > (uint64_t)a.nchild) atomicOr(a.status, ST_INTERNAL);
            }
            sp = sp_new + npush;
            // append entries
            const unsigned be = __ballot_sync(FULL, emit);
            const unsigned bn = __ballot_sync(FULL, isnode);
            const int nem = __popc(be);
            cnt_pn += __popc(be & bn);
            cnt_pp += __popc(be & ~bn);
            if (cc + nem > kChunk) {
                __syncwarp();
                float tx = 0.f, ty = 0.f, tz = 0.f;
                eval_chunk<kSplit>(ch, cc, xi, yi, zi, p, tx, ty, tz);
                kahan_add(sx, kx, tx);
                kahan_add(sy, ky, ty);
                kahan_add(sz, kz, tz);
                cc = 0;
                __syncwarp();
            }
            if (emit) ch[cc + __popc(be & lt)] = make_uint4(r.x, r.y, r.z, __float_as_uint(r.m));
            if (kDump && nem > 0) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.list_cursor, (unsigned long long)nem);
                base = __shfl_sync(FULL, base, 0);
                if (emit) {
                    unsigned long long pos = base + __popc(be & lt);
                    if (pos < (unsigned long long)a.list_cap) {
                        a.lists[2 * pos] = (uint32_t)g;
                        a.lists[2 * pos + 1] = ci;
                    } else {
                        atomicOr(a.status, ST_LIST_OVF);
                    }
                }
            }
            cc += nem;
            __syncwarp();
        }
        if (overflow) {
            if (lane == 0) atomicOr(a.status, ST_STACK_OVF);
            __syncwarp();
            continue;
        }
        __syncwarp();
        {
            float tx = 0.f, ty = 0.f, tz = 0.f;
            eval_chunk<kSplit>(ch, cc, xi, yi, zi, p, tx, ty, tz);
            kahan_add(sx, kx, tx);
            kahan_add(sy, ky, ty);
            kahan_add(sz, kz, tz);
        }
        __syncwarp();
        if (active) {
            a.acc[i] = __fsub_rn(sx, kx) * p.out_scale;
            a.acc[a.n + i] = __fsub_rn(sy, ky) * p.out_scale;
            a.acc[2 * a.n + i] = __fsub_rn(sz, kz) * p.out_scale;
            a.npp[i] = cnt_pp - 1u;
            a.npn[i] = cnt_pn;
        }
        if (lane == 0)
            atomicAdd(a.inter, (unsigned long long)(ge - gb) *
                                   (unsigned long long)(cnt_pp - 1u + cnt_pn));
    }
}

template <int kOpen, bool kSplit, bool kDump>
void launch_walk(const WalkArgs &a, cudaStream_t s, int sms) {
    const size_t smem = kWarps * (kStackCap * sizeof(uint2) + kChunk * sizeof(uint4));
    static bool attr = false;
    static int per_sm = 1;
    if (!attr) {
        cudaFuncSetAttribute(k_walk<kOpen, kSplit, kDump>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<kOpen, kSplit, kDump>,
                                                      kWarps * 32, smem);
        if (per_sm < 1) per_sm = 1;
        attr = true;
    }
    int64_t want = (a.ngroups + kWarps - 1) / kWarps;
    int64_t grid = (int64_t)sms * per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    k_walk<kOpen, kSplit, kDump><<<(unsigned)grid, kWarps * 32, smem, s>>>(a);
}

}  // namespace

WalkParams make_walk_params(const og_params &p, int opening, double theta) {
    WalkParams w{};
    const double two32 = 4294967296.0;
    w.opening = opening;
    w.split = p.r_s > 0.0;
    w.dump = (p.flags & OG_DEBUG_DUMP_LISTS) != 0;
    w.th2 = theta * theta;
    w.G = p.G;
    const double s = p.box / two32;
    w.s2 = s * s;
    w.alpha = p.alpha;
    if (w.split) {
        const double rcg = (p.rcut_over_rs * p.r_s) / p.box * two32;
        w.rc2 = (float)(rcg * rcg);
        w.rprune = (unsigned long long)(rcg * rcg * (1.0 + 1.0 / 1024.0));
        w.inv_2rs = (float)(1.0 / (2.0 * p.r_s / p.box * two32));
    } else {
        w.rc2 = __builtin_huge_valf();
        w.rprune = ~0ull;
        w.inv_2rs = 0.0f;
    }
    const double hg = 2.8 * p.eps / p.box * two32;
    w.h = (float)hg;
    w.inv_h = hg > 0.0 ? (float)(1.0 / hg) : 0.0f;
    w.out_scale = (float)(p.G * (two32 / p.box) * (two32 / p.box));
    return w;
}

og_status walk_pass(og_tree *t, const WalkParams &wp, const float *a_old_sorted, float *acc_sorted,
                    float *ms_out) {
    cudaStream_t s = t->ctx->stream;
    WalkArgs a{};
    a.n = t->n;
    a.ngroups = t->ngroups;
    a.gbeg = t->gbeg;
    a.gend = t->gend;
    a.gbox = t->gbox;
    a.crec = t->crec;
    a.nchild = t->nchild;
    a.max_rounds = t->nchild + 2;
    uint32_t root[2];
    // root child range (cbeg[0] = 0 by construction of the scan; ccnt read back)
    cudaMemcpyAsync(root, t->ncbeg, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(root + 1, t->nccnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    a.root_cbeg = root[0];
    a.root_ccnt = root[1];
    a.px = t->px;
    a.py = t->py;
    a.pz = t->pz;
    a.a_old = a_old_sorted;
    a.acc = acc_sorted;
    a.npp = t->npp_sorted;
    a.npn = t->npn_sorted;
    a.lists = t->lists;
    a.list_cap = t->list_cap;
    a.work = t->ctx->d_counters;
    a.inter = t->ctx->d_counters + 1;
    a.list_cursor = t->ctx->d_counters + 2;
    a.status = t->ctx->d_status;
    a.p = wp;
    cudaMemsetAsync(t->ctx->d_counters, 0, 3 * sizeof(unsigned long long), s);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (wp.opening == OG_OPEN_BH) {
        if (wp.split) {
            if (wp.dump) launch_walk<OG_OPEN_BH, true, true>(a, s, sms);
            else launch_walk<OG_OPEN_BH, true, false>(a, s, sms);
        } else {
            if (wp.dump) launch_walk<OG_OPEN_BH, false, true>(a, s, sms);
            else launch_walk<OG_OPEN_BH, false, false>(a, s, sms);
        }
    } else {
        if (wp.split) {
            if (wp.dump) launch_walk<OG_OPEN_REL, true, true>(a, s, sms);
            else launch_walk<OG_OPEN_REL, true, false>(a, s, sms);
        } else {
            if (wp.dump) launch_walk<OG_OPEN_REL, false, true>(a, s, sms);
            else launch_walk<OG_OPEN_REL, false, false>(a, s, sms);
        }
    }
    cudaEventRecord(e1, s);
    unsigned long long h[3] = {0, 0, 0};
    cudaMemcpyAsync(h, t->ctx->d_counters, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaError_t err = cudaStreamSynchronize(s);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "walk");
    if ((err = cudaGetLastError()) != cudaSuccess) return cuda_fail(err, "walk launch");
    if (ms_out) *ms_out = ms;
    t->interactions_last = (int64_t)h[1];
    t->interactions += (int64_t)h[1];
    if (wp.dump) t->list_len = (int64_t)(h[2] < (unsigned long long)t->list_cap ? h[2] : t->list_cap);
    return OG_OK;
}

}  // namespace og
