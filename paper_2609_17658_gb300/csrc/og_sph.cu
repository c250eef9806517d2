// og_sph.cu -- grouped neighbour search and SPH density at given smoothing
// lengths (Sect. 3.4 "Neighbour search", Sect. 6 "Smoothed Particle
// Hydrodynamics").
//
// rho_i = sum_j m_j W(|x_i - x_j|, h_i) over the particles j (i included)
// closer than h_i, with the cubic spline W = 8 / (pi h^3) w(r / h),
// w(q) = 1 - 6 q^2 + 6 q^3 below 1/2, 2 (1 - q)^3 up to 1.
//
// The search is done once per walk group (at most 32 particles that are
// neighbours in key order), as the paper does: one warp per group walks the
// tree from the root with a shared-memory stack of child ranges.  A node is
// opened unless its cell lies farther from the group's integer box than the
// group's largest h (exact 64-bit squared gaps, with a small margin: the
// margin only adds candidates); a particle within that distance of the box is
// a candidate and goes to the warp's shared chunk.  When the chunk fills,
// every lane (one target each) runs over it: j is a neighbour of i iff
// r2 < h2 in float32, r2 = (fx fx + fy fy) + fz fz from the exact integer
// separations and h2 = hg hg, hg = float32(h 2^32 / L), each operation
// rounded on its own, so the neighbour count is the same integer the oracle
// computes.  The density sums w in float32 and is scaled in float64.
//
// A round takes whole ranges from the top of the stack while they hold at most
// 32 child records together (a first range with more, a bucket of coincident
// particles, gives 32 and keeps the rest), one record per lane, so the records
// are loaded at once.  Stack depth: a round pushes at most 32 ranges, so while
// the depth is at most kSphDeep it ends at most 31 above; beyond kSphDeep a
// round takes a single range (one node, at most 8 child nodes), a plain depth-
// first walk that adds at most 7 entries per tree level, 7 x 21 for the
// deepest path: 31 + 147 < 200 entries above kSphDeep.  A push past the
// capacity would still only set the stack-overflow status and drop the range.
// The round count is bounded by the number of nodes plus the buckets' extra
// rounds.
#include <cmath>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kSphWarps = 4;      // warps (groups) per block: 20 KB of shared memory
constexpr int kSphStack = 512;    // child ranges per warp: first entry | count << 32
constexpr int kSphDeep = kSphStack - 200;  // above this depth a round takes one range
constexpr int kSphChunk = 64;     // candidate particles per warp
constexpr int kSphSmem = kSphWarps * (kSphStack * 8 + kSphChunk * 16);
static_assert(kSphSmem <= 48 * 1024, "shared memory of one block");

struct SphArgs {
    const CRec *crec;
    const uint32_t *ncbeg, *nccnt;
    const uint32_t *gbeg, *gend, *gbox;
    const uint32_t *px, *py, *pz;
    const uint32_t *perm;   // outputs to the caller's order; null: key order
    const uint8_t *done;    // null, or per particle (key order): converged, skip
    const float *hg;        // smoothing length in grid units, sorted order
    int64_t ngroups;
    int64_t max_rounds;     // nodes + 2 + buckets' extra rounds (<= n / 32)
    double dens;            // 8 / pi * (2^32 / L)^3
    float *rho;             // caller order (key order without perm)
    uint32_t *nngb;         // same order, or null
    uint32_t *status;
};

// interval [lo, lo + len] on the circle of 2^32 grid units
__device__ __forceinline__ uint32_t gap_point(uint32_t c, uint32_t lo, uint32_t len) {
    const uint32_t d = c - lo;
    if (d <= len) return 0u;
    const uint32_t fwd = d - len, back = 0u - d;
    return fwd < back ? fwd : back;
}

__device__ __forceinline__ uint32_t gap_boxes(uint32_t alo, uint32_t la, uint32_t blo, uint32_t lb) {
    if (blo - alo <= la || alo - blo <= lb) return 0u;
    const uint32_t a = blo - (alo + la), b = alo - (blo + lb);
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long sq(uint32_t g) {
    return (unsigned long long)g * (unsigned long long)g;
}

// smoothing lengths to grid units in key order; 0 < h < L / 2
__global__ void k_sph_prep(int64_t n, const uint32_t *__restrict__ perm, const float *__restrict__ h,
                           double to_grid, float *__restrict__ hg, uint32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = (double)h[perm ? perm[i] : (uint32_t)i];
    if (!(v > 0.0) || !(v * to_grid < 2147483648.0)) {   // also false for NaN
        atomicOr(status, ST_BAD_INPUT);
        hg[i] = 0.0f;
        return;
    }
    hg[i] = __double2float_rn(v * to_grid);
}

__global__ void __launch_bounds__(32 * kSphWarps) k_sph_density(SphArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t g = (int64_t)blockIdx.x * kSphWarps + warp;
    if (g >= a.ngroups) return;  // the whole warp
    unsigned long long *stk = reinterpret_cast<unsigned long long *>(smem_raw) + (size_t)warp * kSphStack;
    uint4 *chunk = reinterpret_cast<uint4 *>(smem_raw + (size_t)kSphWarps * kSphStack * 8) +
                   (size_t)warp * kSphChunk;

    const uint32_t b = a.gbeg[g], e = a.gend[g];
    const uint32_t me = b + lane;
    const bool active = me < e;
    const uint32_t xi = active ? a.px[me] : 0u, yi = active ? a.py[me] : 0u, zi = active ? a.pz[me] : 0u;
    if (a.done && __all_sync(0xffffffffu, !active || a.done[me] != 0)) return;  // nothing to redo
    const float hgi = active ? a.hg[me] : 0.0f;
    const float h2i = __fmul_rn(hgi, hgi);
    const float inv_h = active && hgi > 0.0f ? 1.0f / hgi : 0.0f;
    // the group's search radius: the largest h, widened by a margin
    const float hmax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(hgi)));
    const unsigned long long hm = (unsigned long long)(hmax * 1.0001f) + 2ull;
    const unsigned long long hm2 = hm * hm;
    uint32_t lo[3], gl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = a.gbox[6 * g + k];
        gl[k] = a.gbox[6 * g + 3 + k] - lo[k];
    }

    float sum = 0.0f;
    uint32_t cnt = 0;
    auto flush = [&](int nc) {
        __syncwarp();
        for (int t = 0; t < nc; ++t) {
            const uint4 c = chunk[t];
            const float fx = (float)(int32_t)(c.x - xi), fy = (float)(int32_t)(c.y - yi),
                        fz = (float)(int32_t)(c.z - zi);
            const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)), __fmul_rn(fz, fz));
            if (r2 < h2i) {
                ++cnt;
                const float q = sqrtf(r2) * inv_h;
                const float u = 1.0f - q;
                const float w = q < 0.5f ? 1.0f - 6.0f * q * q * u : 2.0f * u * u * u;
                sum = fmaf(__uint_as_float(c.w), w, sum);
            }
        }
        __syncwarp();
    };

    int sp = 0, nc = 0;
    if (lane == 0) stk[0] = (unsigned long long)a.ncbeg[0] | ((unsigned long long)a.nccnt[0] << 32);
    sp = 1;
    __syncwarp();
    for (int64_t round = 0; sp > 0 && round < a.max_rounds; ++round) {
        // the top ranges of the stack (lane l holds the l-th from the top) and
        // the running record count over them
        const int top = sp > kSphDeep ? 1 : (sp < 32 ? sp : 32);
        unsigned long long r = 0ull;
        if ((int)lane < top) r = stk[sp - 1 - (int)lane];
        const uint32_t beg = (uint32_t)r, c = (uint32_t)(r >> 32);
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
            if ((int)lane >= d) incl += v;
        }
        const uint32_t excl = incl - c;    // records of the ranges above this one
        // whole ranges while they fit in 32 records; a first range of more than
        // 32 records (a bucket) gives 32 and keeps the rest on the stack
        const unsigned fit = __ballot_sync(0xffffffffu, (int)lane < top && incl <= 32u);
        int take = __popc(fit);            // ranges taken whole (a prefix of the lanes)
        uint32_t total;
        if (take == 0) {
            total = 32;
            if (lane == 0) stk[sp - 1] = (unsigned long long)(beg + 32u) | ((unsigned long long)(c - 32u) << 32);
            take = 1;
        } else {
            total = __shfl_sync(0xffffffffu, incl, take - 1);
            sp -= take;
        }
        __syncwarp();
        // record t of the round belongs to the range l with excl(l) <= t < incl(l):
        // mark where each taken range starts (every range holds a record) and
        // count the starts at or below t
        const unsigned starts = __reduce_or_sync(0xffffffffu, (int)lane < take ? 1u << excl : 0u);
        const uint32_t owner = (uint32_t)__popc(starts & (0xffffffffu >> (31u - lane))) - 1u;
        const uint32_t obeg = __shfl_sync(0xffffffffu, beg, owner);
        const uint32_t oexcl = __shfl_sync(0xffffffffu, excl, owner);
        const bool has = lane < total;
        CRec rec{};
        if (has) rec = a.crec[obeg + (lane - oexcl)];
        const bool node = has && (rec.info >> 31);
        bool push = false, app = false;
        if (node) {
            const uint32_t lev = (rec.info >> 26) & 31u;
            const uint32_t side = 1u << (32u - lev);    // lev >= 1 for a child node
            const uint32_t msk = ~(side - 1u);
            const unsigned long long g2 = sq(gap_boxes(lo[0], gl[0], rec.x & msk, side - 1u)) +
                                          sq(gap_boxes(lo[1], gl[1], rec.y & msk, side - 1u)) +
                                          sq(gap_boxes(lo[2], gl[2], rec.z & msk, side - 1u));
            push = g2 <= hm2;
        } else if (has) {
            const unsigned long long g2 = sq(gap_point(rec.x, lo[0], gl[0])) +
                                          sq(gap_point(rec.y, lo[1], gl[1])) +
                                          sq(gap_point(rec.z, lo[2], gl[2]));
            app = g2 <= hm2;
        }
        const unsigned bp = __ballot_sync(0xffffffffu, push);
        if (push) {
            const int pos = sp + __popc(bp & lt);
            if (pos < kSphStack) stk[pos] = (unsigned long long)rec.ref | ((unsigned long long)(rec.info & 0x3ffffffu) << 32);
            else atomicOr(a.status, ST_STACK_OVF);
        }
        sp += __popc(bp);
        if (sp > kSphStack) sp = kSphStack;
        const unsigned ba = __ballot_sync(0xffffffffu, app);
        if (app) chunk[nc + __popc(ba & lt)] = make_uint4(rec.x, rec.y, rec.z, __float_as_uint(rec.m));
        nc += __popc(ba);
        if (nc > kSphChunk - 32) {
            flush(nc);
            nc = 0;
        }
        __syncwarp();
    }
    if (sp > 0) atomicOr(a.status, ST_INTERNAL);   // the round bound was reached
    flush(nc);
    if (active) {
        const uint32_t i = a.perm ? a.perm[me] : me;
        const double hd = (double)hgi;
        a.rho[i] = __double2float_rn(a.dens * (double)sum / (hd * hd * hd));
        if (a.nngb) a.nngb[i] = cnt;
    }
}

// One step of the smoothing-length iteration for every particle not yet
// converged (key order): N_eff = (4 pi / 3) h^3 rho / m against the target N.
// Within tol N it is done; else the step keeps a bracket [lo, hi] of h (lo:
// too few neighbours, hi: too many), expands or shrinks h by 1.26 until both
// ends are known, then bisects in volume, h = cbrt((lo^3 + hi^3) / 2).  A
// particle whose h would reach the cap (just below L / 2) stops there.
__global__ void k_sph_update(int64_t n, double nt, double tol, double hcap, const double *__restrict__ m,
                             const float *__restrict__ rho, float *__restrict__ h, float *__restrict__ lo,
                             float *__restrict__ hi, uint8_t *__restrict__ done,
                             unsigned long long *__restrict__ left) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || done[i]) return;
    const double hh = (double)h[i];
    if (!(m[i] > 0.0)) {   // a massless particle has no neighbour relation to meet
        done[i] = 1;
        return;
    }
    const double neff = (4.0 * M_PI / 3.0) * hh * hh * hh * (double)rho[i] / m[i];
    if (fabs(neff - nt) <= tol * nt) {
        done[i] = 1;
        return;
    }
    double l = (double)lo[i], u = (double)hi[i];
    if (neff < nt) l = hh; else u = hh;
    double next;
    if (l > 0.0 && u > 0.0) next = cbrt(0.5 * (l * l * l + u * u * u));
    else next = (neff < nt) ? hh * 1.26 : hh / 1.26;
    lo[i] = (float)l;
    hi[i] = (float)u;
    if (next >= hcap) {
        next = hcap;
        if (hh >= hcap) {   // already at the cap and still too few neighbours
            done[i] = 1;
            return;
        }
    }
    h[i] = (float)next;
    atomicAdd(left, 1ull);
}

__global__ void k_sph_to_caller(int64_t n, const uint32_t *__restrict__ perm, const float *__restrict__ hs,
                                const float *__restrict__ rs, const uint32_t *__restrict__ cs,
                                float *__restrict__ h, float *__restrict__ rho, uint32_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    h[j] = hs[i];
    rho[j] = rs[i];
    if (cnt) cnt[j] = cs[i];
}

__global__ void k_sph_gather(int64_t n, const uint32_t *__restrict__ perm, const float *__restrict__ h,
                             float *__restrict__ hs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    hs[i] = h[perm[i]];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace og

using namespace og;

extern "C" og_status og_tree_sph_density(og_tree *t, const float *h, float *rho, uint32_t *n_ngb) {
    if (!t || !h || !rho) { set_error("og_tree_sph_density: NULL argument"); return OG_ERR_ARG; }
    if (t->nseg != 1) { set_error("og_tree_sph_density: a tree of one box only"); return OG_ERR_ARG; }
    if (t->refit) { set_error("og_tree_sph_density: a refitted tree (rebuild it)"); return OG_ERR_STATE; }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int64_t n = t->n;
    if (n == 0) return OG_OK;
    const bool dev = (t->prm.flags & OG_DEVICE_PTRS) != 0;
    const double half = 0.5 * t->prm.box;
    if (!dev)
        for (int64_t i = 0; i < n; ++i)
            if (!(h[i] > 0.0f) || !((double)h[i] < half)) {
                set_error("og_tree_sph_density: h[%lld] = %g is not in (0, L/2)", (long long)i, (double)h[i]);
                return OG_ERR_ARG;
            }
    const size_t bh = (size_t)n * sizeof(float);
    // scratch: hg (sorted) [+ host staging: h in, rho and counts out]
    const size_t off_in = (bh + 255) & ~(size_t)255;
    const size_t total = off_in + (dev ? 0 : 3 * off_in);
    char *buf = nullptr;
    cudaError_t e = dev_malloc_async(&buf, total, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (sph)");
    float *hg = reinterpret_cast<float *>(buf);
    const float *d_h = h;
    float *d_rho = rho;
    uint32_t *d_cnt = n_ngb;
    if (!dev) {
        float *hin = reinterpret_cast<float *>(buf + off_in);
        cudaMemcpyAsync(hin, h, bh, cudaMemcpyHostToDevice, s);
        d_h = hin;
        d_rho = reinterpret_cast<float *>(buf + 2 * off_in);
        d_cnt = n_ngb ? reinterpret_cast<uint32_t *>(buf + 3 * off_in) : nullptr;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    const double to_grid = 4294967296.0 / t->prm.box;
    k_sph_prep<<<nblk(n, 256), 256, 0, s>>>(n, t->perm, d_h, to_grid, hg, c->d_status); note_launch();
    SphArgs a;
    a.crec = t->crec;
    a.ncbeg = t->ncbeg;
    a.nccnt = t->nccnt;
    a.gbeg = t->gbeg;
    a.gend = t->gend;
    a.gbox = t->gbox;
    a.px = t->px;
    a.py = t->py;
    a.pz = t->pz;
    a.perm = t->perm;
    a.done = nullptr;
    a.hg = hg;
    a.ngroups = t->ngroups;
    a.max_rounds = t->nnodes + 2 + (n + 31) / 32;
    a.dens = 8.0 / M_PI * to_grid * to_grid * to_grid;
    a.rho = d_rho;
    a.nngb = d_cnt;
    a.status = c->d_status;
    if (t->ngroups > 0) {
        k_sph_density<<<nblk(t->ngroups, kSphWarps), 32 * kSphWarps, kSphSmem, s>>>(a); note_launch();
    }
    cudaEventRecord(e1, s);
    if (!dev) {
        cudaMemcpyAsync(rho, d_rho, bh, cudaMemcpyDeviceToHost, s);
        if (n_ngb) cudaMemcpyAsync(n_ngb, d_cnt, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    }
    cudaFreeAsync(buf, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "sph density");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->ms_sph = ms;
    return check_status(c);
}

extern "C" og_status og_tree_sph_smoothing(og_tree *t, double n_target, double tol, int32_t max_iter,
                                           float *h, float *rho, uint32_t *n_ngb, int32_t *iters) {
    if (!t || !h || !rho) { set_error("og_tree_sph_smoothing: NULL argument"); return OG_ERR_ARG; }
    if (t->nseg != 1) { set_error("og_tree_sph_smoothing: a tree of one box only"); return OG_ERR_ARG; }
    if (t->refit) { set_error("og_tree_sph_smoothing: a refitted tree (rebuild it)"); return OG_ERR_STATE; }
    if (!(n_target > 32.0 / 3.0) || !std::isfinite(n_target) || !(tol > 0.0) || !(tol < 1.0) ||
        max_iter < 1 || max_iter > 1000) {
        set_error("og_tree_sph_smoothing: need N > 32/3 (the self term), 0 < tol < 1, 1 <= max_iter <= 1000");
        return OG_ERR_ARG;
    }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int64_t n = t->n;
    const bool dev = (t->prm.flags & OG_DEVICE_PTRS) != 0;
    const double half = 0.5 * t->prm.box;
    if (!dev)
        for (int64_t i = 0; i < n; ++i)
            if (!(h[i] > 0.0f) || !((double)h[i] < half)) {
                set_error("og_tree_sph_smoothing: h[%lld] = %g is not in (0, L/2)", (long long)i, (double)h[i]);
                return OG_ERR_ARG;
            }
    // key-order state: h, lo, hi, grid h, rho, counts (4 B each), done (1 B); a
    // counter; host staging of h in/out, rho and counts out
    const size_t b4 = ((size_t)n * 4 + 255) & ~(size_t)255, b1 = ((size_t)n + 255) & ~(size_t)255;
    const size_t total = 6 * b4 + b1 + 256 + (dev ? 0 : 3 * b4);
    char *buf = nullptr;
    cudaError_t e = dev_malloc_async(&buf, total, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (sph smoothing)");
    float *hs = reinterpret_cast<float *>(buf), *lo = reinterpret_cast<float *>(buf + b4);
    float *hi = reinterpret_cast<float *>(buf + 2 * b4), *hg = reinterpret_cast<float *>(buf + 3 * b4);
    float *rs = reinterpret_cast<float *>(buf + 4 * b4);
    uint32_t *cs = reinterpret_cast<uint32_t *>(buf + 5 * b4);
    uint8_t *done = reinterpret_cast<uint8_t *>(buf + 6 * b4);
    unsigned long long *left = reinterpret_cast<unsigned long long *>(buf + 6 * b4 + b1);
    float *d_h = h, *d_rho = rho;
    uint32_t *d_cnt = n_ngb;
    if (!dev) {
        char *st = buf + 6 * b4 + b1 + 256;
        d_h = reinterpret_cast<float *>(st);
        d_rho = reinterpret_cast<float *>(st + b4);
        d_cnt = n_ngb ? reinterpret_cast<uint32_t *>(st + 2 * b4) : nullptr;
        cudaMemcpyAsync(d_h, h, (size_t)n * 4, cudaMemcpyHostToDevice, s);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    k_sph_gather<<<nblk(n, 256), 256, 0, s>>>(n, t->perm, d_h, hs); note_launch();
    cudaMemsetAsync(lo, 0, 2 * b4, s);   // lo and hi: no bracket yet
    cudaMemsetAsync(done, 0, b1, s);
    const double to_grid = 4294967296.0 / t->prm.box;
    SphArgs a;
    a.crec = t->crec;
    a.ncbeg = t->ncbeg;
    a.nccnt = t->nccnt;
    a.gbeg = t->gbeg;
    a.gend = t->gend;
    a.gbox = t->gbox;
    a.px = t->px;
    a.py = t->py;
    a.pz = t->pz;
    a.perm = nullptr;
    a.done = done;
    a.hg = hg;
    a.ngroups = t->ngroups;
    a.max_rounds = t->nnodes + 2 + (n + 31) / 32;
    a.dens = 8.0 / M_PI * to_grid * to_grid * to_grid;
    a.rho = rs;
    a.nngb = cs;
    a.status = c->d_status;
    const double hcap = std::nextafter((float)(half * 0.999), 0.0f);
    int32_t it = 0;
    og_status st = OG_OK;
    while (it < max_iter) {
        k_sph_prep<<<nblk(n, 256), 256, 0, s>>>(n, nullptr, hs, to_grid, hg, c->d_status); note_launch();
        k_sph_density<<<nblk(t->ngroups, kSphWarps), 32 * kSphWarps, kSphSmem, s>>>(a); note_launch();
        ++it;
        cudaMemsetAsync(left, 0, sizeof(unsigned long long), s);
        k_sph_update<<<nblk(n, 256), 256, 0, s>>>(n, n_target, tol, hcap, t->pm64, rs, hs, lo, hi, done, left);
        note_launch();
        unsigned long long h_left = 0;
        cudaMemcpyAsync(&h_left, left, sizeof(h_left), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { st = cuda_fail(e, "sph smoothing"); break; }
        if (h_left == 0) break;
    }
    if (st == OG_OK) {
        // the densities and counts at the final h (a particle that moved in the
        // last step needs them at its new h)
        a.done = nullptr;
        k_sph_prep<<<nblk(n, 256), 256, 0, s>>>(n, nullptr, hs, to_grid, hg, c->d_status); note_launch();
        k_sph_density<<<nblk(t->ngroups, kSphWarps), 32 * kSphWarps, kSphSmem, s>>>(a); note_launch();
        k_sph_to_caller<<<nblk(n, 256), 256, 0, s>>>(n, t->perm, hs, rs, cs, d_h, d_rho, d_cnt); note_launch();
        cudaEventRecord(e1, s);
        if (!dev) {
            cudaMemcpyAsync(h, d_h, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(rho, d_rho, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
            if (n_ngb) cudaMemcpyAsync(n_ngb, d_cnt, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
        }
    }
    cudaFreeAsync(buf, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess && st == OG_OK) st = cuda_fail(e, "sph smoothing");
    float ms = 0.f;
    if (st == OG_OK) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    t->ms_sph = ms;
    if (iters) *iters = it;
    return check_status(c);
}
