// og_capi.cu -- the C-ABI entry points of include/og.h.
//
// Host-side responsibilities: argument validation, the context (device,
// stream, stream-ordered memory pool, device status word), host<->device
// copies for host-pointer calls, the two-pass relative opening
// (Sect. 4.1.2: the relative criterion needs the previous acceleration; a
// Barnes-Hut pass supplies it when the caller has none), and the final
// reordering to the caller's particle order.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <unordered_set>

#include "og_internal.h"

namespace og {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

og_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? OG_ERR_OOM : OG_ERR_CUDA;
}

// injected allocation failures (og_debug_fail_allocations): allocations to
// let through first, then allocations to fail
static std::mutex g_inject_mu;
static int64_t g_inject_skip = 0, g_inject_fail = 0;
static std::atomic<bool> g_inject_on{false};

cudaError_t dev_malloc_raw(void **p, size_t bytes, cudaStream_t s) {
    if (g_inject_on.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_inject_mu);
        if (g_inject_fail > 0) {
            if (g_inject_skip > 0) {
                --g_inject_skip;
            } else {
                --g_inject_fail;
                if (g_inject_fail == 0) g_inject_on.store(false);
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
        }
    }
    return cudaMallocAsync(p, bytes, s);
}

namespace {

constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

__global__ void k_gather_aold(int64_t n, const uint32_t *__restrict__ perm,
                              const float *__restrict__ a_old, float *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t j = perm[i];
    out[i] = a_old[3ull * j + 0];
    out[n + i] = a_old[3ull * j + 1];
    out[2 * n + i] = a_old[3ull * j + 2];
}

// Outputs in caller order, gathered: caller index j reads sorted position
// inv[j] (the sorted arrays were just written by the walk and sit in L2), and
// the stores of consecutive j are contiguous.
__global__ void k_unpermute(int64_t n, const uint32_t *__restrict__ inv,
                            const float *__restrict__ acc_sorted,
                            const uint32_t *__restrict__ npp_s, const uint32_t *__restrict__ npn_s,
                            float *acc, uint32_t *npp, uint32_t *npn) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t i = inv[j];
    if (acc) {
        acc[3ull * j + 0] = acc_sorted[i];
        acc[3ull * j + 1] = acc_sorted[n + i];
        acc[3ull * j + 2] = acc_sorted[2 * n + i];
    }
    if (npp) npp[j] = npp_s[i];
    if (npn) npn[j] = npn_s[i];
}

// FP64 output: the walk's unscaled FP32 sums times G (2^32 / L)^2 in FP64
__global__ void k_unpermute_f64(int64_t n, const uint32_t *__restrict__ inv,
                                const float *__restrict__ acc_sorted,
                                const uint32_t *__restrict__ npp_s, const uint32_t *__restrict__ npn_s,
                                double scale, double *acc, uint32_t *npp, uint32_t *npn) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t i = inv[j];
    acc[3ull * j + 0] = (double)acc_sorted[i] * scale;
    acc[3ull * j + 1] = (double)acc_sorted[n + i] * scale;
    acc[3ull * j + 2] = (double)acc_sorted[2 * n + i] * scale;
    if (npp) npp[j] = npp_s[i];
    if (npn) npn[j] = npn_s[i];
}

__global__ void k_unpermute_pot(int64_t n, const uint32_t *__restrict__ inv,
                                const float *__restrict__ pot_sorted, float *pot) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    pot[j] = pot_sorted[inv[j]];
}

// 1 for a group holding at least one active particle (active: caller order)
__global__ void k_group_active(int64_t ng, const uint32_t *__restrict__ gbeg,
                               const uint32_t *__restrict__ gend, const uint32_t *__restrict__ perm,
                               const uint8_t *__restrict__ active, int64_t n, uint32_t *flag) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    uint32_t f = 0;
    const uint32_t e = gend[g] < (uint64_t)n ? gend[g] : (uint32_t)n;
    for (uint32_t i = gbeg[g]; i < e && !f; ++i) f = active[perm[i]] != 0;
    flag[g] = f;
}

// the flagged groups' ids, in key order, at their exclusive-scan positions
__global__ void k_group_compact(int64_t ng, const uint32_t *__restrict__ flag,
                                const uint32_t *__restrict__ pos, uint32_t *out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng && flag[g]) out[pos[g]] = (uint32_t)g;
}

// k_unpermute for the active particles only
__global__ void k_unpermute_active(int64_t n, const uint32_t *__restrict__ inv,
                                   const uint8_t *__restrict__ active,
                                   const float *__restrict__ acc_sorted,
                                   const uint32_t *__restrict__ npp_s,
                                   const uint32_t *__restrict__ npn_s, float *acc, uint32_t *npp,
                                   uint32_t *npn) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || !active[j]) return;
    const uint32_t i = inv[j];
    acc[3ull * j + 0] = acc_sorted[i];
    acc[3ull * j + 1] = acc_sorted[n + i];
    acc[3ull * j + 2] = acc_sorted[2 * n + i];
    if (npp) npp[j] = npp_s[i];
    if (npn) npn[j] = npn_s[i];
}

}  // namespace

// trees handed out by og_tree_build, so that og_destroy can free the ones the
// caller did not
struct LiveTrees {
    std::mutex mu;
    std::unordered_set<og_tree *> set;
};

void live_add(og_ctx *c, og_tree *t) {
    if (!c->live) c->live = new (std::nothrow) LiveTrees();
    LiveTrees *L = static_cast<LiveTrees *>(c->live);
    if (!L) return;
    std::lock_guard<std::mutex> lk(L->mu);
    L->set.insert(t);
}

void live_remove(og_tree *t) {
    LiveTrees *L = t->ctx ? static_cast<LiveTrees *>(t->ctx->live) : nullptr;
    if (!L) return;
    std::lock_guard<std::mutex> lk(L->mu);
    L->set.erase(t);
}

og_status check_status(og_ctx *c) {
    uint32_t *h = pinned_status(c);
    cudaError_t e = cudaMemcpyAsync(h, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    return status_from(c, *h);
}

og_status status_from(og_ctx *c, uint32_t st) {
    if (st == 0) return OG_OK;
    cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), c->stream);
    cudaStreamSynchronize(c->stream);
    if (st & ST_BAD_INPUT) {
        set_error("non-finite position, negative/non-finite mass, or a smoothing length out of (0, L/2)");
        return OG_ERR_ARG;
    }
    if (st & ST_MASS_RANGE) {
        set_error("masses span more than 128 binary orders (from the lowest set bit of the smallest "
                  "to the top of the largest): the exact node moments hold at most that");
        return OG_ERR_ARG;
    }
    if (st & ST_STACK_OVF) {
        set_error("walk stack overflow");
        return OG_ERR_OVERFLOW;
    }
    if (st & ST_LIST_OVF) {
        set_error("debug list buffer overflow");
        return OG_ERR_OVERFLOW;
    }
    if (st & ST_TIMEOUT) {
        set_error("a device-side wait on another block ran out (the look-back of a one-kernel sort "
                  "pass or scan)");
        return OG_ERR_TIMEOUT;
    }
    set_error("internal consistency check failed (status 0x%x)", st);
    return OG_ERR_STATE;
}

og_status validate(const og_params *p, int64_t n) {
    if (!p) { set_error("params is NULL"); return OG_ERR_ARG; }
    if (n < 1 || n > kMaxN) { set_error("N = %lld out of range [1, %lld]", (long long)n, (long long)kMaxN); return OG_ERR_ARG; }
    if (!(p->box > 0.0) || !std::isfinite(p->box)) { set_error("box must be finite and > 0"); return OG_ERR_ARG; }
    if (!std::isfinite(p->G) || !std::isfinite(p->eps) || p->eps < 0.0) { set_error("G and eps must be finite, eps >= 0"); return OG_ERR_ARG; }
    if (!std::isfinite(p->r_s)) { set_error("r_s must be finite"); return OG_ERR_ARG; }
    if (p->r_s > 0.0) {
        double rc = p->rcut_over_rs * p->r_s;
        if (!(rc > 0.0) || !(rc < 0.5 * p->box)) { set_error("cutoff radius must satisfy 0 < r_cut < box/2"); return OG_ERR_ARG; }
    }
    if (p->opening != OG_OPEN_BH && p->opening != OG_OPEN_REL) { set_error("unknown opening criterion"); return OG_ERR_ARG; }
    if (!(p->theta >= 0.0) || !std::isfinite(p->theta)) { set_error("theta must be >= 0"); return OG_ERR_ARG; }
    if (!(p->alpha >= 0.0) || !std::isfinite(p->alpha)) { set_error("alpha must be >= 0"); return OG_ERR_ARG; }
    if (!(p->theta_first_pass >= 0.0)) { set_error("theta_first_pass must be >= 0"); return OG_ERR_ARG; }
    if (p->leaf_max != 1) { set_error("leaf_max must be 1 (one particle per leaf cell)"); return OG_ERR_ARG; }
    if (p->group_max < 0 || p->group_max > 32) { set_error("group_max must be in [0, 32]"); return OG_ERR_ARG; }
    if (p->walk_warps < 0 || p->walk_warps > 8) { set_error("walk_warps must be in [0, 8]"); return OG_ERR_ARG; }
    if (p->walk_chunk != 0 && (p->walk_chunk < 64 || p->walk_chunk > 1024)) {
        set_error("walk_chunk must be 0 or in [64, 1024]");
        return OG_ERR_ARG;
    }
    return OG_OK;
}

}  // namespace og

using namespace og;

extern "C" {

const char *og_last_error(void) { return g_err; }

int64_t og_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

og_status og_debug_scan_wait_timeout(og_ctx *c, int64_t n) {
    if (!c) { set_error("og_debug_scan_wait_timeout: NULL context"); return OG_ERR_ARG; }
    og_status st = scan_wait_timeout_probe(c, n);
    if (st != OG_OK) return st;
    // the status word: the probe's wait must have run out
    uint32_t *h = pinned_status(c);
    cudaMemcpyAsync(h, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "og_debug_scan_wait_timeout");
    return status_from(c, *h);
}

og_status og_debug_fail_allocations(int32_t skip, int32_t count) {
    if (skip < 0 || count < 0) {
        set_error("og_debug_fail_allocations: skip and count must be >= 0");
        return OG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_skip = skip;
    g_inject_fail = count;
    g_inject_on.store(count > 0);
    return OG_OK;
}

og_status og_device_code_version(int32_t *version) {
    if (!version) {
        set_error("og_device_code_version: NULL pointer");
        return OG_ERR_ARG;
    }
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, k_unpermute);
    if (e != cudaSuccess) return cuda_fail(e, "og_device_code_version: cudaFuncGetAttributes");
    *version = at.binaryVersion;
    return OG_OK;
}

og_status og_params_default(og_params *p) {
    if (!p) return OG_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->box = 1.0;
    p->G = 1.0;
    p->eps = 0.0;
    p->r_s = 0.0;
    p->rcut_over_rs = 4.5;
    p->theta = 0.5;
    p->alpha = 0.005;
    p->theta_first_pass = 0.5;
    p->opening = OG_OPEN_BH;
    p->leaf_max = 1;
    p->group_max = 32;
    p->flags = 0;
    return OG_OK;
}

og_status og_create(og_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) { set_error("ctx is NULL"); return OG_ERR_ARG; }
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) { set_error("no CUDA device %d", device); return OG_ERR_ARG; }
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    og_ctx *c = new (std::nothrow) og_ctx();
    if (!c) { set_error("host allocation failed"); return OG_ERR_OOM; }
    c->device = device;
    c->hbm_budget = hbm_budget_bytes;
    if ((e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    c->stream = c->own_stream;
    if ((e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_to_side, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_from_side, cudaEventDisableTiming)) != cudaSuccess) {
        if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
        if (c->ev_to_side) cudaEventDestroy(c->ev_to_side);
        cudaStreamDestroy(c->own_stream);
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    // keep freed blocks in the stream-ordered pool: repeated builds reuse them
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if ((e = cudaMalloc(&c->d_status, 256)) != cudaSuccess) {
        cudaEventDestroy(c->ev_to_side);
        cudaEventDestroy(c->ev_from_side);
        cudaStreamDestroy(c->copy_stream);
        cudaStreamDestroy(c->own_stream);
        delete c;
        return cuda_fail(e, "cudaMalloc");
    }
    c->d_counters = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(c->d_status) + 64);
    if ((e = cudaMallocHost(&c->h_pinned, 256)) != cudaSuccess) {
        cudaFree(c->d_status);
        cudaEventDestroy(c->ev_to_side);
        cudaEventDestroy(c->ev_from_side);
        cudaStreamDestroy(c->copy_stream);
        cudaStreamDestroy(c->own_stream);
        delete c;
        return cuda_fail(e, "cudaMallocHost");
    }
    memset(c->h_pinned, 0, 256);
    cudaMemset(c->d_status, 0, 256);
    cudaDeviceSynchronize();
    *out = c;
    return OG_OK;
}

og_status og_destroy(og_ctx *c) {
    if (!c) return OG_OK;
    serve_shutdown(c);
    og::tune_free(c);
    og::pm_free(c);
    if (c->live) {
        // trees the caller did not free
        LiveTrees *L = static_cast<LiveTrees *>(c->live);
        std::vector<og_tree *> left;
        {
            std::lock_guard<std::mutex> lk(L->mu);
            left.assign(L->set.begin(), L->set.end());
        }
        for (og_tree *t : left) og_tree_free(t);
        delete L;
        c->live = nullptr;
    }
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_status);
    cudaFreeHost(c->h_pinned);
    cudaStreamSynchronize(c->copy_stream);
    cudaEventDestroy(c->ev_to_side);
    cudaEventDestroy(c->ev_from_side);
    cudaStreamDestroy(c->copy_stream);
    cudaStreamDestroy(c->own_stream);
    delete c;
    return OG_OK;
}

og_status og_set_stream(og_ctx *c, void *stream) {
    if (!c) { set_error("ctx is NULL"); return OG_ERR_ARG; }
    c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
    return OG_OK;
}

og_status og_tree_build(og_ctx *c, const double *pos, const double *mass, int64_t n,
                        const og_params *p, og_tree **out) {
    if (!out) { set_error("out is NULL"); return OG_ERR_ARG; }
    *out = nullptr;
    if (!c || !pos || !mass) { set_error("NULL argument"); return OG_ERR_ARG; }
    og_status st = validate(p, n);
    if (st) return st;
    cudaSetDevice(c->device);
    og_tree *t = new (std::nothrow) og_tree();
    if (!t) { set_error("host allocation failed"); return OG_ERR_OOM; }
    t->ctx = c;
    t->prm = *p;
    t->n = n;
    t->nseg = 1;
    t->h_seg_off = {0u, (uint32_t)n};
    cudaStream_t s = c->stream;
    const double *d_pos = pos, *d_mass = mass;
    void *staging = nullptr;
    cudaError_t e;
    if (!(p->flags & OG_DEVICE_PTRS)) {
        size_t bytes = (size_t)n * 4 * sizeof(double);
        if ((e = dev_malloc_async(&staging, bytes, s)) != cudaSuccess) {
            delete t;
            return cuda_fail(e, "cudaMallocAsync (inputs)");
        }
        double *dp = static_cast<double *>(staging);
        cudaMemcpyAsync(dp, pos, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, s);
        // the masses follow on the side stream once the positions are in (the
        // link is not shared with them), beside the quantization and the sort;
        // the build waits for them before it first reads them
        cudaEventRecord(c->ev_to_side, s);
        cudaStreamWaitEvent(c->copy_stream, c->ev_to_side, 0);
        cudaMemcpyAsync(dp + 3 * n, mass, (size_t)n * sizeof(double), cudaMemcpyHostToDevice,
                        c->copy_stream);
        cudaEventRecord(c->ev_from_side, c->copy_stream);
        t->mass_ready = c->ev_from_side;
        d_pos = dp;
        d_mass = dp + 3 * n;
    }
    if (t->prm.group_max == 0) {
        // measured group size and walk launch shape for this kind of input
        // (og_tune.cu); explicit launch-shape fields stay as given.  The
        // tuner's builds read the masses at once.
        if (t->mass_ready) cudaStreamWaitEvent(s, t->mass_ready, 0);
        WalkConfig w{32, kDefaultWalkWarps, kDefaultWalkChunk};
        st = tuned_walk(c, d_pos, d_mass, n, t->prm, &w);
        if (st) {
            if (staging) cudaFreeAsync(staging, s);
            delete t;
            return st;
        }
        t->prm.group_max = w.group_max;
        if (t->prm.walk_warps == 0) t->prm.walk_warps = w.warps;
        if (t->prm.walk_chunk == 0) t->prm.walk_chunk = w.chunk;
    }
    if (t->prm.walk_warps == 0) t->prm.walk_warps = kDefaultWalkWarps;
    if (t->prm.walk_chunk == 0) t->prm.walk_chunk = kDefaultWalkChunk;
    t->seg_prm.assign(1, t->prm);
    st = build_tree(t, d_pos, d_mass);
    // the staging buffer is freed in stream order after the masses' copy,
    // also when the build stopped before it waited for them
    if (t->mass_ready) cudaStreamWaitEvent(s, t->mass_ready, 0);
    t->mass_ready = nullptr;
    if (staging) cudaFreeAsync(staging, s);
    if (st == OG_OK) st = status_from(c, t->build_status);   // read by the build's synchronisation
    if (st != OG_OK) {
        og_tree_free(t);
        return st;
    }
    live_add(c, t);
    *out = t;
    return OG_OK;
}

}  // extern "C"

namespace og {

// Both passes of the force on a built tree (sorted order, device results in
// t->a_sorted, t->npp_sorted, t->npn_sorted).  d_aold: previous accelerations
// in input order on the device, or null.
og_status force_sorted(og_tree *t, const float *d_aold, float *ms_walk_out, const uint32_t *subset,
                       int64_t nsubset, float *pot_sorted, bool defer) {
    cudaStream_t s = t->ctx->stream;
    const int64_t n = t->n;
    cudaError_t e;
    float ms_walk = 0, ms = 0;
    t->interactions = 0;
    if (t->prm.flags & OG_DEBUG_DUMP_LISTS) {
        if (!t->lists) {
            t->list_cap = (int64_t)1 << 28;
            if ((e = cudaMalloc(&t->lists, (size_t)t->list_cap * 2 * sizeof(uint32_t))) != cudaSuccess) {
                t->lists = nullptr;
                return cuda_fail(e, "cudaMalloc (lists)");
            }
        }
        t->list_len = 0;
    }
    const float *a_old_sorted = nullptr;
    if (t->prm.opening == OG_OPEN_REL) {
        if (d_aold) {
            k_gather_aold<<<nblk(n), kT, 0, s>>>(n, t->perm, d_aold, t->a_old_sorted); note_launch();
        } else {
            // first pass: Barnes-Hut with theta_first_pass
            og_status st = walk_pass(t, OG_OPEN_BH, true, nullptr, t->a_old_sorted, &ms, false,
                                     subset, nsubset, nullptr, defer);
            if (st) return st;
            ms_walk += ms;
        }
        a_old_sorted = t->a_old_sorted;
    }
    og_status st = walk_pass(t, t->prm.opening, false, a_old_sorted, t->a_sorted, &ms, true,
                             subset, nsubset, pot_sorted, defer);
    if (st) return st;
    ms_walk += ms;
    if (ms_walk_out) *ms_walk_out = ms_walk;
    return OG_OK;
}

}  // namespace og

extern "C" {

og_status og_tree_force(og_tree *t, const float *a_old, float *acc, uint32_t *n_pp,
                        uint32_t *n_pn) {
    if (!t || !acc) { set_error("NULL argument"); return OG_ERR_ARG; }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int64_t n = t->n;
    const bool dev = (t->prm.flags & OG_DEVICE_PTRS) != 0;
    cudaError_t e;
    float ms_walk = 0, ms = 0;
    void *tmp = nullptr;
    const float *d_aold = nullptr;
    // on an error after passes were enqueued: wait for them, then drop them
    auto fail = [&](og_status st) {
        cudaStreamSynchronize(s);
        finish_deferred(t, nullptr);
        return st;
    };
    if (t->prm.opening == OG_OPEN_REL && a_old) {
        d_aold = a_old;
        if (!dev) {
            if ((e = dev_malloc_async(&tmp, (size_t)n * 3 * sizeof(float), s)) != cudaSuccess)
                return cuda_fail(e, "cudaMallocAsync (a_old)");
            cudaMemcpyAsync(tmp, a_old, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
            d_aold = static_cast<const float *>(tmp);
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    // the passes are enqueued without waiting: one host synchronisation for
    // the whole call, after the results and the status word are copied back
    og_status st = force_sorted(t, d_aold, &ms_walk, nullptr, 0, t->pot_next, true);
    if (tmp) cudaFreeAsync(tmp, s);
    float *d_acc = acc;
    uint32_t *d_npp = n_pp, *d_npn = n_pn;
    void *out_tmp = nullptr;
    if (st == OG_OK && !dev) {
        size_t bytes = (size_t)n * 3 * sizeof(float) + 2 * (size_t)n * sizeof(uint32_t) + 512;
        if ((e = dev_malloc_async(&out_tmp, bytes, s)) != cudaSuccess) st = cuda_fail(e, "cudaMallocAsync (out)");
        d_acc = static_cast<float *>(out_tmp);
        d_npp = n_pp ? reinterpret_cast<uint32_t *>(d_acc + 3 * n) : nullptr;
        d_npn = n_pn ? reinterpret_cast<uint32_t *>(d_acc + 3 * n) + n : nullptr;
    }
    if (st != OG_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(st);
    }
    // back to caller order
    if (!dev && (n_pp || n_pn)) {
        // host outputs: the counts first, their copy on the side stream beside
        // the accelerations' reordering (the copies share the link, the
        // reordering does not)
        k_unpermute<<<nblk(n), kT, 0, s>>>(n, t->inv, t->a_sorted, t->npp_sorted, t->npn_sorted,
                                           nullptr, d_npp, d_npn); note_launch();
        cudaEventRecord(c->ev_to_side, s);
        cudaStreamWaitEvent(c->copy_stream, c->ev_to_side, 0);
        if (n_pp) cudaMemcpyAsync(n_pp, d_npp, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->copy_stream);
        if (n_pn) cudaMemcpyAsync(n_pn, d_npn, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->copy_stream);
        cudaEventRecord(c->ev_from_side, c->copy_stream);
        k_unpermute<<<nblk(n), kT, 0, s>>>(n, t->inv, t->a_sorted, t->npp_sorted, t->npn_sorted,
                                           d_acc, nullptr, nullptr); note_launch();
        cudaMemcpyAsync(acc, d_acc, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s);
        cudaStreamWaitEvent(s, c->ev_from_side, 0);
        cudaFreeAsync(out_tmp, s);
    } else {
        k_unpermute<<<nblk(n), kT, 0, s>>>(n, t->inv, t->a_sorted, t->npp_sorted, t->npn_sorted,
                                           d_acc, d_npp, d_npn); note_launch();
        if (!dev) {
            cudaMemcpyAsync(acc, d_acc, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s);
            cudaFreeAsync(out_tmp, s);
        }
    }
    cudaEventRecord(e1, s);
    uint32_t *hst = pinned_status(c);
    cudaMemcpyAsync(hst, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    st = finish_deferred(t, &ms_walk);
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "force");
    if (st != OG_OK) return st;
    t->ms_force = ms;
    t->ms_walk = ms_walk;
    return status_from(c, *hst);
}

og_status og_tree_force_f64(og_tree *t, const float *a_old, double *acc, uint32_t *n_pp,
                            uint32_t *n_pn) {
    if (!t || !acc) { set_error("NULL argument"); return OG_ERR_ARG; }
    if (t->nseg != 1) { set_error("og_tree_force_f64: a tree of one box only"); return OG_ERR_ARG; }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int64_t n = t->n;
    const bool dev = (t->prm.flags & OG_DEVICE_PTRS) != 0;
    cudaError_t e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    float ms_walk = 0, ms = 0;
    void *tmp = nullptr;
    const float *d_aold = nullptr;
    if (t->prm.opening == OG_OPEN_REL && a_old) {
        d_aold = a_old;
        if (!dev) {
            if ((e = dev_malloc_async(&tmp, (size_t)n * 3 * sizeof(float), s)) != cudaSuccess)
                return cuda_fail(e, "cudaMallocAsync (a_old)");
            cudaMemcpyAsync(tmp, a_old, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
            d_aold = static_cast<const float *>(tmp);
        }
    }
    t->unscaled_out = true;
    og_status st = force_sorted(t, d_aold, &ms_walk, nullptr, 0, nullptr);
    t->unscaled_out = false;
    if (tmp) cudaFreeAsync(tmp, s);
    if (st) return st;
    const double g = 4294967296.0 / t->prm.box;
    const double scale = t->prm.G * g * g;
    double *d_acc = acc;
    uint32_t *d_npp = n_pp, *d_npn = n_pn;
    void *out_tmp = nullptr;
    if (!dev) {
        size_t bytes = (size_t)n * 3 * sizeof(double) + 2 * (size_t)n * sizeof(uint32_t) + 512;
        if ((e = dev_malloc_async(&out_tmp, bytes, s)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (out)");
        d_acc = static_cast<double *>(out_tmp);
        d_npp = n_pp ? reinterpret_cast<uint32_t *>(d_acc + 3 * n) : nullptr;
        d_npn = n_pn ? reinterpret_cast<uint32_t *>(d_acc + 3 * n) + n : nullptr;
    }
    k_unpermute_f64<<<nblk(n), kT, 0, s>>>(n, t->inv, t->a_sorted, t->npp_sorted, t->npn_sorted,
                                           scale, d_acc, d_npp, d_npn); note_launch();
    if (!dev) {
        cudaMemcpyAsync(acc, d_acc, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (n_pp) cudaMemcpyAsync(n_pp, d_npp, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (n_pn) cudaMemcpyAsync(n_pn, d_npn, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(out_tmp, s);
    }
    cudaEventRecord(e1, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "force");
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->ms_force = ms;
    t->ms_walk = ms_walk;
    return check_status(c);
}

og_status og_tree_force_pot(og_tree *t, const float *a_old, float *acc, float *pot,
                            uint32_t *n_pp, uint32_t *n_pn) {
    if (!t || !acc || !pot) { set_error("NULL argument"); return OG_ERR_ARG; }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int64_t n = t->n;
    const bool dev = (t->prm.flags & OG_DEVICE_PTRS) != 0;
    cudaError_t e;
    void *tmp = nullptr;
    if ((e = dev_malloc_async(&tmp, (size_t)n * 2 * sizeof(float) + 512, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync (potential)");
    float *pot_sorted = static_cast<float *>(tmp);
    float *d_pot = dev ? pot : pot_sorted + ((n + 63) & ~(int64_t)63);
    // the force call with the potential output of its last pass
    t->pot_next = pot_sorted;
    og_status st = og_tree_force(t, a_old, acc, n_pp, n_pn);
    t->pot_next = nullptr;
    if (st == OG_OK) {
        k_unpermute_pot<<<nblk(n), kT, 0, s>>>(n, t->inv, pot_sorted, d_pot); note_launch();
        if (!dev) cudaMemcpyAsync(pot, d_pot, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "potential");
    }
    cudaFreeAsync(tmp, s);
    return st;
}

og_status og_tree_force_active(og_tree *t, const uint8_t *active, const float *a_old, float *acc,
                               uint32_t *n_pp, uint32_t *n_pn, int64_t *groups_walked) {
    if (!t || !active || !acc) { set_error("NULL argument"); return OG_ERR_ARG; }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int64_t n = t->n, ng = t->ngroups;
    const bool dev = (t->prm.flags & OG_DEVICE_PTRS) != 0;
    cudaError_t e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    // scratch: active mask (host input), group flags, scan positions, group list,
    // count, scan scratch, and for host outputs a staging copy of the outputs
    const size_t al = 256;
    auto up = [&](size_t b) { return (b + al - 1) & ~(al - 1); };
    const size_t b_mask = dev ? 0 : up((size_t)n);
    const size_t b_g = up((size_t)ng * sizeof(uint32_t));
    const size_t b_scan = up(scan_scratch_bytes(ng));
    const size_t b_out = dev ? 0 : up((size_t)n * 3 * sizeof(float)) + 2 * up((size_t)n * sizeof(uint32_t));
    const size_t b_aold = (!dev && a_old && t->prm.opening == OG_OPEN_REL) ? up((size_t)n * 3 * sizeof(float)) : 0;
    void *tmp = nullptr;
    if ((e = dev_malloc_async(&tmp, b_mask + 3 * b_g + al + b_scan + b_out + b_aold, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync (active set)");
    char *q = static_cast<char *>(tmp);
    const uint8_t *d_active = active;
    if (!dev) {
        cudaMemcpyAsync(q, active, (size_t)n, cudaMemcpyHostToDevice, s);
        d_active = reinterpret_cast<const uint8_t *>(q);
        q += b_mask;
    }
    uint32_t *flag = reinterpret_cast<uint32_t *>(q); q += b_g;
    uint32_t *pos = reinterpret_cast<uint32_t *>(q); q += b_g;
    uint32_t *list = reinterpret_cast<uint32_t *>(q); q += b_g;
    uint32_t *d_total = reinterpret_cast<uint32_t *>(q); q += al;
    void *scan_scr = q; q += b_scan;
    float *d_acc = acc;
    uint32_t *d_npp = n_pp, *d_npn = n_pn;
    if (!dev) {
        d_acc = reinterpret_cast<float *>(q); q += up((size_t)n * 3 * sizeof(float));
        d_npp = n_pp ? reinterpret_cast<uint32_t *>(q) : nullptr; q += up((size_t)n * sizeof(uint32_t));
        d_npn = n_pn ? reinterpret_cast<uint32_t *>(q) : nullptr; q += up((size_t)n * sizeof(uint32_t));
    }
    const float *d_aold = nullptr;
    if (t->prm.opening == OG_OPEN_REL && a_old) {
        d_aold = a_old;
        if (!dev) {
            cudaMemcpyAsync(q, a_old, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
            d_aold = reinterpret_cast<const float *>(q);
        }
    }
    k_group_active<<<nblk(ng), kT, 0, s>>>(ng, t->gbeg, t->gend, t->perm, d_active, n, flag); note_launch();
    scan_exclusive_u32(flag, pos, ng, d_total, scan_scr, s);
    k_group_compact<<<nblk(ng), kT, 0, s>>>(ng, flag, pos, list); note_launch();
    uint32_t nact = 0;
    cudaMemcpyAsync(&nact, d_total, sizeof(nact), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        cudaFreeAsync(tmp, s);
        return cuda_fail(e, "active set");
    }
    float ms_walk = 0;
    og_status st = OG_OK;
    t->interactions = 0;
    if (nact > 0) st = force_sorted(t, d_aold, &ms_walk, list, (int64_t)nact);
    if (st == OG_OK && nact > 0) {
        if (!dev) {
            // the inactive entries of the caller's outputs stay as they are
            cudaMemcpyAsync(d_acc, acc, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
            if (n_pp) cudaMemcpyAsync(d_npp, n_pp, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
            if (n_pn) cudaMemcpyAsync(d_npn, n_pn, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
        }
        k_unpermute_active<<<nblk(n), kT, 0, s>>>(n, t->inv, d_active, t->a_sorted, t->npp_sorted,
                                                  t->npn_sorted, d_acc, d_npp, d_npn); note_launch();
        if (!dev) {
            cudaMemcpyAsync(acc, d_acc, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s);
            if (n_pp) cudaMemcpyAsync(n_pp, d_npp, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
            if (n_pn) cudaMemcpyAsync(n_pn, d_npn, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        }
    }
    cudaFreeAsync(tmp, s);
    if (st) return st;
    cudaEventRecord(e1, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "active force");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->ms_force = ms;
    t->ms_walk = ms_walk;
    if (groups_walked) *groups_walked = (int64_t)nact;
    return check_status(c);
}

og_status og_batch_force(og_ctx *c, int64_t nbox, const og_box *boxes, og_batch_info *info) {
    if (!c || !boxes || nbox < 1) { set_error("og_batch_force: NULL argument or no boxes"); return OG_ERR_ARG; }
    const og_params &p0 = boxes[0].params;
    int64_t total = 0;
    for (int64_t b = 0; b < nbox; ++b) {
        const og_box &x = boxes[b];
        if (!x.pos || !x.mass || !x.acc) { set_error("og_batch_force: box %lld has a NULL pointer", (long long)b); return OG_ERR_ARG; }
        og_status st = validate(&x.params, x.n);
        if (st) return st;
        if (x.params.opening != p0.opening || (x.params.r_s > 0.0) != (p0.r_s > 0.0) ||
            x.params.group_max != p0.group_max || x.params.flags != p0.flags ||
            x.params.walk_warps != p0.walk_warps || x.params.walk_chunk != p0.walk_chunk ||
            (x.a_old != nullptr) != (boxes[0].a_old != nullptr)) {
            set_error("og_batch_force: opening, split on/off, group_max, walk_warps, walk_chunk, "
                      "flags and a_old presence must agree across boxes");
            return OG_ERR_ARG;
        }
        total += x.n;
    }
    if (total > kMaxN) { set_error("og_batch_force: %lld particles in total exceed %lld", (long long)total, (long long)kMaxN); return OG_ERR_ARG; }
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const bool dev = (p0.flags & OG_DEVICE_PTRS) != 0;
    const cudaMemcpyKind in_kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind out_kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    og_tree *t = new (std::nothrow) og_tree();
    if (!t) { set_error("host allocation failed"); return OG_ERR_OOM; }
    t->ctx = c;
    t->prm = p0;
    if (t->prm.group_max == 0) t->prm.group_max = 32;
    if (t->prm.walk_warps == 0) t->prm.walk_warps = kDefaultWalkWarps;
    if (t->prm.walk_chunk == 0) t->prm.walk_chunk = kDefaultWalkChunk;
    t->n = total;
    t->nseg = nbox;
    t->seg_prm.resize((size_t)nbox);
    t->h_seg_off.resize((size_t)nbox + 1);
    uint32_t off = 0;
    for (int64_t b = 0; b < nbox; ++b) {
        t->seg_prm[b] = boxes[b].params;
        t->h_seg_off[b] = off;
        off += (uint32_t)boxes[b].n;
    }
    t->h_seg_off[nbox] = off;
    // inputs, concatenated: positions, masses, previous accelerations
    const bool have_aold = p0.opening == OG_OPEN_REL && boxes[0].a_old != nullptr;
    size_t in_bytes = (size_t)total * 4 * sizeof(double) + (have_aold ? (size_t)total * 3 * sizeof(float) : 0) + 512;
    void *in = nullptr;
    cudaError_t e;
    if ((e = dev_malloc_async(&in, in_bytes, s)) != cudaSuccess) { delete t; return cuda_fail(e, "cudaMallocAsync (batch inputs)"); }
    double *d_pos = static_cast<double *>(in);
    double *d_mass = d_pos + 3 * total;
    float *d_aold = have_aold ? reinterpret_cast<float *>(d_mass + total) : nullptr;
    for (int64_t b = 0; b < nbox; ++b) {
        const int64_t o = t->h_seg_off[b], nb = boxes[b].n;
        cudaMemcpyAsync(d_pos + 3 * o, boxes[b].pos, (size_t)nb * 3 * sizeof(double), in_kind, s);
        cudaMemcpyAsync(d_mass + o, boxes[b].mass, (size_t)nb * sizeof(double), in_kind, s);
        if (have_aold) cudaMemcpyAsync(d_aold + 3 * o, boxes[b].a_old, (size_t)nb * 3 * sizeof(float), in_kind, s);
    }
    og_status st = build_tree(t, d_pos, d_mass);
    if (st == OG_OK) st = check_status(c);
    float ms_walk = 0;
    if (st == OG_OK) st = force_sorted(t, d_aold, &ms_walk);
    cudaFreeAsync(in, s);
    if (st != OG_OK) {
        og_tree_free(t);
        return st;
    }
    // results back to every box in its own order
    void *out = nullptr;
    size_t out_bytes = (size_t)total * (3 * sizeof(float) + 2 * sizeof(uint32_t)) + 512;
    if ((e = dev_malloc_async(&out, out_bytes, s)) != cudaSuccess) { og_tree_free(t); return cuda_fail(e, "cudaMallocAsync (batch outputs)"); }
    float *o_acc = static_cast<float *>(out);
    uint32_t *o_pp = reinterpret_cast<uint32_t *>(o_acc + 3 * total);
    uint32_t *o_pn = o_pp + total;
    k_unpermute<<<nblk(total), kT, 0, s>>>(total, t->inv, t->a_sorted, t->npp_sorted, t->npn_sorted,
                                           o_acc, o_pp, o_pn); note_launch();
    for (int64_t b = 0; b < nbox; ++b) {
        const int64_t o = t->h_seg_off[b], nb = boxes[b].n;
        cudaMemcpyAsync(boxes[b].acc, o_acc + 3 * o, (size_t)nb * 3 * sizeof(float), out_kind, s);
        if (boxes[b].n_pp) cudaMemcpyAsync(boxes[b].n_pp, o_pp + o, (size_t)nb * sizeof(uint32_t), out_kind, s);
        if (boxes[b].n_pn) cudaMemcpyAsync(boxes[b].n_pn, o_pn + o, (size_t)nb * sizeof(uint32_t), out_kind, s);
    }
    cudaFreeAsync(out, s);
    cudaEventRecord(e1, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { og_tree_free(t); return cuda_fail(e, "batch"); }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (info) {
        info->boxes = nbox;
        info->particles = total;
        info->groups = t->ngroups;
        info->interactions = t->interactions;
        info->ms_total = ms;
        info->ms_build = t->ms_build;
        info->ms_walk = ms_walk;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st = check_status(c);
    og_tree_free(t);
    return st;
}

og_status og_tree_info_get(const og_tree *t, og_tree_info *info) {
    if (!t || !info) { set_error("NULL argument"); return OG_ERR_ARG; }
    info->n = t->n;
    info->nodes = t->nnodes;
    info->children = t->nchild;
    info->groups = t->ngroups;
    info->list_entries = t->list_len;
    info->interactions = t->interactions;
    info->interactions_last_pass = t->interactions_last;
    info->ms_build = t->ms_build;
    info->ms_force = t->ms_force;
    info->ms_walk = t->ms_walk;
    info->group_max = t->prm.group_max;
    info->walk_warps = t->prm.walk_warps;
    info->walk_chunk = t->prm.walk_chunk;
    info->pad = 0;
    info->ms_pm = t->ms_pm;
    info->ms_sph = t->ms_sph;
    return OG_OK;
}

og_status og_tree_export(const og_tree *t, int field, void *dst, size_t bytes) {
    if (!t || !dst) { set_error("NULL argument"); return OG_ERR_ARG; }
    const int64_t n = t->n, m = t->nnodes, g = t->ngroups, c = t->nchild;
    const void *src = nullptr;
    size_t need = 0;
    switch (field) {
    case OG_F_SKEY: src = t->skey; need = n * 8; break;
    case OG_F_PERM: src = t->perm; need = n * 4; break;
    case OG_F_SPOS: need = 3 * n * 4; break;
    case OG_F_LEVEL: src = t->nlev; need = m; break;
    case OG_F_NBEG: src = t->nbeg; need = m * 4; break;
    case OG_F_NEND: src = t->nend; need = m * 4; break;
    case OG_F_PARENT: src = t->npar; need = m * 4; break;
    case OG_F_CBEG: src = t->ncbeg; need = m * 4; break;
    case OG_F_CCNT: src = t->nccnt; need = m * 4; break;
    case OG_F_CHILD: src = t->child; need = c * 4; break;
    case OG_F_MASS: src = t->nmom; need = m * 8; break;
    case OG_F_COM: src = t->ncom; need = 3 * m * 4; break;
    case OG_F_NEXTNODE: src = t->nnext; need = m * 4; break;
    case OG_F_SIBLING: src = t->nsib; need = m * 4; break;
    case OG_F_PNEXT: src = t->pnext; need = n * 4; break;
    case OG_F_GBEG: src = t->gbeg; need = g * 4; break;
    case OG_F_GEND: src = t->gend; need = g * 4; break;
    case OG_F_GBOX: src = t->gbox; need = 6 * g * 4; break;
    case OG_F_LISTS: src = t->lists; need = t->list_len * 8; break;
    case OG_F_EXTENT:
        if (!t->refit) { set_error("no extents before a refit"); return OG_ERR_STATE; }
        need = 6 * m * 4;
        break;
    case OG_F_MSUM: need = 3 * m * 8; break;
    default: set_error("unknown field %d", field); return OG_ERR_ARG;
    }
    if (bytes != need) { set_error("field %d needs %zu bytes, got %zu", field, need, bytes); return OG_ERR_ARG; }
    if (need == 0) return OG_OK;
    cudaSetDevice(t->ctx->device);
    cudaStream_t s = t->ctx->stream;
    if (field == OG_F_EXTENT) {
        char *d = static_cast<char *>(dst);
        cudaMemcpyAsync(d, t->next_s, 3 * m * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(d + 3 * m * 4, t->next_l, 3 * m * 4, cudaMemcpyDeviceToHost, s);
    } else if (field == OG_F_MASS) {
        // the masses out of the nodes' 32-byte moment records
        cudaMemcpy2DAsync(dst, sizeof(double), &t->nmom[0].M, sizeof(NodeMom), sizeof(double), m,
                          cudaMemcpyDeviceToHost, s);
    } else if (field == OG_F_MSUM) {
        // the three sums out of the nodes' 32-byte moment records
        cudaMemcpy2DAsync(dst, 3 * sizeof(double), &t->nmom[0].Sx, sizeof(NodeMom), 3 * sizeof(double),
                          m, cudaMemcpyDeviceToHost, s);
    } else if (field == OG_F_SPOS) {
        char *d = static_cast<char *>(dst);
        cudaMemcpyAsync(d, t->px, n * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(d + n * 4, t->py, n * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(d + 2 * n * 4, t->pz, n * 4, cudaMemcpyDeviceToHost, s);
    } else {
        cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "export");
    return OG_OK;
}

og_status og_tree_free(og_tree *t) {
    if (!t) return OG_OK;
    live_remove(t);
    cudaSetDevice(t->ctx->device);
    if (t->arena) cudaFreeAsync(t->arena, t->ctx->stream);
    if (t->ext_arena) cudaFreeAsync(t->ext_arena, t->ctx->stream);
    if (t->lists) {
        cudaStreamSynchronize(t->ctx->stream);
        cudaFree(t->lists);
    }
    delete t;
    return OG_OK;
}

og_status og_tree_refit(og_tree *t, const double *pos) {
    if (!t || !pos) { set_error("NULL argument"); return OG_ERR_ARG; }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int64_t n = t->n;
    const double *d_pos = pos;
    void *tmp = nullptr;
    cudaError_t e;
    if (!(t->prm.flags & OG_DEVICE_PTRS)) {
        if ((e = dev_malloc_async(&tmp, (size_t)n * 3 * sizeof(double), s)) != cudaSuccess)
            return cuda_fail(e, "cudaMallocAsync (refit)");
        cudaMemcpyAsync(tmp, pos, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, s);
        d_pos = static_cast<const double *>(tmp);
    }
    og_status st = refit_tree(t, d_pos);
    if (tmp) cudaFreeAsync(tmp, s);
    if (st == OG_OK) st = check_status(c);
    return st;
}

}  // extern "C"
