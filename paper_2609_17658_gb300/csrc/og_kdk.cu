// og_kdk.cu -- kick-drift-kick leapfrog with individual power-of-two time
// steps (Sect. 3.2).
//
// One maximum step dt_max is 2^B ticks (B = max_bin).  A particle in bin b
// steps by dt_b = dt_max / 2^b and is active at the ticks that are multiples of
// 2^(B - b).  Its bin is the smallest b with dt_max / 2^b <= sqrt(2 eta eps / |a|)
// (the acceleration criterion of Sect. 3.2, eta the integration tolerance),
// at most B, and only a bin whose period divides the current tick may be
// entered.  Per tick: every particle drifts (k > 0), the tree follows the
// positions (rebuilt every rebuild_every ticks, refitted in between), the
// active particles get new accelerations from the walk over their groups
// only, then their closing half kick with the old bin (k > 0) and, unless it
// is the last tick, a new bin and the opening half kick.  FP64 kinematics,
// products and sums rounded separately.
#include <cstring>
#include <new>
#include <vector>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

__global__ void k_kdk_drift(int64_t n, const double *__restrict__ vel, double *pos, double dt,
                            double box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 3; ++a) {
        double x = __dadd_rn(pos[3 * i + a], __dmul_rn(vel[3 * i + a], dt));
        if (x >= box) x = __dsub_rn(x, box);
        if (x < 0.0) x = __dadd_rn(x, box);
        pos[3 * i + a] = x;
    }
}

// active at tick k: every particle at k = 0, else k a multiple of 2^(B - b)
__global__ void k_kdk_active(int64_t n, const int32_t *__restrict__ bins, uint64_t k, int max_bin,
                             uint8_t *active, unsigned long long *count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t on = 0;
    if (i < n) {
        const uint64_t period = 1ull << (max_bin - bins[i]);
        on = (k == 0 || (k & (period - 1)) == 0) ? 1u : 0u;
        active[i] = (uint8_t)on;
    }
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, (unsigned long long)__popc(m));
}

__device__ __forceinline__ double half_step(double dt_max, int b) {
    return __ddiv_rn(dt_max, (double)(1ull << b)) * 0.5;   // exact scalings by powers of two
}

__global__ void k_kdk_close(int64_t n, const uint8_t *__restrict__ active,
                            const float *__restrict__ acc, const int32_t *__restrict__ bins,
                            double dt_max, double *vel) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !active[i]) return;
    const double h = half_step(dt_max, bins[i]);
    for (int a = 0; a < 3; ++a)
        vel[3 * i + a] = __dadd_rn(vel[3 * i + a], __dmul_rn((double)acc[3 * i + a], h));
}

__global__ void k_kdk_open(int64_t n, const uint8_t *__restrict__ active,
                           const float *__restrict__ acc, double eps, double eta, double dt_max,
                           int max_bin, int min_bin, int32_t *bins, double *vel) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !active[i]) return;
    const double ax = acc[3 * i], ay = acc[3 * i + 1], az = acc[3 * i + 2];
    const double a = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)),
                                          __dmul_rn(az, az)));
    int b = 0;
    if (a > 0.0) {
        const double dt_crit = __dsqrt_rn(__ddiv_rn(__dmul_rn(__dmul_rn(2.0, eta), eps), a));
        while (b < max_bin && __ddiv_rn(dt_max, (double)(1ull << b)) > dt_crit) ++b;
    }
    if (b < min_bin) b = min_bin;
    bins[i] = b;
    const double h = half_step(dt_max, b);
    for (int q = 0; q < 3; ++q)
        vel[3 * i + q] = __dadd_rn(vel[3 * i + q], __dmul_rn((double)acc[3 * i + q], h));
}

int trailing_zeros(uint64_t k) { return k ? __builtin_ctzll(k) : 64; }

}  // namespace
}  // namespace og

using namespace og;

extern "C" og_status og_kdk_run(og_ctx *c, int64_t n, double *pos, double *vel, const double *mass,
                                const og_params *p, const og_kdk_params *kp, float *acc_out,
                                int32_t *bins_out, og_kdk_stats *stats) {
    if (!c || !pos || !vel || !mass || !p || !kp) { set_error("og_kdk_run: NULL argument"); return OG_ERR_ARG; }
    og_status st = validate(p, n);
    if (st) return st;
    if (!(kp->dt_max > 0.0) || !(kp->eta > 0.0) || kp->max_bin < 0 || kp->max_bin > 30 ||
        kp->nsteps < 1 || kp->rebuild_every < 1 || !(p->eps > 0.0)) {
        set_error("og_kdk_run: need dt_max > 0, eta > 0, 0 <= max_bin <= 30, nsteps >= 1, "
                  "rebuild_every >= 1, eps > 0");
        return OG_ERR_ARG;
    }
    const uint64_t ticks = (uint64_t)kp->nsteps << kp->max_bin;
    if (ticks > (1ull << 40)) { set_error("og_kdk_run: too many ticks"); return OG_ERR_ARG; }
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const bool dev = (p->flags & OG_DEVICE_PTRS) != 0;
    cudaError_t e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    // device state: positions, velocities, masses (f64), accelerations (f32),
    // bins, active mask, a counter
    const size_t b_v = (size_t)n * 3 * sizeof(double);
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // every piece below is taken rounded up to 256 bytes: the total is the sum
    // of the rounded sizes
    const size_t bytes = 2 * up(b_v) + up((size_t)n * sizeof(double)) +
                         up((size_t)n * 3 * sizeof(float)) + up((size_t)n * sizeof(int32_t)) +
                         up((size_t)n) + up(64);
    void *mem = nullptr;
    if ((e = dev_malloc_async(&mem, bytes, s)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (kdk)");
    char *q = static_cast<char *>(mem);
    auto take = [&](size_t b) { char *r = q; q += up(b); return r; };
    double *d_pos = reinterpret_cast<double *>(take(b_v));
    double *d_vel = reinterpret_cast<double *>(take(b_v));
    double *d_mass = reinterpret_cast<double *>(take((size_t)n * sizeof(double)));
    float *d_acc = reinterpret_cast<float *>(take((size_t)n * 3 * sizeof(float)));
    int32_t *d_bins = reinterpret_cast<int32_t *>(take((size_t)n * sizeof(int32_t)));
    uint8_t *d_active = reinterpret_cast<uint8_t *>(take((size_t)n));
    unsigned long long *d_count = reinterpret_cast<unsigned long long *>(take(64));
    const cudaMemcpyKind in_kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind out_kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaMemcpyAsync(d_pos, pos, b_v, in_kind, s);
    cudaMemcpyAsync(d_vel, vel, b_v, in_kind, s);
    cudaMemcpyAsync(d_mass, mass, (size_t)n * sizeof(double), in_kind, s);
    cudaMemsetAsync(d_acc, 0, (size_t)n * 3 * sizeof(float), s);
    cudaMemsetAsync(d_bins, 0, (size_t)n * sizeof(int32_t), s);
    og_params tp = *p;
    tp.flags = (p->flags | OG_DEVICE_PTRS) & ~OG_DEBUG_DUMP_LISTS;
    og_kdk_stats sx{};
    og_tree *tree = nullptr;
    const double dt_tick = kp->dt_max / (double)(1ull << kp->max_bin);
    for (uint64_t k = 0; k <= ticks && st == OG_OK; ++k) {
        if (k > 0) {
            k_kdk_drift<<<nblk(n), kT, 0, s>>>(n, d_vel, d_pos, dt_tick, p->box); note_launch();
        }
        // the tree at the current positions
        if (!tree || k % (uint64_t)kp->rebuild_every == 0) {
            if (tree) og_tree_free(tree);
            tree = nullptr;
            st = og_tree_build(c, d_pos, d_mass, n, &tp, &tree);
            sx.rebuilds++;
        } else {
            st = refit_tree(tree, d_pos);
            if (st == OG_OK) st = check_status(c);
            sx.refits++;
        }
        if (st) break;
        cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s);
        k_kdk_active<<<nblk(n), kT, 0, s>>>(n, d_bins, k, kp->max_bin, d_active, d_count); note_launch();
        int64_t walked = 0;
        // relative criterion: the previous accelerations (a Barnes-Hut first
        // pass at tick 0, when there are none yet)
        st = og_tree_force_active(tree, d_active, k == 0 ? nullptr : d_acc, d_acc, nullptr, nullptr,
                                  &walked);
        if (st) break;
        unsigned long long nact = 0;
        cudaMemcpyAsync(&nact, d_count, sizeof(nact), cudaMemcpyDeviceToHost, s);
        sx.forces += (int64_t)nact;
        sx.groups_walked += walked;
        sx.interactions += tree->interactions;
        if (k > 0) {
            k_kdk_close<<<nblk(n), kT, 0, s>>>(n, d_active, d_acc, d_bins, kp->dt_max, d_vel); note_launch();
        }
        if (k < ticks) {
            const int tz = trailing_zeros(k);
            const int min_bin = tz >= kp->max_bin ? 0 : kp->max_bin - tz;
            k_kdk_open<<<nblk(n), kT, 0, s>>>(n, d_active, d_acc, p->eps, kp->eta, kp->dt_max,
                                              kp->max_bin, min_bin, d_bins, d_vel); note_launch();
        }
        sx.ticks = (int64_t)k;
    }
    if (tree) og_tree_free(tree);
    if (st == OG_OK) {
        cudaMemcpyAsync(pos, d_pos, b_v, out_kind, s);
        cudaMemcpyAsync(vel, d_vel, b_v, out_kind, s);
        if (acc_out) cudaMemcpyAsync(acc_out, d_acc, (size_t)n * 3 * sizeof(float), out_kind, s);
        if (bins_out) cudaMemcpyAsync(bins_out, d_bins, (size_t)n * sizeof(int32_t), out_kind, s);
    }
    cudaFreeAsync(mem, s);
    cudaEventRecord(e1, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess && st == OG_OK) st = cuda_fail(e, "kdk");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (stats) {
        sx.ms = ms;
        *stats = sx;
    }
    return st;
}
