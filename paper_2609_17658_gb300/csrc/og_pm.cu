// og_pm.cu -- long-range particle-mesh (PM) force of a built tree (Sect. 4.2
// "Particle Mesh").
//
// The tree walk evaluates the erfc part of the split potential; the mesh gives
// the erf part.  One call, on the tree's sorted u32 positions and FP32 masses:
//
//   k_pm_deposit   cloud-in-cell assignment: every particle adds m * w to the 8
//                  mesh points around it, as 64-bit fixed-point integers
//                  (atomicAdd of integers is exact, so the density does not
//                  depend on the order of the additions: one value per input);
//                  a warp first sums the contributions of its runs of
//                  particles that share a cell
//   k_pm_density   fixed point -> FP32 density (the FFT's input)
//   cuFFT R2C      forward transform (library call, FP32)
//   k_pm_green     multiply every mode by the filtered Green's function
//                  -4 pi G / k^2 * exp(-k^2 r_s^2), divided by the squared CIC
//                  window prod_a sinc^4(k_a D / 2) (one window for the
//                  assignment, one for the interpolation); k = 0 is zero.  The
//                  per-axis factors come from a table of Ng entries, since
//                  exp(-k^2 r_s^2) and the window are products over the axes
//   cuFFT C2R      inverse transform: the potential on the mesh
//   k_pm_interp    per particle, a = -grad phi by the fourth-order central
//                  difference [8 (phi(i+1) - phi(i-1)) - (phi(i+2) - phi(i-2))] / 12 D
//                  at the 8 CIC mesh points, interpolated with the CIC weights
//                  and written in the caller's order
//
// Mesh point (i, j, l) sits at (i, j, l) D, D = L / Ng, Ng a power of two, so a
// particle's mesh coordinate is its u32 coordinate shifted right by
// 32 - log2 Ng bits: integer mesh index and fraction without rounding.
//
// cuFFT is loaded with dlopen the first time a context needs it: the library
// itself has no link dependency on it, and a missing cuFFT is an error of this
// call (OG_ERR_CUDA), not of the library.
#include <cufft.h>
#include <dlfcn.h>

#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }
constexpr int kFixBits = 52;  // the total mass maps to at most 2^52 fixed-point units

// ---- cuFFT entry points (dlopen) ------------------------------------------
struct CufftApi {
    bool tried = false, ok = false;
    cufftResult (*plan3d)(cufftHandle *, int, int, int, cufftType) = nullptr;
    cufftResult (*exec_r2c)(cufftHandle, cufftReal *, cufftComplex *) = nullptr;
    cufftResult (*exec_c2r)(cufftHandle, cufftComplex *, cufftReal *) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
};

std::mutex g_api_mu;
CufftApi g_api;

const CufftApi *cufft_api() {
    std::lock_guard<std::mutex> lk(g_api_mu);
    if (g_api.tried) return g_api.ok ? &g_api : nullptr;
    g_api.tried = true;
    void *h = nullptr;
    for (const char *name : {"libcufft.so.12", "libcufft.so.13", "libcufft.so"}) {
        h = dlopen(name, RTLD_NOW | RTLD_GLOBAL);
        if (h) break;
    }
    if (!h) return nullptr;
    g_api.plan3d = reinterpret_cast<decltype(g_api.plan3d)>(dlsym(h, "cufftPlan3d"));
    g_api.exec_r2c = reinterpret_cast<decltype(g_api.exec_r2c)>(dlsym(h, "cufftExecR2C"));
    g_api.exec_c2r = reinterpret_cast<decltype(g_api.exec_c2r)>(dlsym(h, "cufftExecC2R"));
    g_api.set_stream = reinterpret_cast<decltype(g_api.set_stream)>(dlsym(h, "cufftSetStream"));
    g_api.destroy = reinterpret_cast<decltype(g_api.destroy)>(dlsym(h, "cufftDestroy"));
    g_api.ok = g_api.plan3d && g_api.exec_r2c && g_api.exec_c2r && g_api.set_stream && g_api.destroy;
    return g_api.ok ? &g_api : nullptr;
}

// ---- per-context plans ------------------------------------------------------
struct Plans {
    cufftHandle r2c = 0, c2r = 0;
};

struct PmState {
    std::mutex mu;
    std::map<int, Plans> plans;  // by mesh size
};

PmState *pm_state(og_ctx *c) {
    if (!c->pm) c->pm = new (std::nothrow) PmState();
    return static_cast<PmState *>(c->pm);
}

og_status plans_for(og_ctx *c, int ng, Plans *out) {
    const CufftApi *api = cufft_api();
    if (!api) { set_error("og_tree_pm_force: cuFFT could not be loaded"); return OG_ERR_CUDA; }
    PmState *ps = pm_state(c);
    if (!ps) { set_error("host allocation failed"); return OG_ERR_OOM; }
    std::lock_guard<std::mutex> lk(ps->mu);
    auto it = ps->plans.find(ng);
    if (it != ps->plans.end()) {
        *out = it->second;
        return OG_OK;
    }
    Plans p;
    cufftResult r = api->plan3d(&p.r2c, ng, ng, ng, CUFFT_R2C);
    if (r != CUFFT_SUCCESS) { set_error("cufftPlan3d (R2C, %d^3) failed: %d", ng, (int)r); return OG_ERR_CUDA; }
    r = api->plan3d(&p.c2r, ng, ng, ng, CUFFT_C2R);
    if (r != CUFFT_SUCCESS) {
        api->destroy(p.r2c);
        set_error("cufftPlan3d (C2R, %d^3) failed: %d", ng, (int)r);
        return OG_ERR_CUDA;
    }
    ps->plans[ng] = p;
    *out = p;
    return OG_OK;
}

// ---- kernels ----------------------------------------------------------------
__device__ __forceinline__ float frac_of(uint32_t q, int s) {
    return (float)(q & ((1u << s) - 1u)) * __int_as_float((127 - s) << 23);  // exact scaling by 2^-s
}

// 2^(kFixBits - e) with M_total <= 2^e, as an FP32 factor (clamped to 2^127)
__device__ __forceinline__ float fix_scale(double mtot) {
    int e = 0;
    frexp(mtot, &e);  // mtot = f 2^e, f in [0.5, 1)
    int x = kFixBits - e;
    if (x > 127) x = 127;
    if (x < -126) x = -126;
    return __int_as_float((x + 127) << 23);
}

// Particles come in key order, so the particles of one mesh cell (same CIC
// base point, the key's top 3 log2 Ng bits) are contiguous.  Each warp sums the
// contributions of every such run with a segmented suffix sum (integers: the
// order does not change the result) and the run's first lane adds the 8 sums,
// so a dense cell costs 8 atomics per warp instead of 8 per particle.
__global__ void k_pm_deposit(int64_t n, int shift, int ng, const uint32_t *__restrict__ px,
                             const uint32_t *__restrict__ py, const uint32_t *__restrict__ pz,
                             const float *__restrict__ pm32, const NodeMom *__restrict__ root,
                             unsigned long long *__restrict__ mesh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) >= n) return;  // whole warps only
    const bool valid = i < n;
    const unsigned lane = threadIdx.x & 31u;
    const float sc = fix_scale(root->M);
    const uint32_t qx = valid ? px[i] : 0u, qy = valid ? py[i] : 0u, qz = valid ? pz[i] : 0u;
    const int m1 = ng - 1;
    const int ix = (int)(qx >> shift), iy = (int)(qy >> shift), iz = (int)(qz >> shift);
    const float fx = frac_of(qx, shift), fy = frac_of(qy, shift), fz = frac_of(qz, shift);
    const float m = valid ? pm32[i] * sc : 0.0f;
    // runs of equal base points within the warp (past-the-end lanes form their own run)
    const uint32_t cell = valid ? (uint32_t)(((ix * ng) + iy) * ng + iz) : 0xffffffffu;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, cell, 1);
    const bool head = lane == 0 || cell != prev;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned later = lane == 31 ? 0u : heads & (0xfffffffeu << lane);
    const unsigned end = later ? (unsigned)__ffs(later) - 2u : 31u;   // last lane of this run
    const float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const size_t bx = (size_t)((ix + a) & m1) * ng;
        const float ma = m * wx[a];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const size_t by = (bx + ((iy + b) & m1)) * ng;
            const float mab = ma * wy[b];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                unsigned long long v = __float2ull_rn(mab * wz[c]);
#pragma unroll
                for (unsigned d = 1; d < 32; d <<= 1) {
                    const unsigned long long u = __shfl_down_sync(0xffffffffu, v, d);
                    if (lane + d <= end) v += u;
                }
                if (head && valid && v) atomicAdd(&mesh[by + ((iz + c) & m1)], v);
            }
        }
    }
}

// density in units of the fixed point -> FP32 (the Green's factor carries the rest)
__global__ void k_pm_density(int64_t cells, const unsigned long long *__restrict__ fix,
                             float *__restrict__ rho) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cells) return;
    rho[i] = __ull2float_rn(fix[i]);
}

// tab[n] = (k_n^2, exp(-k_n^2 r_s^2) / sinc^4(k_n D / 2)) for the full-axis index n
__global__ void k_pm_green(int ng, int nzh, const float2 *__restrict__ tab, float cfac,
                           float2 *__restrict__ rk) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)ng * ng * nzh;
    if (idx >= total) return;
    const int iz = (int)(idx % nzh);
    const int64_t r = idx / nzh;
    const int iy = (int)(r % ng), ix = (int)(r / ng);
    const float2 tx = tab[ix], ty = tab[iy], tz = tab[iz];
    const float k2 = (tx.x + ty.x) + tz.x;
    float g = 0.0f;
    if (idx != 0) g = cfac * ((tx.y * ty.y) * tz.y) / k2;
    float2 v = rk[idx];
    v.x *= g;
    v.y *= g;
    rk[idx] = v;
}

__global__ void k_pm_interp(int64_t n, int shift, int ng, const uint32_t *__restrict__ px,
                            const uint32_t *__restrict__ py, const uint32_t *__restrict__ pz,
                            const uint32_t *__restrict__ perm, const float *__restrict__ phi,
                            const NodeMom *__restrict__ root, float out_scale,
                            float *__restrict__ acc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // the FFT input was the density in fixed-point units: undo that scale here
    const float s = out_scale / fix_scale(root->M);
    const uint32_t qx = px[i], qy = py[i], qz = pz[i];
    const int m1 = ng - 1;
    const int ix = (int)(qx >> shift), iy = (int)(qy >> shift), iz = (int)(qz >> shift);
    const float fx = frac_of(qx, shift), fy = frac_of(qy, shift), fz = frac_of(qz, shift);
    const float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
    auto at = [&](int x, int y, int z) -> float {
        return __ldg(&phi[((size_t)(x & m1) * ng + (size_t)(y & m1)) * ng + (size_t)(z & m1)]);
    };
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int x = ix + a, y = iy + b, z = iz + c;
                const float w = (wx[a] * wy[b]) * wz[c];
                const float gx = 8.0f * (at(x + 1, y, z) - at(x - 1, y, z)) - (at(x + 2, y, z) - at(x - 2, y, z));
                const float gy = 8.0f * (at(x, y + 1, z) - at(x, y - 1, z)) - (at(x, y + 2, z) - at(x, y - 2, z));
                const float gz = 8.0f * (at(x, y, z + 1) - at(x, y, z - 1)) - (at(x, y, z + 2) - at(x, y, z - 2));
                ax = fmaf(w, gx, ax);
                ay = fmaf(w, gy, ay);
                az = fmaf(w, gz, az);
            }
        }
    }
    const size_t o = 3 * (size_t)perm[i];
    acc[o + 0] = -ax * s;
    acc[o + 1] = -ay * s;
    acc[o + 2] = -az * s;
}

}  // namespace

void pm_free(og_ctx *c) {
    PmState *ps = static_cast<PmState *>(c->pm);
    if (!ps) return;
    const CufftApi *api = cufft_api();
    if (api)
        for (auto &kv : ps->plans) {
            api->destroy(kv.second.r2c);
            api->destroy(kv.second.c2r);
        }
    delete ps;
    c->pm = nullptr;
}

}  // namespace og

using namespace og;

extern "C" og_status og_tree_pm_force(og_tree *t, int32_t mesh, float *acc) {
    if (!t || !acc) { set_error("og_tree_pm_force: NULL argument"); return OG_ERR_ARG; }
    if (t->nseg != 1) { set_error("og_tree_pm_force: a tree of one box only"); return OG_ERR_ARG; }
    if (mesh < 2 || mesh > 1024 || (mesh & (mesh - 1))) {
        set_error("og_tree_pm_force: mesh must be a power of two in [2, 1024], got %d", mesh);
        return OG_ERR_ARG;
    }
    const og_params &p = t->prm;
    if (!(p.r_s > 0.0)) { set_error("og_tree_pm_force: the mesh force needs r_s > 0"); return OG_ERR_ARG; }
    og_ctx *c = t->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int ng = mesh;
    int lg = 0;
    while ((1 << lg) < ng) ++lg;
    const int shift = 32 - lg;
    const int nzh = ng / 2 + 1;
    const int64_t n = t->n;
    const int64_t cells = (int64_t)ng * ng * ng;
    const int64_t modes = (int64_t)ng * ng * nzh;
    Plans plans;
    og_status st = plans_for(c, ng, &plans);
    if (st) return st;
    const CufftApi *api = cufft_api();
    // per-axis table: k_n^2 and exp(-k_n^2 r_s^2) / sinc^4(k_n D / 2), FP64 on the host
    const double L = p.box, D = L / ng, rs = p.r_s;
    std::vector<float2> h_tab(ng);
    for (int i = 0; i < ng; ++i) {
        const int nsig = i < ng / 2 ? i : i - ng;
        const double k = 2.0 * M_PI * nsig / L;
        const double x = 0.5 * k * D;
        const double sinc = nsig == 0 ? 1.0 : std::sin(x) / x;
        const double s2 = sinc * sinc;
        h_tab[i] = make_float2((float)(k * k), (float)(std::exp(-k * k * rs * rs) / (s2 * s2)));
    }
    // buffers: fixed-point mesh (8 B/point), real mesh (4 B/point, density then
    // potential), modes (8 B/mode), the table
    const size_t b_fix = (size_t)cells * 8, b_real = (size_t)cells * 4, b_modes = (size_t)modes * 8;
    const size_t b_tab = (size_t)ng * sizeof(float2);
    const size_t off_real = (b_fix + 255) & ~(size_t)255, off_modes = off_real + ((b_real + 255) & ~(size_t)255);
    const size_t off_tab = off_modes + ((b_modes + 255) & ~(size_t)255);
    const size_t b_out = (p.flags & OG_DEVICE_PTRS) ? 0 : (size_t)n * 3 * sizeof(float);
    const size_t off_out = off_tab + ((b_tab + 255) & ~(size_t)255);
    const size_t total = off_out + b_out;
    if (c->hbm_budget && total > c->hbm_budget) {
        set_error("og_tree_pm_force: %zu bytes of mesh buffers exceed the context budget", total);
        return OG_ERR_BUDGET;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    char *buf = nullptr;
    cudaError_t e = dev_malloc_async(&buf, total, s);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "cudaMallocAsync (mesh)");
    }
    unsigned long long *fix = reinterpret_cast<unsigned long long *>(buf);
    float *real = reinterpret_cast<float *>(buf + off_real);
    float2 *rk = reinterpret_cast<float2 *>(buf + off_modes);
    float2 *tab = reinterpret_cast<float2 *>(buf + off_tab);
    float *d_acc = b_out ? reinterpret_cast<float *>(buf + off_out) : acc;
    cudaMemcpyAsync(tab, h_tab.data(), b_tab, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(fix, 0, b_fix, s);
    if (n > 0) {
        k_pm_deposit<<<nblk(n), kT, 0, s>>>(n, shift, ng, t->px, t->py, t->pz, t->pm32, t->nmom, fix);
        note_launch();
    }
    k_pm_density<<<nblk(cells), kT, 0, s>>>(cells, fix, real); note_launch();
    cufftResult r = api->set_stream(plans.r2c, s);
    if (r == CUFFT_SUCCESS) r = api->exec_r2c(plans.r2c, real, reinterpret_cast<cufftComplex *>(rk));
    if (r == CUFFT_SUCCESS) {
        // -4 pi G / k^2 of the density (mass / D^3), over Ng^3 for the unnormalised inverse FFT
        const double cfac = -4.0 * M_PI * p.G / (D * D * D) / (double)cells;
        k_pm_green<<<nblk(modes), kT, 0, s>>>(ng, nzh, tab, (float)cfac, rk); note_launch();
        r = api->set_stream(plans.c2r, s);
    }
    if (r == CUFFT_SUCCESS) r = api->exec_c2r(plans.c2r, reinterpret_cast<cufftComplex *>(rk), real);
    if (r != CUFFT_SUCCESS) {
        cudaFreeAsync(buf, s);
        cudaStreamSynchronize(s);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_error("og_tree_pm_force: cuFFT execution failed: %d", (int)r);
        return OG_ERR_CUDA;
    }
    if (n > 0) {
        k_pm_interp<<<nblk(n), kT, 0, s>>>(n, shift, ng, t->px, t->py, t->pz, t->perm, real, t->nmom,
                                           (float)(1.0 / (12.0 * D)), d_acc);
        note_launch();
    }
    if (b_out && n > 0) cudaMemcpyAsync(acc, d_acc, b_out, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(buf, s);
    cudaEventRecord(e1, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "pm force");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->ms_pm = ms;
    return check_status(c);
}
