// og_peak.cu -- measured FP32 throughput of this GPU, the denominator the walk
// (an FP32-ALU-bound kernel, not a contraction) is compared against.
//
// Every thread runs kChains independent fused multiply-add chains a = a * b + c
// (b, c runtime values, so nothing folds), enough chains per warp to cover the
// FMA latency; the grid fills every SM to full occupancy.  One FMA is 2 flops;
// one f32x2 FMA is 4.  A thread stores its sum only if it equals a value the
// chains cannot reach, which keeps the work live without memory traffic.
#include "og_internal.h"

namespace og {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float b, float c, int iters, float *out) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.2345e30f) out[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_fma2_peak(float b, float c, int iters, float *out) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    if (s == -1.2345e30f) out[0] = s;
}

}  // namespace
}  // namespace og

using namespace og;

extern "C" og_status og_measure_fp32_peak(og_ctx *c, double *tflops_fma, double *tflops_fma2) {
    if (!c || !tflops_fma || !tflops_fma2) { set_error("og_measure_fp32_peak: NULL argument"); return OG_ERR_ARG; }
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0);
    if (sms < 1 || per_sm < 1) { set_error("og_measure_fp32_peak: no occupancy"); return OG_ERR_CUDA; }
    const unsigned grid = (unsigned)(sms * per_sm);
    const int iters = 4096;
    float *out = nullptr;
    cudaError_t e = dev_malloc_async(&out, sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (peak)");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double threads = (double)grid * kPeakThreads;
    const double fmas = threads * kChains * 16.0 * iters;
    double best[2] = {0.0, 0.0};
    for (int rep = 0; rep < 4; ++rep) {      // the first round warms up
        for (int v = 0; v < 2; ++v) {
            cudaEventRecord(e0, s);
            if (v == 0) k_fma_peak<<<grid, kPeakThreads, 0, s>>>(1.0000001f, 1e-7f, iters, out);
            else k_fma2_peak<<<grid, kPeakThreads, 0, s>>>(1.0000001f, 1e-7f, iters, out);
            note_launch();
            cudaEventRecord(e1, s);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double tf = fmas * (v == 0 ? 2.0 : 4.0) / (ms * 1e-3) / 1e12;
            if (rep > 0 && tf > best[v]) best[v] = tf;
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "peak");
    *tflops_fma = best[0];
    *tflops_fma2 = best[1];
    return OG_OK;
}
