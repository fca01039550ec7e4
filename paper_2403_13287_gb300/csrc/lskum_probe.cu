// lskum_probe_peak: measured arithmetic peaks of the GPU the library runs
// on, the denominators of the ALU rooflines of the flux kernels. Not part of
// the method (the paper has no counterpart): a throughput report needs the
// FP64 and FP32 fused multiply-add rates of this part, which are not in the
// HBM/tensor peak record.
//
// Each thread runs 8 independent multiply-add chains a <- a*b + c (b just
// below 1, so the chains stay near c/(1-b) and never go subnormal or
// overflow); the grid fills every SM several times. The result is written
// only if it is NaN, which never happens, so the chains cannot be removed
// (the sink is a real device buffer all the same).
#include <cuda_runtime.h>

#include "lskum.h"
#include "lskum_kernels.h"

namespace lskum {

static constexpr int kChains = 8;
static constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(int iters, T b, T c, T *sink)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s != s) sink[threadIdx.x] = s;
}

// packed FP32 pairs: one FFMA2 instruction does two multiply-adds
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma2(int iters, float b, float c, float *sink)
{
    float2 a[kChains];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    if (s != s) sink[threadIdx.x] = s;
}

}  // namespace lskum

using namespace lskum;

extern "C" lskum_status lskum_probe_peak(int kind, int reps, void *cuda_stream, double *gflops)
{
    if (!gflops || kind < 0 || kind > 2 || reps < 1 || reps > 100)
        return LSKUM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return LSKUM_ERR_CUDA;
    // FP64 is the slow pipe on this part: fewer iterations keep the probe short
    const int iters = kind == 0 ? 2048 : 16384;
    const unsigned blocks = (unsigned)sms * 8u;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LSKUM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LSKUM_ERR_CUDA;
    }
    double *sink = nullptr;
    if (cudaMalloc(&sink, 2 * kProbeThreads * sizeof(double)) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return LSKUM_ERR_OOM;
    }
    float *sinkf = reinterpret_cast<float *>(sink);
    lskum_status st = LSKUM_OK;
    float best = 0.0f;
    for (int r = 0; r <= reps && st == LSKUM_OK; ++r) {   // r = 0: warm-up
        cudaEventRecord(e0, s);
        if (kind == 0) k_probe_fma<double><<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999999, 1e-7, sink);
        else if (kind == 1) k_probe_fma<float><<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sinkf);
        else k_probe_fma2<<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sinkf);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = LSKUM_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaFree(sink);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LSKUM_OK) return st;
    const double fma_per_thread = (double)iters * kChains * (kind == 2 ? 2.0 : 1.0);
    const double flops = 2.0 * fma_per_thread * blocks * kProbeThreads;
    *gflops = flops / (best * 1e-3) / 1e9;
    return LSKUM_OK;
}
