// pat_peaks.cu -- arithmetic peaks of the GPU, measured by dependent-chain
// kernels: FP32 fused multiply-add (scalar and packed pairs), FP64 fused
// multiply-add and the special-function unit (rsqrt).  Each thread runs
// kChains independent chains, enough to cover the pipe latency, on a grid of
// 8 CTAs of 256 threads per SM.  These are the denominators of the roofline of
// ALU-bound kernels (no vendor figure exists for them on this part).
#include <cuda_runtime.h>

#include "pat.h"

namespace {

constexpr int kChains = 8;
constexpr int kInner = 32;
constexpr int kThreadsPeak = 256;

__global__ void peak_ffma_kernel(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * threadIdx.x + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kInner; ++j)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.f) out[blockIdx.x] = s; // never true for a, b > 0; keeps the chains live
}

__global__ void peak_ffma2_kernel(float *out, int iters, float a, float b)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(1e-3f * threadIdx.x + c, 2e-3f * threadIdx.x + c);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kInner; ++j)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1.f) out[blockIdx.x] = s;
}

__global__ void peak_dfma_kernel(double *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * threadIdx.x + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kInner; ++j)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) out[blockIdx.x] = s;
}

__global__ void peak_rsqrt_kernel(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.f + 1e-3f * threadIdx.x + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kInner; ++j)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = rsqrtf(x[c]); // stays in [~0.5, ~2]
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.f) out[blockIdx.x] = s;
}

template <class Launch>
pat_status timed(Launch launch, cudaStream_t st, double ops, double *rate)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PAT_ERR_CUDA;
    launch(); // warm-up (clocks, instruction cache)
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    pat_status rc = PAT_OK;
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
        rc = PAT_ERR_CUDA;
    else
        *rate = ops / (1e-3 * ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

} // namespace

extern "C" pat_status pat_measure_peaks(pat_peaks *out, void *stream)
{
    if (!out) return PAT_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PAT_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = 8 * nsm;
    void *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks) != cudaSuccess) return PAT_ERR_CUDA;
    const double threads = (double)blocks * kThreadsPeak, per = (double)kChains * kInner;
    const int it32 = 4000, it64 = 60, itsfu = 400;
    pat_status rc = timed([&] { peak_ffma_kernel<<<blocks, kThreadsPeak, 0, st>>>((float *)buf, it32, 0.999f, 1e-3f); },
                          st, 2.0 * threads * per * it32, &out->fp32_ffma_flops);
    if (rc == PAT_OK)
        rc = timed([&] { peak_ffma2_kernel<<<blocks, kThreadsPeak, 0, st>>>((float *)buf, it32 / 2, 0.999f, 1e-3f); },
                   st, 4.0 * threads * per * (it32 / 2), &out->fp32_ffma2_flops);
    if (rc == PAT_OK)
        rc = timed([&] { peak_dfma_kernel<<<blocks, kThreadsPeak, 0, st>>>((double *)buf, it64, 0.999, 1e-3); },
                   st, 2.0 * threads * per * it64, &out->fp64_dfma_flops);
    if (rc == PAT_OK)
        rc = timed([&] { peak_rsqrt_kernel<<<blocks, kThreadsPeak, 0, st>>>((float *)buf, itsfu); }, st,
                   threads * per * itsfu, &out->sfu_rsqrt_ops);
    cudaFree(buf);
    return rc;
}
