/* Throughput probes of the arithmetic pipes the stage kernels are bound by:
 * the measured denominators of their rooflines.  Each thread runs eight
 * independent dependency chains (enough to cover the pipe latency at full
 * occupancy) of one operation; the grid fills every SM. */
#include <cuda_runtime.h>

#include "../../include/genogks.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_probe(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) dfma_probe(double *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

/* the same FMA work as ffma_probe, issued as packed two-lane FMAs
 * (fma.rn.f32x2): one instruction per pair of chains */
__global__ void __launch_bounds__(256) ffma2_probe(float *out, int iters, float a, float b)
{
    float2 x[kChains / 2];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k)
        x[k] = make_float2(1e-3f * (float)(threadIdx.x + 2 * k), 1e-3f * (float)(threadIdx.x + 2 * k + 1));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

/* the special-function unit: x <- 2^-x (ex2.approx, the instruction behind
 * the FP32 exponentials), bounded in (0, 1] */
__global__ void __launch_bounds__(256) mufu_probe(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[k]));
                x[k] = y;
            }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

} // namespace

extern "C" int gks_pipe_probe(int kind, int iters, double *ops_per_s, void *stream)
{
    if (!ops_per_s || iters < 1 || kind < 0 || kind > 3) return GKS_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GKS_ERR_CUDA;
    const int threads = 256, blocks = nsm * 8; /* 2048 threads per SM */
    const long n = (long)threads * blocks;
    cudaStream_t s = (cudaStream_t)stream;
    void *buf = nullptr;
    if (cudaMallocAsync(&buf, sizeof(double) * n, s) != cudaSuccess) return GKS_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int it) {
        if (kind == 0) ffma_probe<<<blocks, threads, 0, s>>>((float *)buf, it, 0.9999f, 1e-4f);
        else if (kind == 1) dfma_probe<<<blocks, threads, 0, s>>>((double *)buf, it, 0.9999, 1e-4);
        else if (kind == 2) mufu_probe<<<blocks, threads, 0, s>>>((float *)buf, it);
        else ffma2_probe<<<blocks, threads, 0, s>>>((float *)buf, it, 0.9999f, 1e-4f);
    };
    launch(iters); /* warm-up */
    cudaEventRecord(e0, s);
    launch(iters);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    if (e != cudaSuccess || !(ms > 0.f)) return GKS_ERR_CUDA;
    /* operations: FMA = 2 flops; one ex2 = 1 op */
    const double per_chain_step = (kind == 2) ? 1.0 : 2.0;
    *ops_per_s = per_chain_step * kChains * 4.0 * (double)iters * (double)n / (ms * 1e-3);
    return GKS_OK;
}
