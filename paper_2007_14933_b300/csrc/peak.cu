// peak.cu -- FP64 FMA throughput measurement (the roofline denominator of the FP64 path: the
// measured peaks cover HBM and bf16 only).  Independent FMA chains per thread.
#include <cuda_runtime.h>

#include "osbli.h"

namespace {
__global__ void k_dfma_chains(double *out, int iters, double a, double b)
{
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; i++) acc[i] = (double)(threadIdx.x + i);
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < 8; i++) acc[i] = fma(acc[i], a, b);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" int osbli_fp64_peak(double *tflops)
{
    if (!tflops) return OSBLI_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OSBLI_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return OSBLI_ECUDA;
    const int blocks = sms * 4, threads = 256, iters = 20000;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return OSBLI_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_dfma_chains<<<blocks, threads>>>(out, 100, 0.999, 0.001);
    cudaEventRecord(e0);
    k_dfma_chains<<<blocks, threads>>>(out, iters, 0.999, 0.001);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return OSBLI_ECUDA;
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    return OSBLI_OK;
}
