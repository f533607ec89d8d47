// peak.cu -- FP64 / FP32 FMA throughput measurement (roofline denominators of the FP64 and
// mixed paths: the measured peaks cover HBM and bf16 only).  Independent FMA chains.
#include <cuda_runtime.h>

#include "osbli.h"

namespace {
template <typename T>
__global__ void k_dfma_chains(T *out, int iters, T a, T b)
{
    T acc[8];
#pragma unroll
    for (int i = 0; i < 8; i++) acc[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < 8; i++) acc[i] = fma(acc[i], a, b);
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

template <typename T>
static int fma_peak(double *tflops, int blocks_per_sm)
{
    if (!tflops) return OSBLI_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OSBLI_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return OSBLI_ECUDA;
    const int blocks = sms * blocks_per_sm, threads = 256, iters = 20000;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return OSBLI_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_dfma_chains<T><<<blocks, threads>>>(out, 100, (T)0.999, (T)0.001);
    cudaEventRecord(e0);
    k_dfma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
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

extern "C" int osbli_fp64_peak(double *tflops) { return fma_peak<double>(tflops, 4); }
extern "C" int osbli_fp32_peak(double *tflops) { return fma_peak<float>(tflops, 8); }
