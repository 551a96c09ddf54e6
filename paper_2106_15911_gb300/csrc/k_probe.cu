// k_probe.cu -- FMA throughput probe: the FP32 / FP64 pipe peaks that the nearfield and M2L
// rooflines are measured against (the measured-peaks file holds only HBM and BF16 figures).
#include <cuda_runtime.h>

#include "../../include/pfmm.h"

namespace {

template <typename R>
__global__ void k_fma_probe(R *out, int iters, R seed)
{
    R a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + R(threadIdx.x + i);
    const R b = R(0.999999), c = R(1e-7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = a[i] * b + c;
    }
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == R(-1.2345)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

template <typename R>
int probe(double *tflops, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256, iters = sizeof(R) == 8 ? 2048 : 32768;
    R *out = nullptr;
    if (cudaMalloc(&out, sizeof(R) * blocks * threads) != cudaSuccess) return PFMM_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_probe<R><<<blocks, threads, 0, st>>>(out, iters / 8, R(1));  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) k_fma_probe<R><<<blocks, threads, 0, st>>>(out, iters, R(1));
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.f) return PFMM_ERR_CUDA;
    double flops = 5.0 * blocks * threads * (double)iters * 8 * 2;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return PFMM_OK;
}

}  // namespace

extern "C" int pfmm_probe_fma_rate(int32_t fp64, double *tflops, void *stream)
{
    if (!tflops) return PFMM_ERR_INVALID_ARG;
    return fp64 ? probe<double>(tflops, (cudaStream_t)stream) : probe<float>(tflops, (cudaStream_t)stream);
}
