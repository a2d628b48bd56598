// FP32 throughput probe: the denominator of the force walk's ALU roofline, measured on the device
// the library runs on.  Every thread runs eight independent chains of fused multiply-adds
// (a <- a * b + c); a fused multiply-add counts as 2 floating-point operations.  The grid fills
// every SM with 2048 resident threads.  Nothing of the force step uses this.
#include <cuda_runtime.h>
#include <stdint.h>

#include "evol_internal.cuh"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;
constexpr int PK_UNROLL = 64;

__global__ void __launch_bounds__(PK_THREADS) k_ffma_chains(int iters, float b, float c, float *sink)
{
    float a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u) {
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;       // keeps the chains live; never true in practice
}

}  // namespace

extern "C" int evol_fp32_peak(int iters, double *tflops, float *ms)
{
    if (!tflops || iters < 1) return EVOL_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EVOL_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return EVOL_ECUDA;
    const int blocks = sms * (2048 / PK_THREADS);
    float *sink = nullptr;
    if (cudaMalloc((void **)&sink, blocks * sizeof(float)) != cudaSuccess) return EVOL_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    k_ffma_chains<<<blocks, PK_THREADS, 0, st>>>(iters / 8 + 1, 0.99999994f, 1e-7f, sink);   // warm-up
    cudaEventRecord(e0, st);
    k_ffma_chains<<<blocks, PK_THREADS, 0, st>>>(iters, 0.99999994f, 1e-7f, sink);
    cudaEventRecord(e1, st);
    int rc = cudaStreamSynchronize(st) == cudaSuccess ? EVOL_OK : EVOL_ECUDA;
    float t = 0.f;
    if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = EVOL_ECUDA;
    if (!rc) {
        const double flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * (double)blocks * PK_THREADS;
        *tflops = flops / (t * 1e-3) / 1e12;
        if (ms) *ms = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(sink);
    return rc;
}
