// FP32 throughput probe: the denominator of the force walk's ALU roofline, measured on the device
// the library runs on.  Every thread runs eight independent chains of fused multiply-adds
// (a <- a * b + c); a fused multiply-add counts as 2 floating-point operations.  The grid fills
// every SM with 2048 resident threads.  Two forms are timed: scalar FP32 FMAs and packed
// two-wide FP32 FMAs (fma.rn.f32x2, one instruction for two FMAs); the roofline takes the larger
// rate.  Nothing of the force step uses this.
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

// The same chains with packed two-wide FMAs: each 64-bit register holds two chains.
__global__ void __launch_bounds__(PK_THREADS) k_ffma2_chains(int iters, float b, float c, float *sink)
{
    unsigned long long a[PK_CHAINS / 2], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int k = 0; k < PK_CHAINS / 2; ++k) {
        const float x0 = (float)(threadIdx.x + 2 * k) * 1e-3f, x1 = (float)(threadIdx.x + 2 * k + 1) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(x0), "f"(x1));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u) {
#pragma unroll
            for (int k = 0; k < PK_CHAINS / 2; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS / 2; ++k) {
        float x0, x1;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(x1) : "l"(a[k]));
        s += x0 + x1;
    }
    if (s == 1234.5f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int evol_fp32_peak(int iters, double *tflops, double *tflops_packed, float *ms)
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
    const double flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * (double)blocks * PK_THREADS;
    int rc = EVOL_OK;
    for (int form = 0; form < 2 && !rc; ++form) {
        if (form == 1 && !tflops_packed) break;
        for (int rep = 0; rep < 2; ++rep) {                 // the first launch warms up
            const int it = rep == 0 ? iters / 8 + 1 : iters;
            cudaEventRecord(e0, st);
            if (form == 0)
                k_ffma_chains<<<blocks, PK_THREADS, 0, st>>>(it, 0.99999994f, 1e-7f, sink);
            else
                k_ffma2_chains<<<blocks, PK_THREADS, 0, st>>>(it, 0.99999994f, 1e-7f, sink);
            cudaEventRecord(e1, st);
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = EVOL_ECUDA;
        float t = 0.f;
        if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = EVOL_ECUDA;
        if (!rc) {
            const double r = flops / (t * 1e-3) / 1e12;
            if (form == 0) {
                *tflops = r;
                if (ms) *ms = t;
            } else {
                *tflops_packed = r;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(sink);
    return rc;
}
