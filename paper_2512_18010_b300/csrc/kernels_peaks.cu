// ALU peak microbenchmark (measurement utility, not part of the method): the
// FP32 and FP64 rooflines of the direct q-evaluation kernels are quoted
// against the rate of dependent fused multiply-add chains measured here at
// the clock the GPU holds under that load.
#include <cuda_runtime.h>

#include "scff_internal.h"

namespace scff {
namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hides the FMA latency)
constexpr int kThreads = 256;

// x <- x a + b on kChains chains for `iters` rounds; a < 1 keeps every chain
// bounded (it converges to b / (1 - a)).  The sum is stored only when it
// equals an impossible value, so the compiler keeps the chains and the
// kernel writes nothing in practice.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T a, T b, T *__restrict__ sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1) sink[blockIdx.x] = s;
}

// The same chains on packed FP32 pairs (f32x2: two FMAs per instruction).
__global__ void __launch_bounds__(kThreads) fma2_chain_kernel(int iters, float a, float b, float *__restrict__ sink) {
    unsigned long long x[kChains], a2, b2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(b2) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float v0 = (float)(threadIdx.x + c) * 1e-3f, v1 = (float)(threadIdx.x + 2 * c) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(v0), "f"(v1));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == -1.f) sink[blockIdx.x] = s;
}

}  // namespace

// mode: 0 FP32 FMA chains, 1 FP64, 2 FP32 as packed f32x2 pairs.
cudaError_t measure_alu_peak(int fp64, int iters, double *tflops, double *ms) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8;  // 8 CTAs of 8 warps per SM: 64 resident warps
    void *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(double) * blocks)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
        float best = 0.f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms the clock up
            cudaEventRecord(e0, 0);
            if (fp64 == 1)
                fma_chain_kernel<double><<<blocks, kThreads>>>(iters, 0.999999, 1e-6, (double *)sink);
            else if (fp64 == 2)
                fma2_chain_kernel<<<blocks, kThreads>>>(iters, 0.9999f, 1e-4f, (float *)sink);
            else
                fma_chain_kernel<float><<<blocks, kThreads>>>(iters, 0.9999f, 1e-4f, (float *)sink);
            cudaEventRecord(e1, 0);
            e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && rep > 0 && (best == 0.f || t < best)) best = t;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) {
            const double flops = (fp64 == 2 ? 4.0 : 2.0) * kChains * (double)iters * kThreads * blocks;
            *ms = best;
            *tflops = flops / (best * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return e;
}

}  // namespace scff
