// probe.cu -- arithmetic-rate probe: the throughput of plain fused multiply-adds
// on this GPU, measured as the denominator of the ALU roofline of the FP64
// march (whose FFTs and screen run on the FP64 pipe) and of the FP32 issue
// budget.  Measurement aid; the paper has no counterpart.
//
// Every thread runs kChains independent FMA chains for `iters` rounds, so the
// pipe never waits on a dependency; the rounds are unrolled kUnroll at a time
// so that loop control takes a few percent of the issue slots at most; the
// result feeds a store that never happens in practice but that the compiler
// cannot rule out.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/nlse.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;  // rounds per loop trip (iters is rounded up to a multiple)
constexpr int kProbeThreads = 256;

template <typename T> __global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T seed, T* sink) {
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = seed + (T)(threadIdx.x & 7) + (T)i;
    const T m = (T)0.9999999, c = (T)1e-7;
#pragma unroll 1
    for (int it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
    }
    T s = (T)0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == (T)-1) sink[blockIdx.x] = s;
}

// packed FP32x2: each instruction is two FMAs
__global__ void __launch_bounds__(kProbeThreads) k_fma2_probe(int iters, float seed, float* sink) {
    unsigned long long a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float x = seed + (float)(threadIdx.x & 7) + (float)i, y = x + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(x), "f"(y));
    }
    unsigned long long m, c;
    asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(0.9999999f));
    asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(1e-7f));
#pragma unroll 1
    for (int it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(m), "l"(c));
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[i]));
        s += x + y;
    }
    if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" nlse_status nlse_alu_probe(int32_t kind, int32_t iters, int32_t blocks, void* cuda_stream,
                                      void* sink_dev) {
    if (iters < 1 || blocks < 1 || !sink_dev) return NLSE_EINVAL;
    if (reinterpret_cast<uintptr_t>(sink_dev) % 8 != 0) return NLSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    switch (kind) {
        case 0: k_fma_probe<float><<<blocks, kProbeThreads, 0, s>>>(iters, 1.0f, static_cast<float*>(sink_dev)); break;
        case 1: k_fma_probe<double><<<blocks, kProbeThreads, 0, s>>>(iters, 1.0, static_cast<double*>(sink_dev)); break;
        case 2: k_fma2_probe<<<blocks, kProbeThreads, 0, s>>>(iters, 1.0f, static_cast<float*>(sink_dev)); break;
        default: return NLSE_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}
