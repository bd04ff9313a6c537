// moments.cuh -- spatial moments of the fluence (arXiv 2306.15678, Eq. 8):
// M(p, q) = sum over the grid of I^p (x^2 + y^2)^q dx^2 on the cell centres
// x_j = (j - n/2 + 1/2) dx, I = |U|^2, with Eq. 8's Q^m = M(m, m).
#pragma once
#include <cuda_runtime.h>

namespace nlse {

constexpr int kMomMax = 8;

struct MomentSpec {
    int count;
    int p[kMomMax], q[kMomMax];
};

__device__ __forceinline__ double ipow(double x, int e) {
    double r = 1.0;
    for (; e > 0; e >>= 1, x *= x)
        if (e & 1) r *= x;
    return r;
}

// Per-block FP64 partial sums of every moment (without the dx^2), written to
// partials[block * kMomMax + k]; the host adds the blocks in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_moments(const T* __restrict__ flu, int n, double dx, MomentSpec ms,
                                                 double* __restrict__ partials) {
    __shared__ double red[256];
    double acc[kMomMax];
#pragma unroll
    for (int k = 0; k < kMomMax; ++k) acc[k] = 0.0;
    const size_t nn = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / n), x = (int)(i % n);
        const double xc = ((double)x - n / 2 + 0.5) * dx, yc = ((double)y - n / 2 + 0.5) * dx;
        const double r2 = xc * xc + yc * yc, I = (double)flu[i];
#pragma unroll
        for (int k = 0; k < kMomMax; ++k)
            if (k < ms.count) acc[k] += ipow(I, ms.p[k]) * ipow(r2, ms.q[k]);
    }
    for (int k = 0; k < ms.count; ++k) {
        red[threadIdx.x] = acc[k];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMomMax + k] = red[0];
        __syncthreads();
    }
}

}  // namespace nlse
