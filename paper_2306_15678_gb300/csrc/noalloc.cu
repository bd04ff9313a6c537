// noalloc.cu -- power and peak of a caller's field computed without any device
// allocation: the per-row partial sums of the readout reduction live in a
// file-scope __device__ array instead of a caller workspace.
//
// Who needs this: callers that may not allocate device memory after start-up
// -- for example a service that hands all device memory to its own pool when
// it starts, or a host loop that cannot accept the device-wide synchronisation
// that cudaMalloc and cudaFree may cause.  They pass the field and a two-double
// output buffer they already own; nothing else is needed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/nlse.h"

namespace {

constexpr int kNoallocMaxRows = 8192;  // largest n accepted by nlse_power_peak_noalloc

// (sum |U|^2, max |U|^2) per row: 8192 x 2 doubles = 128 KiB.  Every device that
// loads the library holds this array until the process exits, and every call
// on that device shares it.
static __device__ __align__(256) double g_noalloc_rows[2 * kNoallocMaxRows];

// One block per row: FP64 sum and max of |U|^2 over the row, in a fixed order.
template <typename V>
__global__ void __launch_bounds__(256) k_noalloc_rows(const V* __restrict__ field, int n,
                                                      double* __restrict__ rows) {
    __shared__ double ss[256];
    __shared__ double sm[256];
    const V* line = field + (size_t)blockIdx.x * n;
    double s = 0.0, m = 0.0;
    for (int x = threadIdx.x; x < n; x += 256) {
        const V u = line[x];
        const double a = (double)u.x * (double)u.x + (double)u.y * (double)u.y;
        s += a;
        m = fmax(m, a);
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rows[2 * blockIdx.x] = ss[0];
        rows[2 * blockIdx.x + 1] = sm[0];
    }
}

// One block: fixed-order FP64 combination of the n row partials.
__global__ void __launch_bounds__(256) k_noalloc_total(const double* __restrict__ rows, int n,
                                                       double dx2, double* __restrict__ out) {
    __shared__ double ss[256];
    __shared__ double sm[256];
    double s = 0.0, m = 0.0;
    for (int r = threadIdx.x; r < n; r += 256) {
        s += rows[2 * r];
        m = fmax(m, rows[2 * r + 1]);
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = ss[0] * dx2;
        out[1] = sm[0];
    }
}

// Device address of g_noalloc_rows, looked up once per device with that device
// current.  The host-side name of the array is only a stand-in for it.
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64];
bool g_noalloc_ready[64];

nlse_status noalloc_scratch(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NLSE_ECUDA;
    if (dev < 0 || dev >= 64) return NLSE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ready[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_rows) != cudaSuccess || p == nullptr)
            return NLSE_ECUDA;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
        g_noalloc_ready[dev] = true;
    }
    *out = g_noalloc_ptr[dev];
    return NLSE_OK;
}

}  // namespace

extern "C" nlse_status nlse_power_peak_noalloc(const void* field_dev, int32_t n, int32_t precision,
                                               double L, void* cuda_stream, double* out_dev) {
    if (!field_dev || !out_dev) return NLSE_EINVAL;
    if (n < 1 || !(L > 0.0) || !std::isfinite(L)) return NLSE_EINVAL;
    // the kernels read whole complex values (16 bytes in FP64, 8 in FP32) and
    // store doubles: a misaligned pointer is refused here, not faulted on
    const uintptr_t fa = reinterpret_cast<uintptr_t>(field_dev), oa = reinterpret_cast<uintptr_t>(out_dev);
    if ((fa % (precision == NLSE_FP64 ? 16u : 8u)) != 0 || (oa % 8u) != 0) return NLSE_EINVAL;
    if (n > kNoallocMaxRows) return NLSE_EUNSUPPORTED;  // beyond the static scratch
    if (precision != NLSE_FP64 && precision != NLSE_FP32) return NLSE_EUNSUPPORTED;
    double* rows = nullptr;
    nlse_status st = noalloc_scratch(&rows);
    if (st != NLSE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const double dx = L / (double)n;
    // every row slot [0, n) is rewritten before it is read: nothing to clear
    if (precision == NLSE_FP64)
        k_noalloc_rows<double2><<<n, 256, 0, s>>>(static_cast<const double2*>(field_dev), n, rows);
    else
        k_noalloc_rows<float2><<<n, 256, 0, s>>>(static_cast<const float2*>(field_dev), n, rows);
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    k_noalloc_total<<<1, 256, 0, s>>>(rows, n, dx * dx, out_dev);
    return cudaGetLastError() == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}
