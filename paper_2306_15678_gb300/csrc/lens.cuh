// lens.cuh -- kernels of the effective-lens screen (arXiv 2306.15678, Sec. 2,
// Eqs. 4-6) on a grid's row-major field:
//   fluence w = |U|^2 into a complex work array, its Gaussian low-pass
//   w_dif = F^-1 exp(-l_dif k^2) F w (Eq. 4; the transforms are k_dft_lines),
//   the lenses = regions of w_dif >= w_l (labelled by the hot-area kernels),
//   the centre of each lens = its pixel of largest w_dif (first in row-major
//   order on a tie), and the screen D_f = sum over centres of the radial
//   ansatz f_lens(|r - r_c|) (Eqs. 5-6), applied as U <- U exp(+i D_f) (Eq. 2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace nlse {

constexpr int kLensSeg = 8;

// Eq. 6: n_re segments of the real part (segment j on r_re[j-1] <= r < r_re[j],
// value a[j] cos(omega[j] r + psi[j])), n_im of the imaginary part; zero beyond
// the last joint.  reach2: a squared distance in cells beyond which both parts
// are zero for certain ((last joint / dx + 1)^2: pixels inside it are decided
// by the joints themselves).
struct LensCoef {
    int n_re, n_im;
    double reach2;
    double r_re[kLensSeg], a[kLensSeg], omega[kLensSeg], psi[kLensSeg];
    double r_im[kLensSeg], b[kLensSeg], nu[kLensSeg], eta[kLensSeg];
};

// wbuf = (|U|^2, 0)
template <typename T>
__global__ void k_lens_fluence(const typename vec2<T>::type* __restrict__ field, typename vec2<T>::type* __restrict__ wbuf,
                               size_t nn) {
    using V = typename vec2<T>::type;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        const V u = field[i];
        wbuf[i] = mk<V>(u.x * u.x + u.y * u.y, (T)0);
    }
}

// spectrum bin (q, p) *= fx[p] fy[q], the separable factors of the low-pass
// exp(-l_dif (kx^2 + ky^2)) = exp(-l_dif kx^2) exp(-l_dif ky^2), with the 1/n^2
// of the inverse transform folded into fy (tables built on the host in FP64)
template <typename T>
__global__ void k_lens_filter(typename vec2<T>::type* wbuf, int n, const T* __restrict__ fx,
                              const T* __restrict__ fy) {
    using V = typename vec2<T>::type;
    const size_t nn = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        const T f = fx[i % n] * fy[i / n];
        const V v = wbuf[i];
        wbuf[i] = mk<V>(v.x * f, v.y * f);
    }
}

// order-preserving key of a positive value
__device__ __forceinline__ unsigned long long lens_key(float w) { return (unsigned long long)__float_as_uint(w); }
__device__ __forceinline__ unsigned long long lens_key(double w) { return (unsigned long long)__double_as_longlong(w); }

// keymax[root] = largest key of the lens (keymax zeroed before)
template <typename T>
__global__ void k_lens_keymax(const typename vec2<T>::type* __restrict__ wd, const int* __restrict__ label,
                              unsigned long long* __restrict__ keymax, size_t nn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        const int root = label[i];
        if (root >= 0) atomicMax(&keymax[root], lens_key(wd[i].x));
    }
}

// centre[root] = smallest index holding the lens's largest value (centre set
// to INT_MAX-like values before)
template <typename T>
__global__ void k_lens_argmax(const typename vec2<T>::type* __restrict__ wd, const int* __restrict__ label,
                              const unsigned long long* __restrict__ keymax, int* __restrict__ centre, size_t nn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        const int root = label[i];
        if (root >= 0 && lens_key(wd[i].x) == keymax[root]) atomicMin(&centre[root], (int)i);
    }
}

// list of the centres, in no particular order (the host sorts it)
__global__ void k_lens_gather(const int* __restrict__ label, const int* __restrict__ centre, int* __restrict__ list,
                              int* __restrict__ count, size_t nn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
        if (label[i] == (int)i) list[atomicAdd(count, 1)] = centre[i];
}

__device__ __forceinline__ void lens_value(const LensCoef& c, double r, double& re, double& im) {
    re = 0.0;
    im = 0.0;
    for (int j = 0; j < c.n_re; ++j)
        if (r < c.r_re[j]) {
            re = c.a[j] * cos(c.omega[j] * r + c.psi[j]);
            break;
        }
    for (int j = 0; j < c.n_im; ++j)
        if (r < c.r_im[j]) {
            im = c.b[j] * cos(c.nu[j] * r + c.eta[j]);
            break;
        }
}

// U <- U exp(i Re D_f - Im D_f), D_f = sum over the centres (in list order) of
// f_lens(dx |r - r_c|), distances across the window (not periodic), in FP64.
// One block per TS x TS tile of pixels (blockDim = (TS, TS), TS*TS a multiple
// of 32): the centres are scanned in chunks of TS*TS; those that reach the tile
// are compacted into shared memory in list order (ballot prefix), so every
// pixel adds its non-zero terms in the list's order.
template <typename T>
__global__ void __launch_bounds__(256) k_lens_apply(typename vec2<T>::type* field, int n, double dx,
                                                    const int* __restrict__ cent, int ncent, LensCoef c) {
    using V = typename vec2<T>::type;
    __shared__ int cand[256];
    __shared__ int wcount[8];
    const int TS = blockDim.x, nt = TS * TS;
    const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int tid = threadIdx.y * TS + threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double dre = 0.0, dim = 0.0;
    for (int base = 0; base < ncent; base += nt) {
        const int k = base + tid;
        bool keep = false;
        int cc = 0;
        if (k < ncent) {
            cc = __ldg(&cent[k]);
            const int cx = cc % n, cy = cc / n;
            const int gx = cx < x0 ? x0 - cx : (cx > x0 + TS - 1 ? cx - (x0 + TS - 1) : 0);
            const int gy = cy < y0 ? y0 - cy : (cy > y0 + TS - 1 ? cy - (y0 + TS - 1) : 0);
            keep = (double)gx * gx + (double)gy * gy < c.reach2;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        int off = 0, total = 0;
        for (int w = 0; w < nt / 32; ++w) {
            if (w < warp) off += wcount[w];
            total += wcount[w];
        }
        if (keep) cand[off + __popc(bal & ((1u << lane) - 1u))] = cc;
        __syncthreads();
        for (int j = 0; j < total; ++j) {
            const int cj = cand[j];
            const double ex = (double)(x - cj % n), ey = (double)(y - cj / n);
            const double d2 = ex * ex + ey * ey;
            if (d2 >= c.reach2) continue;  // beyond the last joint: f_lens = 0
            double fr, fi;
            lens_value(c, dx * sqrt(d2), fr, fi);
            dre += fr;
            dim += fi;
        }
        __syncthreads();  // cand and wcount are rewritten by the next chunk
    }
    if (dre == 0.0 && dim == 0.0) return;
    double sn, cs;
    sincos(dre, &sn, &cs);
    const double amp = exp(-dim);
    const size_t i = (size_t)y * n + x;
    const V u = field[i];
    field[i] = mk<V>((T)(amp * ((double)u.x * cs - (double)u.y * sn)), (T)(amp * ((double)u.x * sn + (double)u.y * cs)));
}

// out = Re(wbuf): w_dif for callers that want it
template <typename T>
__global__ void k_lens_real(const typename vec2<T>::type* __restrict__ wbuf, T* __restrict__ out, size_t nn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
        out[i] = wbuf[i].x;
}

}  // namespace nlse
