// turbulence.cuh -- kernels of the turbulent layer (arXiv 2306.15678, Sec. 3.3,
// Eqs. 9-10): the step spectrum of the random screen, the unnormalised 2D DFT
// of row-major arrays (also used by the effective lens), and the layer's phase
// factor exp(-i thickness eps_t / (2 k0)) on the row-major field.
#pragma once
#include "kernels.cuh"

namespace nlse {

// Spectral amplitude of the turbulent screen: out = tau xi on the bins with
// p~^2 + q~^2 <= m2max (signed bin numbers; m2max = floor((k_h L / 2 pi)^2),
// the same set as comparing the integer p~^2 + q~^2 with the real bound), 0
// elsewhere; row-major, rows = k_y.  out may alias xi.
template <typename T>
__global__ void k_turb_spectrum(const typename vec2<T>::type* xi, typename vec2<T>::type* out, int n, T tau,
                                long long m2max) {
    using V = typename vec2<T>::type;
    const size_t nn = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(i / n), p = (int)(i % n);
        const long long qq = q < n / 2 ? q : q - n, pp = p < n / 2 ? p : p - n;
        const V v = xi[i];
        out[i] = pp * pp + qq * qq <= m2max ? mk<V>(tau * v.x, tau * v.y) : mk<V>((T)0, (T)0);
    }
}

// Lines per block of the column transform: adjacent columns are read together,
// so that a warp's loads fill whole 32-byte sectors (4 complex64 or 2
// complex128 columns), within 1024 threads per block; small grids keep the row
// kernels' lines per block.
template <typename T, int N> __host__ __device__ constexpr int dft_cols_per_block() {
    constexpr int TL = threads_per_line<T, N>();
    constexpr int sect = 32 / (2 * (int)sizeof(T));
    constexpr int by_threads = 1024 / TL;
    constexpr int l = sect < by_threads ? sect : by_threads;
    constexpr int rpb = rows_per_block<T, N>();
    return rpb > l ? rpb : l;
}
template <typename T, int N, bool COLS> __host__ __device__ constexpr int dft_lines_per_block() {
    return COLS ? dft_cols_per_block<T, N>() : rows_per_block<T, N>();
}

// Unnormalised DFT (forward, or inverse when INV) of every line of a row-major
// n x n array, in place: rows (along x) when COLS is false, columns (along y)
// when true.  Column blocks hold adjacent columns with the column index fastest
// across the threads (coalesced sectors).  Every line is loaded before the
// first exchange barrier and stored after the last, so the transform may
// overwrite its input.
template <typename T, int N, bool COLS, bool INV>
__global__ void __launch_bounds__(threads_per_line<T, N>() * dft_lines_per_block<T, N, COLS>(),
                                  min_blocks<threads_per_line<T, N>() * dft_lines_per_block<T, N, COLS>()>())
k_dft_lines(typename vec2<T>::type* data, const typename tab_of<T>::type* __restrict__ tw) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), LPB = dft_lines_per_block<T, N, COLS>();
    constexpr int LS = line_stride<T, N, LPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = COLS ? (int)(threadIdx.x % LPB) : row_of_thread<TL, LPB>();
    const int j = COLS ? (int)(threadIdx.x / LPB) : lane_in_row<TL, LPB>();
    const size_t line = (size_t)blockIdx.x * LPB + g;
    const size_t base = COLS ? line : line * N, stride = COLS ? N : 1;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = data[base + (size_t)(j + m * TL) * stride];
    fft_stockham<V, N, E, INV>(v, smem + g * LS, tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) data[base + (size_t)(j + m * TL) * stride] = v[m];
}

// The turbulent layer on the row-major field: U <- U exp(-i c Re(eps)),
// c = thickness / (2 k0); the phase and its sine and cosine in the grid
// precision (sincos_ in kernels.cuh).
template <typename T>
__global__ void k_turb_apply(typename vec2<T>::type* field, const typename vec2<T>::type* __restrict__ eps, T c,
                             size_t nn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        T sn, cs;
        sincos_(-c * eps[i].x, &sn, &cs);
        const typename vec2<T>::type u = field[i];
        field[i] = mk<typename vec2<T>::type>(u.x * cs - u.y * sn, u.x * sn + u.y * cs);
    }
}

}  // namespace nlse
