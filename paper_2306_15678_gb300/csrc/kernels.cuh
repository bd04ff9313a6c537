// kernels.cuh -- the two HBM sweeps of one split-step z step (arXiv 2306.15678,
// Eq. 2 with the terms of Eq. 1 and Eq. 3) plus the readout kernels.
//
// State between steps: S = F_x U, the field Fourier-transformed along x only
// (unnormalised), row-major [y][kx].  One step is
//   column pass: S <- B_y( P_x(kx) P_y(ky) / n^2 * F_y S )      (diffraction)
//   row pass:    v = B_x S;  U = v exp(s(|v|^2));  S <- F_x U   (screen)
// where F is the forward and B the unnormalised inverse DFT.  Because the
// screen is pointwise it sits between the inverse and forward row transforms
// in registers, and because P is separable the whole propagator sits between
// the forward and inverse column transforms: every step reads and writes the
// field exactly twice.
#pragma once
#include "fft.cuh"

namespace nlse {

// Coefficients of the screen exponent in scaled intensity u = |v|^2 / I_ref:
//   Re s = re_k u + re_p u^K + re_a u^(K-1),  Im s = im_k u + im_p u^K + im_a u^(K-1)
// (built in FP64 on the host from Eq. 3 and the gains theta, then rounded).
template <typename T> struct ScreenCoef {
    T inv_iref;
    T re_k, re_p, re_a;
    T im_k, im_p, im_a;
    int K;       // multiphoton order
    int active;  // 0: no nonlinear term (screen is the identity)
};

template <typename T> __device__ __forceinline__ T ipow(T u, int e) {
    T r = (T)1;
    T b = u;
    while (e > 0) {  // uniform across the grid: K is a launch constant
        if (e & 1) r *= b;
        b *= b;
        e >>= 1;
    }
    return r;
}

__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }

// U = v exp(s(|v|^2)) (Eq. 2: screen evaluated on the field entering it)
template <typename V, typename T>
__device__ __forceinline__ V apply_screen(V v, const ScreenCoef<T>& c) {
    const T I = v.x * v.x + v.y * v.y;
    const T u = I * c.inv_iref;
    const T uk1 = ipow(u, c.K - 1);
    const T uk = uk1 * u;
    const T re = c.re_k * u + c.re_p * uk + c.re_a * uk1;
    const T im = c.im_k * u + c.im_p * uk + c.im_a * uk1;
    const T amp = exp_(re);
    T sn, cs;
    sincos_(im, &sn, &cs);
    const T pr = amp * cs, pi = amp * sn;
    return mk<V>(v.x * pr - v.y * pi, v.x * pi + v.y * pr);
}

// ------------------------------------------------------------- reductions --

// Per-thread (sum, max) -> per-block FP64 partials, fixed combination order.
template <typename T>
__device__ __forceinline__ void block_partials(T tsum, T tmax, double* __restrict__ partials) {
    __shared__ double red_s[32];
    __shared__ double red_m[32];
    double s = (double)tsum, m = (double)tmax;
    if (blockDim.x < 32) {  // tiny grids: blocks narrower than a warp
        red_s[threadIdx.x] = s;
        red_m[threadIdx.x] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double ss = 0.0, mm = 0.0;
            for (int t = 0; t < (int)blockDim.x; ++t) { ss += red_s[t]; mm = fmax(mm, red_m[t]); }
            partials[2 * blockIdx.x] = ss;
            partials[2 * blockIdx.x + 1] = mm;
        }
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red_s[warp] = s; red_m[warp] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double ss = 0.0, mm = 0.0;
        for (int w = 0; w < nw; ++w) { ss += red_s[w]; mm = fmax(mm, red_m[w]); }
        partials[2 * blockIdx.x] = ss;
        partials[2 * blockIdx.x + 1] = mm;
    }
}

// Deterministic FP64 reduction of nparts (sum, max) pairs; one block of 256.
// out[0] = scale * sum, out[1] = max; flags NONFINITE in *status.
static __global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ partials, int nparts,
                                                  double scale, double* __restrict__ out,
                                                  int* __restrict__ status) {
    __shared__ double ss[256];
    __shared__ double sm[256];
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 256) {
        s += partials[2 * i];
        m = fmax(m, partials[2 * i + 1]);
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
        const double p = ss[0] * scale;
        out[0] = p;
        out[1] = sm[0];
        if (!isfinite(p) || !isfinite(sm[0])) *status |= 1;  // bit 0: non-finite
    }
}

// ----------------------------------------------------------------- passes --

template <typename T> struct KCfg {
    // elements per thread: 16 complex64 or 8 complex128 in registers
    static constexpr int E_MAX = sizeof(T) == 4 ? 16 : 8;
};

template <typename T, int N> __host__ __device__ constexpr int elems() { return N < KCfg<T>::E_MAX ? N : KCfg<T>::E_MAX; }
template <typename T, int N> __host__ __device__ constexpr int threads_per_line() { return N / elems<T, N>(); }
// rows per block of the row-oriented kernels: at least 128 threads per block
template <typename T, int N> __host__ __device__ constexpr int rows_per_block() {
    return threads_per_line<T, N>() >= 128 ? 1
           : (128 / threads_per_line<T, N>() > N ? N : 128 / threads_per_line<T, N>());
}
// shared-memory stride between the lines a block holds; the extra offset
// spreads lines that share a warp over different banks
template <typename T, int N, int LINES> __host__ __device__ constexpr int line_stride() {
    constexpr int banks = 128 / (2 * (int)sizeof(T));
    constexpr int pl = padded_len<N, elems<T, N>()>();
    constexpr int base = (pl + banks - 1) / banks * banks;
    return LINES > 1 ? base + (banks / LINES > 0 ? banks / LINES : 1) : pl;
}

// Row pass of the march: per row v = B_x S, screen, S = F_x U.  With DIAG the
// block also reduces sum |U|^2 and max |U|^2 of its rows into partials.
template <typename T, int N, bool DIAG>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>())
k_row_pass(typename vec2<T>::type* __restrict__ field, const typename tab_of<T>::type* __restrict__ tw,
           ScreenCoef<T> sc, double* __restrict__ partials) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), RPB = rows_per_block<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = threadIdx.x / TL, j = threadIdx.x % TL;
    const int row = blockIdx.x * RPB + g;
    V* line = field + (size_t)row * N;
    V* sm = smem + g * LS;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = line[j + m * TL];
    fft_stockham<V, N, E, true>(v, sm, tw, j);
    T tsum = (T)0, tmax = (T)0;
    if (sc.active) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = apply_screen(v[m], sc);
    }
    if constexpr (DIAG) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const T a = v[m].x * v[m].x + v[m].y * v[m].y;
            tsum += a;
            tmax = fmax(tmax, a);
        }
    }
    fft_stockham<V, N, E, false>(v, sm, tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) line[j + m * TL] = v[m];
    if constexpr (DIAG) block_partials<T>(tsum, tmax, partials);
}

// Column pass: per column kx, S <- B_y(P_x(kx) P_y(ky) F_y S); P_y carries 1/n^2.
template <typename T, int N, int C>
__global__ void __launch_bounds__(threads_per_line<T, N>() * C)
k_col_pass(typename vec2<T>::type* __restrict__ field, const typename tab_of<T>::type* __restrict__ tw,
           const typename tab_of<T>::type* __restrict__ px, const typename tab_of<T>::type* __restrict__ py) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>();
    constexpr int LS = line_stride<T, N, C>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int col = blockIdx.x * C + c;
    V* sm = smem + c * LS;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = field[(size_t)(j + m * TL) * N + col];
    fft_stockham<V, N, E, false>(v, sm, tw, j);
    const auto pxc = __ldg(&px[col]);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = twmul<false>(twmul<false>(v[m], pxc), __ldg(&py[j + m * TL]));
    fft_stockham<V, N, E, true>(v, sm, tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) field[(size_t)(j + m * TL) * N + col] = v[m];
}

// Forward row transform S = F_x U (load prologue); src may equal dst.
template <typename T, int N>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>())
k_row_forward(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
              const typename tab_of<T>::type* __restrict__ tw) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), RPB = rows_per_block<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = threadIdx.x / TL, j = threadIdx.x % TL;
    const size_t row = (size_t)blockIdx.x * RPB + g;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = src[row * N + j + m * TL];
    fft_stockham<V, N, E, false>(v, smem + g * LS, tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) dst[row * N + j + m * TL] = v[m];
}

// Readout: U = B_x S / n per row; reduces sum/max |U|^2 into partials and
// optionally writes U (field_out) and |U|^2 (flu_out).
template <typename T, int N>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>())
k_readout(const typename vec2<T>::type* __restrict__ state, const typename tab_of<T>::type* __restrict__ tw,
          typename vec2<T>::type* __restrict__ field_out, T* __restrict__ flu_out,
          double* __restrict__ partials) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), RPB = rows_per_block<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = threadIdx.x / TL, j = threadIdx.x % TL;
    const size_t row = (size_t)blockIdx.x * RPB + g;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = state[row * N + j + m * TL];
    fft_stockham<V, N, E, true>(v, smem + g * LS, tw, j);
    const T inv = (T)1 / (T)N;
    T tsum = (T)0, tmax = (T)0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        v[m] = cscale(v[m], inv);
        const T a = v[m].x * v[m].x + v[m].y * v[m].y;
        tsum += a;
        tmax = fmax(tmax, a);
        if (field_out) field_out[row * N + j + m * TL] = v[m];
        if (flu_out) flu_out[row * N + j + m * TL] = a;
    }
    block_partials<T>(tsum, tmax, partials);
}

// Mean over aligned ds x ds blocks of an n x n real array.
template <typename T>
__global__ void k_box_mean(const T* __restrict__ in, T* __restrict__ out, int n, int ds) {
    const int m = n / ds;
    const size_t total = (size_t)m * m;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < total;
         o += (size_t)gridDim.x * blockDim.x) {
        const int R = (int)(o / m), C = (int)(o % m);
        double s = 0.0;
        for (int r = 0; r < ds; ++r)
            for (int c = 0; c < ds; ++c) s += (double)in[(size_t)(R * ds + r) * n + C * ds + c];
        out[o] = (T)(s / (double)(ds * ds));
    }
}

}  // namespace nlse
