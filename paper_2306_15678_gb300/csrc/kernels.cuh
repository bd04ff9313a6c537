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
    int K;         // multiphoton order
    int active;    // 0: no nonlinear term (screen is the identity)
    int has_gain;  // 0: Re s = 0 everywhere (pure phase screen)
    int reps;      // screens the row pass applies in a row (2: the two half
                   // screens that meet between symmetric steps), power and peak
                   // taken after the first
    T scale;       // factor on the field entering the screen: 1, or 1/n for a
                   // row pass not preceded by a column pass (whose tables carry
                   // the 1/n^2 of the inverse transforms); a power of two, exact
    int exact;     // 1: the exact pointwise substep (real gains) instead of the
                   // frozen screen; its absorption number is a = ka u^(K-1)
    T ka;          // (K-1) c_A beta_K dz I_ref^(K-1)
    int real_gains;  // 1: re_k = re_p = 0 and im_a = 0 (real gains, e.g. the nominal
                     // ones): the exponent's zero terms are skipped (same values)
};

template <typename T> __device__ __forceinline__ T ipow(T u, int e) {
    T r = (T)1;
    T b = u;
#pragma unroll
    for (int bit = 0; bit < 5; ++bit) {  // K <= 16; e is uniform across the grid
        if (e & (1 << bit)) r *= b;
        b *= b;
    }
    return r;
}

// sin x and cos x - 1 for the screen phase in FP32: Cody-Waite reduction by
// pi/2 (two-term constant, FMA) onto [-pi/4, pi/4] and the Taylor polynomials
// of sin (to x^9) and cos - 1 (to x^10), whose truncation errors there are
// below 2e-9 and 2e-10.  Returning cos - 1 instead of cos keeps the rounding
// error of the small screen phases relative to the phase, not to 1.  The
// reduction stays accurate to |x| ~ 1e5 rad; beyond (a diverged march) the
// reduced argument is clamped so the results stay bounded.  When every lane of
// the warp has |x| <= pi/4 (per-step screen phases usually are) the reduction
// and the quadrant fix-up are skipped: they would leave x unchanged, so the
// results are the same bits either way.
// sin r and cos r - 1 for |r| <= pi/4 (the polynomials above)
__device__ __forceinline__ void sin_cosm1_core(float r, float* sr, float* cr1) {
    const float r2 = r * r;
    float ps = fmaf(r2, 2.75573192239858906e-6f, -1.98412698412698413e-4f);
    ps = fmaf(r2, ps, 8.33333333333333333e-3f);
    ps = fmaf(r2, ps, -1.66666666666666667e-1f);
    *sr = fmaf(r * r2, ps, r);                           // sin r
    float pc = fmaf(r2, -2.75573192239858906e-7f, 2.48015873015873016e-5f);
    pc = fmaf(r2, pc, -1.38888888888888889e-3f);
    pc = fmaf(r2, pc, 4.16666666666666667e-2f);
    pc = fmaf(r2, pc, -0.5f);
    *cr1 = r2 * pc;                                      // cos r - 1
}
// warp: the lanes taking part (all 32 in blocks of whole warps).
__device__ __forceinline__ void sin_cosm1(float x, float* s, float* cm1, unsigned warp = 0xffffffffu) {
    const bool small = __all_sync(warp, fabsf(x) <= 0.7853982f);  // uniform per warp
    float r = x, q = 0.0f;
    if (!small) {
        q = rintf(x * 0.636619772367581343f);           // x / (pi/2)
        r = fmaf(-q, 1.57079637050628662f, x);           // pi/2 rounded to FP32
        r = fmaf(-q, -4.37113900018624283e-8f, r);       // pi/2 - fl32(pi/2)
        r = fminf(fmaxf(r, -0.7853982f), 0.7853982f);
    }
    float sr, cr1;
    sin_cosm1_core(r, &sr, &cr1);
    if (small) {
        *s = sr;
        *cm1 = cr1;
        return;
    }
    // x = r + quad pi/2: quad 0 (sr, cr1), 1 (1 + cr1, -sr - 1),
    // 2 (-sr, -2 - cr1), 3 (-1 - cr1, sr - 1)
    const int quad = ((int)q) & 3;
    const bool odd = quad & 1, neg = quad & 2;
    const float sa = odd ? 1.0f + cr1 : sr;
    *s = neg ? -sa : sa;
    *cm1 = odd ? (neg ? sr : -sr) - 1.0f : (neg ? -2.0f - cr1 : cr1);
}

// exp(x) - 1: Taylor polynomial to x^5 for |x| < 1/16 (error < 3e-11 relative),
// expf(x) - 1 beyond; expf is skipped when no lane of the warp needs it
__device__ __forceinline__ float expm1_core(float x) {  // |x| < 1/16
    float p = fmaf(x, 8.33333333333333333e-3f, 4.16666666666666667e-2f);
    p = fmaf(x, p, 1.66666666666666667e-1f);
    p = fmaf(x, p, 0.5f);
    return fmaf(x * x, p, x);
}
__device__ __forceinline__ float expm1_(float x, unsigned warp = 0xffffffffu) {
    const float small = expm1_core(x);
    const bool in_range = fabsf(x) < 0.0625f;
    if (__all_sync(warp, in_range)) return small;
    return in_range ? small : expf(x) - 1.0f;
}

// U = v exp(s(|v|^2)) (Eq. 2: screen evaluated on the field entering it)
template <typename T> __device__ __forceinline__ void screen_exponent(T u, const ScreenCoef<T>& c,
                                                                      T* re, T* im) {
    T uk1, uk;
    if (c.K == 8) {  // the multiphoton order of O2 at 800 nm: u^7 and u^8 by squaring
        const T u2 = u * u, u4 = u2 * u2;
        uk1 = u4 * u2 * u;
        uk = u4 * u4;
    } else {
        uk1 = ipow(u, c.K - 1);
        uk = uk1 * u;
    }
    *re = c.re_k * u + c.re_p * uk + c.re_a * uk1;
    *im = c.im_k * u + c.im_p * uk + c.im_a * uk1;
}

// FP32: U = v + v d with d = exp(re + i im) - 1 = expm1(re) e^{i im} + (e^{i im} - 1),
// so that the per-step change, not the field, carries the rounding of the factor
__device__ __forceinline__ float2 apply_screen(float2 v, const ScreenCoef<float>& c, unsigned warp) {
    const float u = (v.x * v.x + v.y * v.y) * c.inv_iref;
    float re, im;
    screen_exponent(u, c, &re, &im);
    // one vote for both fast paths: the usual case, every lane's phase within
    // pi/4 and gain below 1/16 (the same bits as the general paths give)
    float em1, sn, cm1;
    if (__all_sync(warp, fabsf(im) <= 0.7853982f && fabsf(re) < 0.0625f)) {
        em1 = c.has_gain ? expm1_core(re) : 0.0f;  // uniform: pure phase screens skip it
        sin_cosm1_core(im, &sn, &cm1);
    } else {
        em1 = c.has_gain ? expm1_(re, warp) : 0.0f;
        sin_cosm1(im, &sn, &cm1, warp);
    }
    const float dre = fmaf(em1, cm1, em1 + cm1);  // (1 + em1)(1 + cm1) - 1
    const float dim = fmaf(em1, sn, sn);          // (1 + em1) sin
    // the whole change v d first (accurate relative to itself), then a single
    // rounding of v + v d: adding the small second-order part after rounding the
    // first-order part would lose it at every step, coherently
    const float ddx = fmaf(v.x, dre, -v.y * dim);
    const float ddy = fmaf(v.x, dim, v.y * dre);
    return cadd(v, mk<float2>(ddx, ddy));
}

// FP64: the factor exp(re) (cos im + i sin im) directly
__device__ __forceinline__ double2 apply_screen(double2 v, const ScreenCoef<double>& c, unsigned) {
    const double u = (v.x * v.x + v.y * v.y) * c.inv_iref;
    double re, im;
    screen_exponent(u, c, &re, &im);
    const double amp = exp(re);
    double sn, cs;
    sincos(im, &sn, &cs);
    const double pr = amp * cs, pi = amp * sn;
    return mk<double2>(v.x * pr - v.y * pi, v.x * pi + v.y * pr);
}

// sine and cosine in the precision of the argument
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }

// Exact pointwise substep (real gains, K >= 2): over the step the intensity
// follows dI/dz = -b I^K, I(dz) = I0 (1 + a)^(-1/(K-1)) with a = ka u^(K-1),
// and the phase is the screen's Kerr and plasma coefficients times the step
// averages of u and u^K:
//   <u>   = u   [(1+a)^((K-2)/(K-1)) - 1] / (a (K-2)/(K-1))   (K = 2: ln(1+a)/a),
//   <u^K> = u^K (K-1) [1 - (1+a)^(-1/(K-1))] / a,
// both 1 at a = 0; log1p and expm1 keep small a exact.  Kept out of line: the
// frozen screen's register allocation in the row pass stays as it is.
template <typename T>
__device__ __noinline__ typename vec2<T>::type apply_screen_exact(typename vec2<T>::type v, T inv_iref, T im_k,
                                                                  T im_p, T ka, int K) {
    const T u = (v.x * v.x + v.y * v.y) * inv_iref;
    const T uk1 = ipow(u, K - 1), uk = uk1 * u;
    const T a = ka * uk1;
    T amp = (T)1, f1 = (T)1, fk = (T)1;
    if (a != (T)0) {
        const T l = log1p(a), km1 = (T)(K - 1);
        amp = exp(-l / ((T)2 * km1));
        if (K == 2) {
            f1 = l / a;
        } else {
            const T e = (T)(K - 2) / km1;
            f1 = expm1(e * l) / (a * e);
        }
        fk = -km1 * expm1(-l / km1) / a;
    }
    const T ph = im_k * u * f1 + im_p * uk * fk;
    T sn, cs;
    sincos_(ph, &sn, &cs);
    const T pr = amp * cs, pi = amp * sn;
    return mk<typename vec2<T>::type>(v.x * pr - v.y * pi, v.x * pi + v.y * pr);
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

// FP32 values: the block's tree in FP32 (FP64 arithmetic runs at a small
// fraction of the FP32 rate on this GPU: even a one-thread FP64 loop per block
// holds up the block's end), the sum over all blocks (k_finalize) in FP64, in
// a fixed order.  The FP32 tree adds about 13 roundings to each block sum;
// they are unbiased and independent between blocks.
template <>
__device__ __forceinline__ void block_partials<float>(float tsum, float tmax, double* __restrict__ partials) {
    __shared__ float red_s[32];
    __shared__ float red_m[32];
    if (blockDim.x < 32) {  // tiny grids: blocks narrower than a warp
        red_s[threadIdx.x] = tsum;
        red_m[threadIdx.x] = tmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float ss = 0.0f, mm = 0.0f;
            for (int t = 0; t < (int)blockDim.x; ++t) { ss += red_s[t]; mm = fmaxf(mm, red_m[t]); }
            partials[2 * blockIdx.x] = (double)ss;
            partials[2 * blockIdx.x + 1] = (double)mm;
        }
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
        tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red_s[warp] = tsum; red_m[warp] = tmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        float ss = 0.0f, mm = 0.0f;
        for (int w = 0; w < nw; ++w) { ss += red_s[w]; mm = fmaxf(mm, red_m[w]); }
        partials[2 * blockIdx.x] = (double)ss;
        partials[2 * blockIdx.x + 1] = (double)mm;
    }
}

// Final FP64 reduction of nparts (sum, max) partials by one whole block, in
// an order fixed by the block size B: thread t sums partials t, t + B, t + 2B,
// ... (sixteen loads in flight at a time: the loop is latency-bound otherwise),
// then a shared-memory tree in scratch (2 B doubles).  out[0] = scale * sum,
// out[1] = max; bit 0 of *status flags a non-finite result.  Partials written
// by other blocks of the same launch are read from L2.
__device__ __forceinline__ void block_finalize(const double* partials, int nparts, double scale, double* out,
                                               int* status, double* scratch) {
    constexpr int PER = 16;
    const double2* pp = reinterpret_cast<const double2*>(partials);
    const int B = blockDim.x;
    double s = 0.0, m = 0.0;
    for (int base = threadIdx.x; base < nparts; base += B * PER) {
        double2 buf[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int i = base + q * B;
            buf[q] = i < nparts ? __ldcg(&pp[i]) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            s += buf[q].x;
            m = fmax(m, buf[q].y);
        }
    }
    double* fs = scratch;
    double* fm = scratch + B;
    fs[threadIdx.x] = s;
    fm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (o < B && (int)threadIdx.x < o && (int)threadIdx.x + o < B) {
            fs[threadIdx.x] += fs[threadIdx.x + o];
            fm[threadIdx.x] = fmax(fm[threadIdx.x], fm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double p = fs[0] * scale;
        out[0] = p;
        out[1] = fm[0];
        if (!isfinite(p) || !isfinite(fm[0])) *status |= 1;  // bit 0: non-finite
    }
}

// Deterministic FP64 reduction of nparts (sum, max) pairs: block_finalize by
// one block of 256 (readouts and losses).
static __global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ partials, int nparts,
                                                  double scale, double* __restrict__ out,
                                                  int* __restrict__ status) {
    __shared__ double scratch[512];
    block_finalize(partials, nparts, scale, out, status, scratch);
}

// The same for `count` recorded steps at once (one block each): step i's
// partials start at partials + 2 i nparts and its (power, peak) go to slot
// (first + i) mod cap of the history ring.  The march records the per-block
// partials of its diagnostic steps and finalises them in batches, off the
// path of the step.
static __global__ void __launch_bounds__(256) k_finalize_batch(const double* __restrict__ partials, int nparts,
                                                        double scale, double* __restrict__ hist,
                                                        long long first, int cap, int* __restrict__ status) {
    __shared__ double scratch[512];
    const long long slot = (first + blockIdx.x) % cap;
    block_finalize(partials + 2 * (size_t)blockIdx.x * nparts, nparts, scale, hist + 2 * slot, status, scratch);
}

// ----------------------------------------------------------------- passes --

// complex conjugate of every element: the inverse transform is computed as
// conj(F(conj x)), so each pass emits the forward transform code once and runs
// it twice (a non-unrolled loop), halving the kernel's instruction footprint
template <typename V, int E> __device__ __forceinline__ void conj_all(V (&v)[E]) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m].y = -v[m].y;
}

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
// minimum resident blocks per SM for a 64-register budget per thread
template <int THREADS> __host__ __device__ constexpr int min_blocks() {
    return THREADS >= 1024 ? 1 : (1024 / THREADS > 8 ? 8 : 1024 / THREADS);
}
// shared-memory stride between the lines a block holds; the extra offset
// spreads lines that share a warp over different banks
template <typename T, int N, int LINES> __host__ __device__ constexpr int line_stride() {
    constexpr int banks = 128 / (2 * (int)sizeof(T));
    constexpr int pl = padded_len<N, elems<T, N>()>();
    constexpr int base = (pl + banks - 1) / banks * banks;
    return LINES > 1 ? base + (banks / LINES > 0 ? banks / LINES : 1) : pl;
}

// State layout (row-pair interleaved): element (y, x) of an n x n state array
// lives at ((y / 2) n + x) 2 + (y mod 2).  The two rows of a pair alternate
// element by element, so that a column is a sequence of pairs (y, y+1) of
// adjacent complex values -- 16 bytes in complex64, the smallest unit a bulk
// tensor copy moves -- and a single column can be staged by one such copy,
// while a row is still read and written in one sweep of its row pair.  Only
// the state between the passes uses this layout; the caller's fields are
// row-major.
template <int N> __host__ __device__ __forceinline__ size_t sidx(size_t y, size_t x) {
    return ((y >> 1) * (size_t)N + x) * 2 + (y & 1);
}

// Thread layout of the row-oriented kernels: RPB rows of TL threads each.
// With an even number of rows, the two rows of each row pair alternate thread
// by thread, so that the consecutive threads of a warp read and write
// consecutive words of the interleaved row pair (see sidx).
template <int TL, int RPB> __device__ __forceinline__ int row_of_thread() {
    if constexpr (RPB % 2 == 0) return (int)(threadIdx.x & 1) + 2 * (int)(threadIdx.x / (2 * TL));
    else return (int)(threadIdx.x / TL);
}
template <int TL, int RPB> __device__ __forceinline__ int lane_in_row() {
    if constexpr (RPB % 2 == 0) return (int)(threadIdx.x % (2 * TL)) >> 1;
    else return (int)(threadIdx.x % TL);
}

// Global-memory access policies of the tile bodies: plain accesses for the
// per-pass kernels, L2-only (.cg) accesses for the persistent batched kernel,
// whose tiles are rewritten by other SMs within the same launch.
// kExactScreen: whether the body carries the exact pointwise substep (the
// batched march takes the frozen screen only, and its persistent kernel keeps
// the registers the substep's call would cost).
struct MemPlain {
    static constexpr bool kExactScreen = true;
    template <typename V> __device__ __forceinline__ static V ld(const V* p) { return *p; }
    template <typename V> __device__ __forceinline__ static void st(V* p, V v) { *p = v; }
};
struct MemCG {
    static constexpr bool kExactScreen = false;
    template <typename V> __device__ __forceinline__ static V ld(const V* p) { return __ldcg(p); }
    template <typename V> __device__ __forceinline__ static void st(V* p, V v) { __stcg(p, v); }
};

// Row pass body for RPB consecutive rows starting at row0 (thread layout:
// row group g = tid / TL, in-row index j = tid % TL): v = B_x S, screen,
// S = F_x U.  With DIAG, adds the thread's sum and max of |U|^2.
template <typename T, int N, int RPB, bool DIAG, class M>
__device__ __forceinline__ void row_tile(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
                                         const typename tab_of<T>::type* __restrict__ tw,
                                         const ScreenCoef<T>& sc, int row0, typename vec2<T>::type* smem,
                                         T& tsum, T& tmax) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    const int g = row_of_thread<TL, RPB>(), j = lane_in_row<TL, RPB>();
    const size_t row = (size_t)row0 + g;
    V* sm = smem + g * LS;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = M::ld(src + sidx<N>(row, j + m * TL));
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        if (half == 0) conj_all(v);
        fft_stockham<V, N, E, false>(v, sm, tw, j);
        if (half == 0) {
            conj_all(v);  // v = B_x S: the field entering the screen
            if (sc.scale != (T)1) {  // (uniform)
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = cscale(v[m], sc.scale);
            }
            // lanes of this warp (blocks of fewer than 32 threads exist for tiny grids)
            const unsigned warp = (blockDim.x & 31) == 0 ? 0xffffffffu : __activemask();
#pragma unroll 1
            for (int rep = 0; rep < sc.reps; ++rep) {
                if (sc.active) {
                    if (M::kExactScreen && sc.exact) {  // (uniform)
#pragma unroll
                        for (int m = 0; m < E; ++m)
                            v[m] = apply_screen_exact<T>(v[m], sc.inv_iref, sc.im_k, sc.im_p, sc.ka, sc.K);
                    } else {
#pragma unroll
                        for (int m = 0; m < E; ++m) v[m] = apply_screen(v[m], sc, warp);
                    }
                }
                if (DIAG && rep == 0) {
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        const T a = v[m].x * v[m].x + v[m].y * v[m].y;
                        tsum += a;
                        tmax = fmax(tmax, a);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) M::st(dst + sidx<N>(row, j + m * TL), v[m]);
}

// Column pass body for C consecutive columns starting at col0 (thread layout:
// column c = tid % C, in-column index j = tid / C):
// S <- B_y(P_x(kx) P_y(ky) rot F_y S), P_y carrying 1/n^2 and rot = exp(i theta)
// this step's global phase (see the march in the host code: it decorrelates
// the FP32 rounding of the slowly rotating spectral values from step to step).
template <typename T, int N, int C, class M>
__device__ __forceinline__ void col_tile(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
                                         const typename tab_of<T>::type* __restrict__ tw,
                                         const typename tab_of<T>::type* __restrict__ px,
                                         const typename tab_of<T>::type* __restrict__ py,
                                         typename tab_of<T>::type rot, int col0,
                                         typename vec2<T>::type* smem) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>();
    constexpr int LS = line_stride<T, N, C>();
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int col = col0 + c;
    V* sm = smem + c * LS;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = M::ld(src + sidx<N>(j + m * TL, col));
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        if (half == 1) conj_all(v);  // second round: B_y = conj(F_y(conj(.)))
        fft_stockham<V, N, E, false>(v, sm, tw, j);
        if (half == 0) {
            const auto pxc = tabmul(ldent(px + col), rot);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = twmul<false>(twmul<false>(v[m], pxc), ldent(py + j + m * TL));
        }
    }
    conj_all(v);
#pragma unroll
    for (int m = 0; m < E; ++m) M::st(dst + sidx<N>(j + m * TL, col), v[m]);
}

// Programmatic dependent launch between the passes of the march: a pass lets
// the next pass's blocks be scheduled as soon as all of its own blocks are
// running (their set-up then overlaps its last wave), and waits for the full
// completion, with its memory, of the pass before it ahead of any access to the
// field.  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Row pass kernel of the march; with DIAG the block also reduces sum |U|^2 and
// max |U|^2 of its rows into partials.
template <typename T, int N, bool DIAG>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>(),
                                  min_blocks<threads_per_line<T, N>() * rows_per_block<T, N>()>())
k_row_pass(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
           const typename tab_of<T>::type* __restrict__ tw, ScreenCoef<T> sc, double* __restrict__ partials) {
    using V = typename vec2<T>::type;
    constexpr int RPB = rows_per_block<T, N>();
    extern __shared__ __align__(16) unsigned char smraw[];
    T tsum = (T)0, tmax = (T)0;
    pdl_trigger();
    pdl_wait();
    row_tile<T, N, RPB, DIAG, MemPlain>(src, dst, tw, sc, blockIdx.x * RPB, reinterpret_cast<V*>(smraw),
                                        tsum, tmax);
    if constexpr (DIAG) block_partials<T>(tsum, tmax, partials);
}

// Column pass kernel of the march.
template <typename T, int N, int C>
__global__ void __launch_bounds__(threads_per_line<T, N>() * C, min_blocks<threads_per_line<T, N>() * C>())
k_col_pass(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
           const typename tab_of<T>::type* __restrict__ tw,
           const typename tab_of<T>::type* __restrict__ px, const typename tab_of<T>::type* __restrict__ py,
           typename tab_of<T>::type rot) {
    using V = typename vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    col_tile<T, N, C, MemPlain>(src, dst, tw, px, py, rot, blockIdx.x * C, reinterpret_cast<V*>(smraw));
}

// Forward row transform S = F_x U (load prologue): src row-major, dst in the
// state layout (a different buffer).
template <typename T, int N>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>(),
                                  min_blocks<threads_per_line<T, N>() * rows_per_block<T, N>()>())
k_row_forward(const typename vec2<T>::type* __restrict__ src, typename vec2<T>::type* __restrict__ dst,
              const typename tab_of<T>::type* __restrict__ tw) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), RPB = rows_per_block<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = row_of_thread<TL, RPB>(), j = lane_in_row<TL, RPB>();
    const size_t row = (size_t)blockIdx.x * RPB + g;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = src[row * N + j + m * TL];
    fft_stockham<V, N, E, false>(v, smem + g * LS, tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) dst[sidx<N>(row, j + m * TL)] = v[m];
}

// Readout: U = B_x S / n per row (S in the state layout); reduces sum/max
// |U|^2 into partials and optionally writes U (field_out) and |U|^2 (flu_out),
// row-major.
template <typename T, int N>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>(),
                                  min_blocks<threads_per_line<T, N>() * rows_per_block<T, N>()>())
k_readout(const typename vec2<T>::type* __restrict__ state, const typename tab_of<T>::type* __restrict__ tw,
          typename vec2<T>::type* __restrict__ field_out, T* __restrict__ flu_out,
          double* __restrict__ partials, typename vec2<T>::type unrot) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), RPB = rows_per_block<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = row_of_thread<TL, RPB>(), j = lane_in_row<TL, RPB>();
    const size_t row = (size_t)blockIdx.x * RPB + g;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = state[sidx<N>(row, j + m * TL)];
    fft_stockham<V, N, E, true>(v, smem + g * LS, tw, j);
    const T inv = (T)1 / (T)N;
    T tsum = (T)0, tmax = (T)0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        v[m] = cscale(v[m], inv);
        const T a = v[m].x * v[m].x + v[m].y * v[m].y;
        tsum += a;
        tmax = fmax(tmax, a);
        if (field_out) field_out[row * N + j + m * TL] = cmul(v[m], unrot);  // remove the global phase
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
