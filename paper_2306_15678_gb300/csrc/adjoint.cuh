// adjoint.cuh -- reverse-mode kernels of the split-step march (the paper has no
// adjoint; this differentiates the discrete march of Eq. 2 with the screen of
// Eq. 3) for the fluence-mismatch loss
//     J = sum (|U_M|^2 - D)^2 / sum D^2.
//
// Gradients use G = dJ/dRe + i dJ/dIm.  In the kernels' representation of one
// step (S = F_x U, T = B_y(rho P / n^2) F_y S, v = B_x T, U' = v e^{s(|v|^2)},
// S' = F_x U') the pullbacks are
//     G_U  = B_x G_S                                   (F_x^H = B_x)
//     G_v  = conj(e^s) G_U + 2 Re(conj(G_U) U' s'(|v|^2)) v
//     G_T  = F_x G_v                                   (B_x^H = F_x)
//     G_S  = B_y(conj(rho P) / n^2) F_y G_T            (the column pass with
//                                                       conjugated tables)
// and dJ/dtheta_j accumulates sum Re(conj(G_U) U' ds/dtheta_j).
#pragma once
#include "kernels.cuh"

namespace nlse {

// screen coefficients plus the unit-gain coefficients that theta multiplies:
// s = -i (t0 + i t1) aK u - i (t2 + i t3) aP u^K + (t4 + i t5) aA u^(K-1)
template <typename T> struct AdjCoef {
    ScreenCoef<T> sc;
    T aK, aP, aA;
};

// (1 + d) = e^s as applied by the forward screen, and s'(I) = ds/dI
template <typename T>
__device__ __forceinline__ void screen_factor_and_slope(T u, const AdjCoef<T>& a, T* er, T* ei,
                                                        T* sr, T* si, T* uk, T* uk1) {
    const ScreenCoef<T>& c = a.sc;
    T k1, k, k2;
    if (c.K == 8) {
        const T u2 = u * u, u4 = u2 * u2;
        k2 = u4 * u2;
        k1 = k2 * u;
        k = u4 * u4;
    } else {
        k1 = ipow(u, c.K - 1);
        k = k1 * u;
        k2 = c.K >= 2 ? ipow(u, c.K - 2) : (T)0;
    }
    const T re = c.re_k * u + c.re_p * k + c.re_a * k1;
    const T im = c.im_k * u + c.im_p * k + c.im_a * k1;
    const T Kf = (T)c.K, K1f = (T)(c.K - 1);
    *sr = (c.re_k + Kf * c.re_p * k1 + K1f * c.re_a * k2) * c.inv_iref;
    *si = (c.im_k + Kf * c.im_p * k1 + K1f * c.im_a * k2) * c.inv_iref;
    *uk = k;
    *uk1 = k1;
    if constexpr (sizeof(T) == 4) {
        const unsigned warp = (blockDim.x & 31) == 0 ? 0xffffffffu : __activemask();
        const float em1 = c.has_gain ? expm1_(re, warp) : 0.0f;
        float sn, cm1;
        sin_cosm1(im, &sn, &cm1, warp);
        *er = 1.0f + fmaf(em1, cm1, em1 + cm1);
        *ei = fmaf(em1, sn, sn);
    } else {
        const double amp = exp(re);
        double sn, cs;
        sincos(im, &sn, &cs);
        *er = amp * cs;
        *ei = amp * sn;
    }
}

// six per-thread partial sums -> per-block FP64 sums added into acc[block][6]
template <typename T>
__device__ __forceinline__ void block_accumulate6(const T (&g)[6], double* __restrict__ acc) {
    __shared__ double red[6][32];
    double s[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) s[q] = (double)g[q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockDim.x >= 32) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 6; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
        if (lane == 0)
            for (int q = 0; q < 6; ++q) red[q][warp] = s[q];
    } else {
        for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = s[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int parts = blockDim.x >= 32 ? (int)(blockDim.x >> 5) : (int)blockDim.x;
        for (int q = 0; q < 6; ++q) {
            double t = 0.0;
            for (int w = 0; w < parts; ++w) t += red[q][w];
            acc[6 * blockIdx.x + q] += t;
        }
    }
}

// Loss and seed.  Per row: U = B_x S / n; F = |U|^2; partial of (F - D)^2 in
// FP64; seed G_U = 4 (F - D) U / sum D^2; gam = F_x G_U / n (= G_S).
template <typename T, int N>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>(),
                                  (min_blocks<threads_per_line<T, N>() * rows_per_block<T, N>()>() + 1) / 2)
k_loss_seed(const typename vec2<T>::type* __restrict__ state, typename vec2<T>::type* __restrict__ gam,
            const double* __restrict__ target, const typename tab_of<T>::type* __restrict__ tw,
            double seed_scale, double* __restrict__ partials) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), RPB = rows_per_block<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = row_of_thread<TL, RPB>(), j = lane_in_row<TL, RPB>();
    const size_t row = (size_t)blockIdx.x * RPB + g;
    V* sm = smem + g * LS;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = state[sidx<N>(row, j + m * TL)];
    fft_stockham<V, N, E, true>(v, sm, tw, j);
    const T inv = (T)1 / (T)N;
    double part = 0.0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const V u = cscale(v[m], inv);
        const double F = (double)(u.x * u.x + u.y * u.y);
        const double d = F - target[row * N + j + m * TL];
        part += d * d;
        const T w = (T)(4.0 * d * seed_scale);  // 4 (F - D) / sum D^2
        v[m] = cscale(u, w * inv);               // and the 1/n of G_S = F_x G_U / n
    }
    fft_stockham<V, N, E, false>(v, sm, tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) gam[sidx<N>(row, j + m * TL)] = v[m];
    block_partials<double>(part, 0.0, partials);
}

// Backward row pass of one step: gam <- F_x( adjoint screen( B_x gam ; B_x tn ) ),
// accumulating dJ/dtheta into acc[block][6].  tn is the column-pass output T of
// the forward step being reversed.
template <typename T, int N>
__global__ void __launch_bounds__(threads_per_line<T, N>() * rows_per_block<T, N>(),
                                  (min_blocks<threads_per_line<T, N>() * rows_per_block<T, N>()>() + 1) / 2)
k_adj_row(typename vec2<T>::type* __restrict__ gam, const typename vec2<T>::type* __restrict__ tn,
          const typename tab_of<T>::type* __restrict__ tw, AdjCoef<T> ac, double* __restrict__ acc) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>(), RPB = rows_per_block<T, N>();
    constexpr int LS = line_stride<T, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = row_of_thread<TL, RPB>(), j = lane_in_row<TL, RPB>();
    const size_t row = (size_t)blockIdx.x * RPB + g;
    V* sm = smem + g * LS;
    V vt[E], gw[E];
#pragma unroll
    for (int m = 0; m < E; ++m) vt[m] = tn[sidx<N>(row, j + m * TL)];
    fft_stockham<V, N, E, true>(vt, sm, tw, j);   // v = B_x T
#pragma unroll
    for (int m = 0; m < E; ++m) gw[m] = gam[sidx<N>(row, j + m * TL)];
    fft_stockham<V, N, E, true>(gw, sm, tw, j);   // G_U = B_x G_S
    T th[6] = {(T)0, (T)0, (T)0, (T)0, (T)0, (T)0};
    if (ac.sc.active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const V v = vt[m], G = gw[m];
            const T u = (v.x * v.x + v.y * v.y) * ac.sc.inv_iref;
            T er, ei, sr, si, uk, uk1;
            screen_factor_and_slope(u, ac, &er, &ei, &sr, &si, &uk, &uk1);
            const V w = mk<V>(v.x * er - v.y * ei, v.x * ei + v.y * er);   // U' = v e^s
            const V c = mk<V>(G.x * w.x + G.y * w.y, G.x * w.y - G.y * w.x);  // conj(G) U'
            const T q = (T)2 * (c.x * sr - c.y * si);                        // 2 Re(c s')
            // conj(e^s) G + q v
            gw[m] = mk<V>(er * G.x + ei * G.y + q * v.x, er * G.y - ei * G.x + q * v.y);
            th[0] += ac.aK * u * c.y;
            th[1] += ac.aK * u * c.x;
            th[2] += ac.aP * uk * c.y;
            th[3] += ac.aP * uk * c.x;
            th[4] += ac.aA * uk1 * c.x;
            th[5] -= ac.aA * uk1 * c.y;
        }
    }
    fft_stockham<V, N, E, false>(gw, sm, tw, j);  // G_T = F_x G_v
#pragma unroll
    for (int m = 0; m < E; ++m) gam[sidx<N>(row, j + m * TL)] = gw[m];
    block_accumulate6<T>(th, acc);
}

// sum of squares of n*n doubles into partials (one block per row, 256 threads)
static __global__ void __launch_bounds__(256) k_sumsq_rows(const double* __restrict__ d, int n,
                                                    double* __restrict__ partials) {
    __shared__ double ss[256];
    double s = 0.0;
    for (int x = threadIdx.x; x < n; x += 256) {
        const double a = d[(size_t)blockIdx.x * n + x];
        s += a * a;
    }
    ss[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) ss[threadIdx.x] += ss[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = ss[0];
        partials[2 * blockIdx.x + 1] = 0.0;
    }
}

}  // namespace nlse
