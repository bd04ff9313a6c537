// pass32.cuh -- the FP32 (complex64) march on the pair engine (pair.cuh):
// the two HBM sweeps of a split-step z step (arXiv 2306.15678, Eq. 2 with the
// terms of Eq. 1 and Eq. 3), the load prologue and the readout.
//
// State between steps: S = F_x U in the unit layout of pair.cuh, unit
// (p n + x) = (re, im) of rows 2p and 2p+1 at column x.  One step is
//   column pass: S <- B_y( P_x(kx) P_y(ky) rot / n^2 * F_y S )   (diffraction)
//   row pass:    v = B_x S;  U = v exp(s(|v|^2));  S <- F_x U    (screen)
// B = swap F swap is the unnormalised inverse DFT.
//
// Row-oriented kernels hold the two rows of a unit as the two lanes of every
// value: an x-transform of length n on each lane.
//
// Column-oriented kernels hold one column, the even rows in one lane and the
// odd rows in the other (again exactly a unit).  The y-transform of length n
// is then two transforms of length n/2, one per lane, joined by one radix-2
// step across the lanes (decimation in time):
//   X[k] = E[k] + W_n^k O[k],  X[k + n/2] = E[k] - W_n^k O[k]   (k < n/2),
// which leaves the pair (X[k], X[k + n/2]) in one value.  The propagator
// multiplies it there, and the inverse starts with the mirror step
// (decimation in frequency) on the swapped values Y = swap(X P):
//   A[k] = Y[k] + Y[k + n/2],  B[k] = (Y[k] - Y[k + n/2]) W_n^k,
// whose two length-n/2 transforms return the even and odd output rows, i.e.
// the unit again.
#pragma once
#include <cuda.h>

#include "adjoint.cuh"
#include "pair.cuh"
#include "tma.cuh"

namespace nlse {

using pr::C2;
using pr::F2;

// ------------------------------------------------------------- geometry --

// Elements (pairs) per thread: E = 16 (radix-16 passes, 128 registers per
// thread, 512 threads per SM) or E = 8 (radix-8 passes, 64 registers, 1024
// threads per SM: twice the warps, one more exchange per transform); at most L.
template <int L, int E> __host__ __device__ constexpr int p_e() { return L < E ? L : E; }
template <int L, int E> __host__ __device__ constexpr int p_tpl() { return L / p_e<L, E>(); }
// row pairs per block of the row-oriented kernels: at least 128 threads
template <int N, int E> __host__ __device__ constexpr int p_rows() {
    return p_tpl<N, E>() >= 128 ? 1 : (128 / p_tpl<N, E>() > N / 2 ? N / 2 : 128 / p_tpl<N, E>());
}
template <int N, int E> __host__ __device__ constexpr int p_row_threads() { return p_tpl<N, E>() * p_rows<N, E>(); }
template <int N, int E> __host__ __device__ constexpr int p_row_smem() {
    return pr::pair_line_stride<N, p_e<N, E>(), p_rows<N, E>()>() * p_rows<N, E>() * 16;
}
// threads per column and shared memory of a C-column tile (sub-transform length n/2)
template <int N, int E> __host__ __device__ constexpr int p_col_tpl() { return p_tpl<N / 2, E>(); }
template <int N, int E, int C> __host__ __device__ constexpr int p_col_smem() {
    return pr::pair_line_stride<N / 2, p_e<N / 2, E>(), C>() * C * 16;
}
// resident blocks per SM for a budget of 128 (E = 16) or 64 (E = 8) registers
// per thread (a block narrower than a warp still takes a whole warp's registers)
template <int THREADS, int E> __host__ __device__ constexpr int p_min_blocks() {
    constexpr int w = (THREADS + 31) / 32 * 32, budget = E >= 16 ? 512 : 1024;
    return w >= budget ? 1 : (budget / w > 32 ? 32 : budget / w);
}
// the same for the column kernels, whose radix-8 form needs about 85 registers
// per thread (the propagator and cross-lane factors on top of the transform)
template <int THREADS, int E> __host__ __device__ constexpr int p_col_min_blocks() {
    constexpr int w = (THREADS + 31) / 32 * 32, budget = E >= 16 ? 512 : 768;
    return w >= budget ? 1 : (budget / w > 32 ? 32 : budget / w);
}

// Per-step FP32 twiddle block (one of kDither dithered copies, byte offsets
// from its start): the single-line table of fft.cuh (n entries of 8 bytes,
// used by the one-off 2D transforms), the pair tables (8-byte entries) of the
// n-point row transform for E = 16 and E = 8, and those of the n/2-point
// column sub-transforms for E = 16 and E = 8.
//
// Per-step propagator tables (one of kDitherP dithered copies): P_x, n entries
// of 8 bytes; P_y, n/2 pair entries of 16 bytes followed by the n/2 cross-lane
// factors W_n^k of the column pass (8 bytes each), all as (cos - 1, sin) of
// their angle (see col_body32).
//
// Why 256 copies (kDither): a few factors multiply most of the energy of a
// smooth beam every step -- the propagator and cross-lane factors of the low
// frequencies, and the pass-2 twiddles of the butterflies with k = 0 (the
// constants W_16^(i j) as table entries), which receive the low-frequency
// outputs of pass 1.  The residual error of a dithered factor over a cycle,
// up to 1/(2 kDither) of an FP32 unit, then changes the power coherently from
// cycle to cycle: with 16 copies the Kerr-only power drifted by 2e-6 over the
// 856 steps to the first collapse at 4096^2; with 256 (and P_x applied to each
// value, see col_body32) it stays within 1e-6.
constexpr int kDitherP = kDither;
__host__ __device__ constexpr size_t py32_copy_bytes(int n) { return (size_t)16 * (n / 2) + (size_t)8 * (n / 2); }
__host__ __device__ constexpr int tw32_min(int a, int b) { return a < b ? a : b; }
// Pair-table entry formats (pair.cuh): 8-byte (wx, wy) for the row transforms
// (half the L1 footprint and traffic of the tables: row pass 111 -> 103 us at
// 4096^2), 16-byte (wx, wx, wy, wy) for the column transforms, whose kernel
// has no registers left for the copies into both lanes (8-byte entries there:
// 90 -> 112 us, with spills).
using RowTab = float2;
using ColTab = float4;
__host__ __device__ constexpr size_t tw32_row_off(int n, int e) {
    return (size_t)8 * n + (e >= 16 ? 0 : sizeof(RowTab) * pr::pair_tab_entries(n, tw32_min(16, n)));
}
__host__ __device__ constexpr size_t tw32_col_off(int n, int e) {
    return tw32_row_off(n, 8) + sizeof(RowTab) * pr::pair_tab_entries(n, tw32_min(8, n)) +
           (e >= 16 ? 0 : sizeof(ColTab) * pr::pair_tab_entries(n / 2, tw32_min(16, n / 2)));
}
__host__ __device__ constexpr size_t tw32_copy_bytes(int n) {
    return (tw32_col_off(n, 8) + sizeof(ColTab) * pr::pair_tab_entries(n / 2, tw32_min(8, n / 2)) + 255) / 256 * 256;
}

// Global-memory access of the units: plain for the per-pass kernels, L2-only
// (.cg) for the persistent batched kernel whose fields other SMs rewrite.
struct UnitPlain {
    static constexpr bool kExactScreen = true;
    // read once per pass: no L1 allocation (the tables stay cached)
    __device__ __forceinline__ static C2 ld(const float4* p) {
        C2 v;
        asm volatile("ld.global.L1::no_allocate.v2.b64 {%0, %1}, [%2];" : "=l"(v.re.b), "=l"(v.im.b) : "l"(p));
        return v;
    }
    __device__ __forceinline__ static void st(float4* p, C2 v) {
        float4 f;
        pr::up(v.re, f.x, f.y);
        pr::up(v.im, f.z, f.w);
        *p = f;
    }
};
struct UnitCG {
    static constexpr bool kExactScreen = false;
    __device__ __forceinline__ static C2 ld(const float4* p) {
        const float4 f = __ldcg(p);
        return {pr::pk(f.x, f.y), pr::pk(f.z, f.w)};
    }
    __device__ __forceinline__ static void st(float4* p, C2 v) {
        float4 f;
        pr::up(v.re, f.x, f.y);
        pr::up(v.im, f.z, f.w);
        __stcg(p, f);
    }
};

// --------------------------------------------------------------- screen --

namespace pr {

// the polynomials of kernels.cuh (expm1 to x^5, sin to x^9, cos - 1 to x^10),
// lane by lane, same operations in the same order
__device__ __forceinline__ F2 expm1_core2(F2 x) {
    F2 p = fma(x, bc(8.33333333333333333e-3f), bc(4.16666666666666667e-2f));
    p = fma(x, p, bc(1.66666666666666667e-1f));
    p = fma(x, p, bc(0.5f));
    return fma(mul(x, x), p, x);
}
__device__ __forceinline__ void sin_cosm1_core2(F2 r, F2& sr, F2& cr1) {
    const F2 r2 = mul(r, r);
    F2 ps = fma(r2, bc(2.75573192239858906e-6f), bc(-1.98412698412698413e-4f));
    ps = fma(r2, ps, bc(8.33333333333333333e-3f));
    ps = fma(r2, ps, bc(-1.66666666666666667e-1f));
    sr = fma(mul(r, r2), ps, r);
    F2 pc = fma(r2, bc(-2.75573192239858906e-7f), bc(2.48015873015873016e-5f));
    pc = fma(r2, pc, bc(-1.38888888888888889e-3f));
    pc = fma(r2, pc, bc(4.16666666666666667e-2f));
    pc = fma(r2, pc, bc(-0.5f));
    cr1 = mul(r2, pc);
}
// sin r to r^5 and cos r - 1 to r^6 (Taylor), for |r| <= 1/32
__device__ __forceinline__ void sin_cosm1_short2(F2 r, F2& sr, F2& cr1) {
    const F2 r2 = mul(r, r);
    const F2 ps = fma(r2, bc(8.33333333333333333e-3f), bc(-1.66666666666666667e-1f));
    sr = fma(mul(r, r2), ps, r);
    F2 pc = fma(r2, bc(-1.38888888888888889e-3f), bc(4.16666666666666667e-2f));
    pc = fma(r2, pc, bc(-0.5f));
    cr1 = mul(r2, pc);
}
__device__ __forceinline__ F2 ipow2(F2 u, int e) {
    F2 r = bc(1.0f), b = u;
#pragma unroll
    for (int bit = 0; bit < 5; ++bit) {  // K <= 16; e is uniform across the grid
        if (e & (1 << bit)) r = mul(r, b);
        b = mul(b, b);
    }
    return r;
}

// the general per-lane path of the screen (reduction of large phases, expf for
// large gains), kept out of line: it is rare, and inlined it would enlarge the
// row pass's instruction footprint
static __device__ __noinline__ void screen_slow2(float re0, float re1, float im0, float im1, int has_gain, unsigned warp,
                                          F2& em1, F2& sn, F2& cm1) {
    float s0, s1, k0, k1;
    sin_cosm1(im0, &s0, &k0, warp);
    sin_cosm1(im1, &s1, &k1, warp);
    em1 = has_gain ? pk(expm1_(re0, warp), expm1_(re1, warp)) : bc(0.0f);
    sn = pk(s0, s1);
    cm1 = pk(k0, k1);
}

// U = v + v d, d = exp(s(|v|^2)) - 1 (kernels.cuh: apply_screen) on both lanes.
// Warp votes over both lanes of every thread pick a short polynomial (phases
// within 1/32 rad) or the full one (within pi/4); otherwise each lane takes
// the general scalar path of kernels.cuh.
__device__ __forceinline__ C2 apply_screen2(C2 v, const ScreenCoef<float>& c, unsigned warp) {
    const F2 u = mul(fma(v.re, v.re, mul(v.im, v.im)), bc(c.inv_iref));
    F2 uk1, uk;
    if (c.K == 8) {
        const F2 u2 = mul(u, u), u4 = mul(u2, u2);
        uk1 = mul(mul(u4, u2), u);
        uk = mul(u4, u4);
    } else {
        uk1 = ipow2(u, c.K - 1);
        uk = mul(uk1, u);
    }
    F2 re, im;
    if (c.real_gains) {  // (uniform) the zero terms of the general form, skipped: same values
        re = mul(bc(c.re_a), uk1);
        im = fma(bc(c.im_k), u, mul(bc(c.im_p), uk));
    } else {
        re = fma(bc(c.re_k), u, fma(bc(c.re_p), uk, mul(bc(c.re_a), uk1)));
        im = fma(bc(c.im_k), u, fma(bc(c.im_p), uk, mul(bc(c.im_a), uk1)));
    }
    float re0, re1, im0, im1;
    up(re, re0, re1);
    up(im, im0, im1);
    F2 em1, sn, cm1;
    const float ai = fmaxf(fabsf(im0), fabsf(im1)), ar = fmaxf(fabsf(re0), fabsf(re1));
    if (__all_sync(warp, ai <= 0.03125f && ar < 0.0625f)) {
        // phases within 1/32 rad (most of the field at most steps): sin to x^5
        // and cos - 1 to x^6, truncation below 1e-13 relative
        em1 = c.has_gain ? expm1_core2(re) : bc(0.0f);
        sin_cosm1_short2(im, sn, cm1);
    } else if (__all_sync(warp, ai <= 0.7853982f && ar < 0.0625f)) {
        em1 = c.has_gain ? expm1_core2(re) : bc(0.0f);
        sin_cosm1_core2(im, sn, cm1);
    } else {
        screen_slow2(re0, re1, im0, im1, c.has_gain, warp, em1, sn, cm1);
    }
    const F2 dre = fma(em1, cm1, add(em1, cm1));  // (1 + em1)(1 + cm1) - 1
    const F2 dim = fma(em1, sn, sn);              // (1 + em1) sin
    const F2 ddx = fma(v.re, dre, mul(v.im, neg(dim)));
    const F2 ddy = fma(v.re, dim, mul(v.im, dre));
    return {add(v.re, ddx), add(v.im, ddy)};
}

}  // namespace pr

// ------------------------------------------------------------- row tile --

// Row pass transforms of one row pair held in v (B_x S swapped in): B_x,
// screen(s), F_x; with DIAG adds the thread's sum and max of |U|^2 (after the
// first screen); EXACT compiles the exact pointwise substep in.  hook runs in
// the forward transform once the line is free (pair.cuh: fft_pair).
template <int N, int ER, bool DIAG, bool EXACT = true, class H = pr::NoHook>
__device__ __forceinline__ void row_body32(C2 (&v)[p_e<N, ER>()], C2* sm, const RowTab* __restrict__ tab,
                                           const ScreenCoef<float>& sc, int j, float& tsum, float& tmax,
                                           const H& hook = H{}) {
    constexpr int E = p_e<N, ER>();
    F2 fsum = pr::bc(0.0f);
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        pr::fft_pair<N, E>(v, sm, tab, j, [&]() {
            if (half == 1) hook();
        });
        if (half == 0) {
            // the field entering the screen, swapped back
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = pr::swp(v[m]);
            if (sc.scale != 1.0f) {  // (uniform)
                const F2 s = pr::bc(sc.scale);
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = {pr::mul(v[m].re, s), pr::mul(v[m].im, s)};
            }
            const unsigned warp = (blockDim.x & 31) == 0 ? 0xffffffffu : __activemask();
#pragma unroll 1
            for (int rep = 0; rep < sc.reps; ++rep) {
                if (sc.active) {
                    if (EXACT && sc.exact) {  // (uniform)
#pragma unroll
                        for (int m = 0; m < E; ++m) {
                            float r0, r1, i0, i1;
                            pr::up(v[m].re, r0, r1);
                            pr::up(v[m].im, i0, i1);
                            const float2 a = apply_screen_exact<float>(make_float2(r0, i0), sc.inv_iref, sc.im_k,
                                                                       sc.im_p, sc.ka, sc.K);
                            const float2 b = apply_screen_exact<float>(make_float2(r1, i1), sc.inv_iref, sc.im_k,
                                                                       sc.im_p, sc.ka, sc.K);
                            v[m] = {pr::pk(a.x, b.x), pr::pk(a.y, b.y)};
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < E; ++m) v[m] = pr::apply_screen2(v[m], sc, warp);
                    }
                }
                if (DIAG && rep == 0) {
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        const F2 a = pr::fma(v[m].re, v[m].re, pr::mul(v[m].im, v[m].im));
                        fsum = pr::add(fsum, a);
                        float a0, a1;
                        pr::up(a, a0, a1);
                        tmax = fmaxf(tmax, fmaxf(a0, a1));
                    }
                }
            }
        }
    }
    if (DIAG) tsum += pr::lo(fsum) + pr::hi(fsum);
}

// Row pass body for the row pairs pair0 .. pair0 + p_rows - 1 (group g of
// p_tpl threads per pair): v = B_x S, screen(s), S = F_x U; with DIAG adds
// the thread's sum and max of |U|^2 (after the first screen).
template <int N, int ER, int RP, bool DIAG, class M>
__device__ __forceinline__ void row_tile32(const float4* src, float4* dst, const unsigned char* twb,
                                           const ScreenCoef<float>& sc, int pair0, C2* smem, float& tsum,
                                           float& tmax) {
    constexpr int E = p_e<N, ER>(), T = p_tpl<N, ER>();
    constexpr int LS = pr::pair_line_stride<N, E, RP>();
    const int g = (int)threadIdx.x / T, j = (int)threadIdx.x % T;
    const size_t row = (size_t)(pair0 + g) * N;
    C2* sm = smem + g * LS;
    const RowTab* tab = reinterpret_cast<const RowTab*>(twb + tw32_row_off(N, ER));
    C2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = pr::swp(M::ld(src + row + j + m * T));  // B_x = swap F_x swap
    row_body32<N, ER, DIAG, M::kExactScreen>(v, sm, tab, sc, j, tsum, tmax);
#pragma unroll
    for (int m = 0; m < E; ++m) M::st(dst + row + j + m * T, v[m]);
}

// ---------------------------------------------------------- column body --

// Factors near 1.  The cross-lane factors W_n^k and the propagator factors
// P_x(k), P_y(k) = e^{i phi} are held as (d, s) = (cos phi - 1, sin phi) and
// applied as x + x (d + i s): the same two fused operations per part as a
// plain product, but the stored numbers are small where phi is small -- the
// low frequencies that carry most of a smooth beam's energy -- so their
// (dithered) rounding, and with it the residual magnitude error that would
// add up coherently over the steps, is relative to d and s, not to 1.
__device__ __forceinline__ void cmul_1d(float xr, float xi, float2 w, float& re, float& im) {
    re = fmaf(xr, w.x, fmaf(xi, -w.y, xr));
    im = fmaf(xi, w.x, fmaf(xr, w.y, xi));
}

// Column transform body: v holds units (j + m T, col) of one column (lanes:
// even and odd rows); computes B_y(P_x(col) rot P_y / n^2 F_y .) and leaves
// the output units in v.  tw: the step's twiddle block; px: n entries (d, s)
// of P_x; py: n/2 entries (d[k], d[k+n/2], s[k], s[k+n/2]) of P_y (without
// its 1/n^2, which goes with P_x: a power of two, exact), then the n/2
// cross-lane factors (d, s).
template <int N, int EC>
__device__ __forceinline__ void col_body32(C2 (&v)[p_e<N / 2, EC>()], C2* sm, const unsigned char* twb,
                                           const float2* __restrict__ px, const float4* __restrict__ py,
                                           float2 rot, int col, int j) {
    constexpr int L = N / 2, E = p_e<L, EC>(), T = p_tpl<L, EC>();
    const ColTab* tab = reinterpret_cast<const ColTab*>(twb + tw32_col_off(N, EC));
    const float2* cross = reinterpret_cast<const float2*>(py + L);  // after the n/2 P_y entries
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        pr::fft_pair<L, E>(v, sm, tab, j);
        if (half == 0) {
            // rot / n^2 (a power of two: exact) and P_x(col) = 1 + d + i s, each
            // applied to every value (their product, rounded once per column,
            // would carry a magnitude error common to the column's values)
            constexpr float inv_n2 = 1.0f / ((float)N * (float)N);
            const F2 qx = pr::bc(rot.x * inv_n2), qy = pr::bc(rot.y * inv_n2), nqy = pr::bc(-rot.y * inv_n2);
            const float2 pxd = pr::ld1(px + col);
            const F2 xd = pr::bc(pxd.x), xs = pr::bc(pxd.y), nxs = pr::bc(-pxd.y);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int k = j + m * T;
                const float2 w = pr::ld1(cross + k);  // (cos - 1, sin) of W_n^k
                // X[k] = E + t, X[k + L] = E - t, t = W_n^k O
                float er, orr, ei, oi;
                pr::up(v[m].re, er, orr);
                pr::up(v[m].im, ei, oi);
                float tr, ti;
                cmul_1d(orr, oi, w, tr, ti);
                C2 X = {pr::pk(er + tr, er - tr), pr::pk(ei + ti, ei - ti)};
                // rot / n^2 and P_x (both lanes), then P_y (per lane): X + X (d + i s)
                X = pr::cmulw(X, qx, qy, nqy);
                X = {pr::fma(X.re, xd, pr::fma(X.im, nxs, X.re)), pr::fma(X.im, xd, pr::fma(X.re, xs, X.im))};
                F2 yd, ys;
                pr::ld_lanes(py + k, yd, ys);
                X = {pr::fma(X.re, yd, pr::fma(X.im, pr::neg(ys), X.re)), pr::fma(X.im, yd, pr::fma(X.re, ys, X.im))};
                // Y = swap(X): A = Y[k] + Y[k + L], B = (Y[k] - Y[k + L]) W_n^k
                float yr0, yr1, yi0, yi1;
                pr::up(X.im, yr0, yr1);
                pr::up(X.re, yi0, yi1);
                float br, bi;
                cmul_1d(yr0 - yr1, yi0 - yi1, w, br, bi);
                v[m] = {pr::pk(yr0 + yr1, br), pr::pk(yi0 + yi1, bi)};
            }
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = pr::swp(v[m]);  // B_y = swap F swap
}

// ---------------------------------------------------------------- kernels --

// Row pass of the march; with DIAG the block also reduces sum |U|^2 and
// max |U|^2 of its rows into partials.
template <int N, int ER, bool DIAG>
__global__ void __launch_bounds__(p_row_threads<N, ER>(), p_min_blocks<p_row_threads<N, ER>(), ER>())
k_row_pass32(const float4* src, float4* dst, const unsigned char* twb, ScreenCoef<float> sc,
             double* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float tsum = 0.0f, tmax = 0.0f;
    pdl_trigger();
    pdl_wait();
    row_tile32<N, ER, p_rows<N, ER>(), DIAG, UnitPlain>(src, dst, twb, sc, blockIdx.x * p_rows<N, ER>(),
                                                         reinterpret_cast<C2*>(smraw), tsum, tmax);
    if constexpr (DIAG) block_partials<float>(tsum, tmax, partials);
}

// One contiguous bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global into shared memory, counted in bytes on bar; the calling
// thread also arrives on bar, expecting those bytes (plus `extra`, a test hook
// that keeps the phase from completing).
__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                             uint32_t extra = 0) {
    mbar_expect_tx(bar, bytes + extra);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// block_partials<float> (kernels.cuh) for partial slot `slot`, usable again by
// the same block: the same reduction order, so the same bits.
__device__ __forceinline__ void block_partials32_at(float tsum, float tmax, double* __restrict__ partials, int slot) {
    __shared__ float red_s[32];
    __shared__ float red_m[32];
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
        partials[2 * slot] = (double)ss;
        partials[2 * slot + 1] = (double)mm;
    }
    __syncthreads();  // red_s / red_m are free again
}

// Row pass with persistent blocks (one row pair per block at a time, n >= 2048
// at radix 16): block b takes row pairs b, b + G, b + 2G, ... (G blocks).  A
// row pair is n contiguous units, so it is moved into the block's transform
// line by one bulk copy; the copy for the next row pair is issued as soon as
// the forward transform has read the line for the last time, and lands while
// the last transform pass, the stores and the partials of the current row
// pair run.  Arithmetic, stores and partials (one slot per row pair) are those
// of k_row_pass32 at radix 16, bit for bit.  The wait for a copy is bounded as
// in the staged column pass (status bits 2 and 4, tma.cuh).  extra_tx (a test
// hook, 0 in use) makes block 0 expect that many bytes more for its first row
// pair than the copy brings, so that its wait runs out.
template <int N, bool DIAG>
__global__ void __launch_bounds__(p_tpl<N, 16>(), p_min_blocks<p_tpl<N, 16>(), 16>())
k_row_pass32_pf(const float4* src, float4* dst, const unsigned char* twb, ScreenCoef<float> sc,
                double* __restrict__ partials, int* __restrict__ status, uint32_t extra_tx) {
    constexpr int E = p_e<N, 16>(), T = p_tpl<N, 16>(), NP = N / 2;
    constexpr uint32_t BYTES = (uint32_t)N * 16;
    static_assert(p_rows<N, 16>() == 1 && T % 32 == 0, "one row pair of whole warps per block");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint64_t bar;
    __shared__ int s_fail;
    C2* line = reinterpret_cast<C2*>(smraw);
    const RowTab* tab = reinterpret_cast<const RowTab*>(twb + tw32_row_off(N, 16));
    const int j = (int)threadIdx.x;
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        if ((int)blockIdx.x < NP)
            bulk_load_1d(line, src + (size_t)blockIdx.x * N, BYTES, &bar, blockIdx.x == 0 ? extra_tx : 0u);
    }
    __syncthreads();
    uint32_t parity = 0;
#pragma unroll 1
    for (int p = blockIdx.x; p < NP; p += gridDim.x) {
        if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, parity)) {
            if (status) atomicOr(status, 2);
            // the copy still targets this block's memory: wait for it once more
            if (!mbar_wait_bounded(&bar, parity) && status) atomicOr(status, 4);
            s_fail = 1;
        }
        parity ^= 1u;
        __syncthreads();
        if (s_fail) return;  // (uniform)
        C2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = pr::swp(line[j + m * T]);  // B_x = swap F_x swap
        __syncthreads();  // the transforms' exchanges reuse the line
        const int next = p + (int)gridDim.x;
        float tsum = 0.0f, tmax = 0.0f;
        row_body32<N, 16, DIAG>(v, line, tab, sc, j, tsum, tmax, [&]() {
            if (threadIdx.x == 0 && next < NP) {
                fence_proxy_async_smem();  // the exchanges' accesses of the line, before the copy's writes
                bulk_load_1d(line, src + (size_t)next * N, BYTES, &bar);
            }
        });
#pragma unroll
        for (int m = 0; m < E; ++m) UnitPlain::st(dst + (size_t)p * N + j + m * T, v[m]);
        if constexpr (DIAG) block_partials32_at(tsum, tmax, partials, p);
    }
}

// Column tile with per-thread unit loads and stores: C columns from col0
// (column c = tid mod C: a warp's accesses cover C adjacent units per row pair).
template <int N, int EC, int C, class M>
__device__ __forceinline__ void col_tile32(const float4* src, float4* dst, const unsigned char* twb,
                                           const float2* __restrict__ px, const float4* __restrict__ py,
                                           float2 rot, int col0, C2* smem) {
    constexpr int L = N / 2, E = p_e<L, EC>(), T = p_tpl<L, EC>();
    constexpr int LS = pr::pair_line_stride<L, E, C>();
    const int c = (int)threadIdx.x % C, j = (int)threadIdx.x / C;
    const int col = col0 + c;
    C2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = M::ld(src + (size_t)(j + m * T) * N + col);
    col_body32<N, EC>(v, smem + c * LS, twb, px, py, rot, col, j);
#pragma unroll
    for (int m = 0; m < E; ++m) M::st(dst + (size_t)(j + m * T) * N + col, v[m]);
}

// Column pass, C columns per block with per-thread unit loads and stores.
template <int N, int EC, int C>
__global__ void __launch_bounds__(p_col_tpl<N, EC>() * C, p_col_min_blocks<p_col_tpl<N, EC>() * C, EC>())
k_col_pass32(const float4* src, float4* dst, const unsigned char* twb, const float2* __restrict__ px,
             const float4* __restrict__ py, float2 rot) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_trigger();
    pdl_wait();
    col_tile32<N, EC, C, UnitPlain>(src, dst, twb, px, py, rot, blockIdx.x * C, reinterpret_cast<C2*>(smraw));
}

// The staged column tile exists where a column is a whole number of 256-unit
// boxes and the lines fit the shared memory.
template <int N, int EC, int C> __host__ __device__ constexpr bool p_col_tma_valid() {
    return N % (2 * kTmaBoxRows) == 0 && p_col_tpl<N, EC>() * C <= 1024 &&
           p_col_smem<N, EC, C>() + kTmaAlignPad <= 232448;
}

// Column pass with the tile staged by bulk tensor copies: column c of the
// block lands at the start of its own transform line (boxes of 256 units of
// one column; the tensor maps describe the state as n/2 row pairs x n columns
// x 4 words), the threads of a column (c = tid / T) read their units from
// there, transform them (col_body32, bit for bit as k_col_pass32) and write
// them back, and one thread stores the lines with bulk tensor copies.  Waits
// are bounded as in k_col_pass_tma (tma.cuh), with the same status bits.
template <int N, int EC, int C>
__global__ void __launch_bounds__(p_col_tpl<N, EC>() * C, p_col_min_blocks<p_col_tpl<N, EC>() * C, EC>())
k_col_pass32_tma(const __grid_constant__ CUtensorMap mload, const __grid_constant__ CUtensorMap mstore,
                 const unsigned char* twb, const float2* __restrict__ px, const float4* __restrict__ py, float2 rot,
                 int* __restrict__ status, uint32_t extra_tx) {
    constexpr int L = N / 2, E = p_e<L, EC>(), T = p_tpl<L, EC>();
    constexpr int LS = pr::pair_line_stride<L, E, C>(), BOXES = L / kTmaBoxRows;
    constexpr uint32_t BYTES = (uint32_t)(C * L * 16);
    static_assert(p_col_tma_valid<N, EC, C>(), "staged column tile");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint64_t bar;
    __shared__ int s_fail;
    const uint32_t pad = (kTmaAlign - (smem_u32(smraw) & (kTmaAlign - 1))) & (kTmaAlign - 1);
    C2* smem = reinterpret_cast<C2*>(smraw + pad);
    const int col0 = blockIdx.x * C;
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, BYTES + (blockIdx.x == 0 ? extra_tx : 0u));
#pragma unroll 1
        for (int c = 0; c < C; ++c)
#pragma unroll 1
            for (int b = 0; b < BOXES; ++b)
                tma_load_3d(smem + c * LS + b * kTmaBoxRows, &mload, 0, col0 + c, b * kTmaBoxRows, &bar);
        if (!mbar_wait_bounded(&bar, 0)) {
            if (status) atomicOr(status, 2);
            // the copies still target this block's memory: wait for them once more
            if (!mbar_wait_bounded(&bar, 0) && status) atomicOr(status, 4);
            s_fail = 1;
        }
    }
    __syncthreads();
    if (s_fail) return;  // (uniform)
    const int c = (int)threadIdx.x / T, j = (int)threadIdx.x % T;
    C2* line = smem + c * LS;
    C2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = line[j + m * T];
    __syncthreads();  // the staged tile is consumed; the transforms reuse its memory
    // the transforms end with a barrier after their last shared-memory read
    col_body32<N, EC>(v, line, twb, px, py, rot, col0 + c, j);
#pragma unroll
    for (int m = 0; m < E; ++m) line[j + m * T] = v[m];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int cc = 0; cc < C; ++cc)
#pragma unroll 1
            for (int b = 0; b < BOXES; ++b)
                tma_store_3d(&mstore, 0, col0 + cc, b * kTmaBoxRows, smem + cc * LS + b * kTmaBoxRows);
        tma_store_commit_and_wait_read();
    }
}

// Forward row transform S = F_x U (load prologue): src row-major complex64,
// dst in the unit layout (a different buffer).
template <int N>
__global__ void __launch_bounds__(p_row_threads<N, 16>(), p_min_blocks<p_row_threads<N, 16>(), 16>())
k_row_forward32(const float2* __restrict__ src, float4* __restrict__ dst, const unsigned char* twb) {
    constexpr int E = p_e<N, 16>(), T = p_tpl<N, 16>(), RP = p_rows<N, 16>();
    constexpr int LS = pr::pair_line_stride<N, E, RP>();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int g = (int)threadIdx.x / T, j = (int)threadIdx.x % T;
    const size_t p = (size_t)blockIdx.x * RP + g;
    const RowTab* tab = reinterpret_cast<const RowTab*>(twb + tw32_row_off(N, 16));
    C2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const float2 a = src[(2 * p) * N + j + m * T], b = src[(2 * p + 1) * N + j + m * T];
        v[m] = {pr::pk(a.x, b.x), pr::pk(a.y, b.y)};
    }
    pr::fft_pair<N, E>(v, reinterpret_cast<C2*>(smraw) + g * LS, tab, j);
#pragma unroll
    for (int m = 0; m < E; ++m) UnitPlain::st(dst + p * N + j + m * T, v[m]);
}

// Readout: U = B_x S / n per row pair (S in the unit layout); reduces sum/max
// |U|^2 into partials and optionally writes U times unrot (field_out) and
// |U|^2 (flu_out), row-major.
template <int N>
__global__ void __launch_bounds__(p_row_threads<N, 16>(), p_min_blocks<p_row_threads<N, 16>(), 16>())
k_readout32(const float4* __restrict__ state, const unsigned char* twb, float2* __restrict__ field_out,
            float* __restrict__ flu_out, double* __restrict__ partials, float2 unrot) {
    constexpr int E = p_e<N, 16>(), T = p_tpl<N, 16>(), RP = p_rows<N, 16>();
    constexpr int LS = pr::pair_line_stride<N, E, RP>();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int g = (int)threadIdx.x / T, j = (int)threadIdx.x % T;
    const size_t p = (size_t)blockIdx.x * RP + g;
    const RowTab* tab = reinterpret_cast<const RowTab*>(twb + tw32_row_off(N, 16));
    C2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = pr::swp(UnitPlain::ld(state + p * N + j + m * T));
    pr::fft_pair<N, E>(v, reinterpret_cast<C2*>(smraw) + g * LS, tab, j);
    const float inv = 1.0f / (float)N;
    float tsum = 0.0f, tmax = 0.0f;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        float r0, r1, i0, i1;
        pr::up(v[m].im, r0, r1);  // swapped back
        pr::up(v[m].re, i0, i1);
        const float2 u[2] = {make_float2(r0 * inv, i0 * inv), make_float2(r1 * inv, i1 * inv)};
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const float a = u[l].x * u[l].x + u[l].y * u[l].y;
            tsum += a;
            tmax = fmaxf(tmax, a);
            const size_t o = (2 * p + l) * N + j + m * T;
            if (field_out)
                field_out[o] = make_float2(u[l].x * unrot.x - u[l].y * unrot.y, u[l].x * unrot.y + u[l].y * unrot.x);
            if (flu_out) flu_out[o] = a;
        }
    }
    block_partials<float>(tsum, tmax, partials);
}

// ------------------------------------------------------ adjoint (FP32) --
// The adjoint's row kernels hold two transforms at once, so they keep the
// single-line engine of fft.cuh (16 complex per thread, the single-line
// table at the start of the step's twiddle block) on one row per thread
// group; a row's element is half of a unit: (re, im) = words (l, 2 + l).

__device__ __forceinline__ float2 unit_get(const float4* st, size_t u, int l) {
    const float* f = reinterpret_cast<const float*>(st + u);
    return make_float2(f[l], f[2 + l]);
}
__device__ __forceinline__ void unit_put(float4* st, size_t u, int l, float2 v) {
    float* f = reinterpret_cast<float*>(st + u);
    f[l] = v.x;
    f[2 + l] = v.y;
}

// Loss and seed (adjoint.cuh: k_loss_seed) on the unit layout.
template <int N>
__global__ void __launch_bounds__(threads_per_line<float, N>() * rows_per_block<float, N>(),
                                  (min_blocks<threads_per_line<float, N>() * rows_per_block<float, N>()>() + 1) / 2)
k_loss_seed32(const float4* __restrict__ state, float4* __restrict__ gam, const double* __restrict__ target,
              const float2* __restrict__ tw, double seed_scale, double* __restrict__ partials) {
    using V = float2;
    constexpr int E = elems<float, N>(), TL = threads_per_line<float, N>(), RPB = rows_per_block<float, N>();
    constexpr int LS = line_stride<float, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = row_of_thread<TL, RPB>(), j = lane_in_row<TL, RPB>();
    const size_t row = (size_t)blockIdx.x * RPB + g;
    const size_t pu = (row >> 1) * N;
    const int l = (int)(row & 1);
    V* sm = smem + g * LS;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = unit_get(state, pu + j + m * TL, l);
    fft_stockham<V, N, E, true>(v, sm, tw, j);
    const float inv = 1.0f / (float)N;
    double part = 0.0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const V u = cscale(v[m], inv);
        const double F = (double)(u.x * u.x + u.y * u.y);
        const double d = F - target[row * N + j + m * TL];
        part += d * d;
        const float w = (float)(4.0 * d * seed_scale);  // 4 (F - D) / sum D^2
        v[m] = cscale(u, w * inv);                       // and the 1/n of G_S = F_x G_U / n
    }
    fft_stockham<V, N, E, false>(v, sm, tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) unit_put(gam, pu + j + m * TL, l, v[m]);
    block_partials<double>(part, 0.0, partials);
}

// Backward row pass (adjoint.cuh: k_adj_row) on the unit layout.
template <int N>
__global__ void __launch_bounds__(threads_per_line<float, N>() * rows_per_block<float, N>(),
                                  (min_blocks<threads_per_line<float, N>() * rows_per_block<float, N>()>() + 1) / 2)
k_adj_row32(float4* __restrict__ gam, const float4* __restrict__ tn, const float2* __restrict__ tw,
            AdjCoef<float> ac, double* __restrict__ acc) {
    using V = float2;
    using T = float;
    constexpr int E = elems<float, N>(), TL = threads_per_line<float, N>(), RPB = rows_per_block<float, N>();
    constexpr int LS = line_stride<float, N, RPB>();
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    const int g = row_of_thread<TL, RPB>(), j = lane_in_row<TL, RPB>();
    const size_t row = (size_t)blockIdx.x * RPB + g;
    const size_t pu = (row >> 1) * N;
    const int l = (int)(row & 1);
    V* sm = smem + g * LS;
    V vt[E], gw[E];
#pragma unroll
    for (int m = 0; m < E; ++m) vt[m] = unit_get(tn, pu + j + m * TL, l);
    fft_stockham<V, N, E, true>(vt, sm, tw, j);  // v = B_x T
#pragma unroll
    for (int m = 0; m < E; ++m) gw[m] = unit_get(gam, pu + j + m * TL, l);
    fft_stockham<V, N, E, true>(gw, sm, tw, j);  // G_U = B_x G_S
    T th[6] = {(T)0, (T)0, (T)0, (T)0, (T)0, (T)0};
    if (ac.sc.active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const V v = vt[m], G = gw[m];
            const T u = (v.x * v.x + v.y * v.y) * ac.sc.inv_iref;
            T er, ei, sr, si, uk, uk1;
            screen_factor_and_slope(u, ac, &er, &ei, &sr, &si, &uk, &uk1);
            const V w = mk<V>(v.x * er - v.y * ei, v.x * ei + v.y * er);      // U' = v e^s
            const V c = mk<V>(G.x * w.x + G.y * w.y, G.x * w.y - G.y * w.x);  // conj(G) U'
            const T q = (T)2 * (c.x * sr - c.y * si);                           // 2 Re(c s')
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
    for (int m = 0; m < E; ++m) unit_put(gam, pu + j + m * TL, l, gw[m]);
    block_accumulate6<T>(th, acc);
}

}  // namespace nlse
