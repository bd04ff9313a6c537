// pair.cuh -- FP32 transform engine of the march that works on two lines at
// once (arXiv 2306.15678, Eq. 2: the diffraction operator is applied in
// Fourier space, the screen of Eq. 3 pointwise).
//
// Lanes.  Every value a thread holds is a pair: the same element of two lines
// that go through identical operations -- two adjacent rows (the row pass), or
// the even and the odd rows of one column (the column pass, see pass32.cuh).
// Real and imaginary parts are kept apart, (re0, re1) and (im0, im1), each in
// one 64-bit register pair, so that every add, subtract, multiply and fused
// multiply-add of the butterflies, twiddles and screen is one packed FP32x2
// instruction (add/sub/mul/fma.rn.f32x2) for both lines; each lane rounds
// exactly as the scalar instruction would.  Multiplying by +-i is a renaming
// of the two parts, and so is the inverse transform: with swap(re, im) =
// (im, re), conj(F(conj x)) = swap(F(swap x)), so the engine only ever runs
// the forward transform.
//
// State layout.  Unit u = (p n + x) of an n x n state array holds, as four
// floats, (re(2p, x), re(2p+1, x), im(2p, x), im(2p+1, x)): one 16-byte load
// gives one pair of the row pass (rows 2p, 2p+1 at x) and of the column pass
// (column x at rows 2p, 2p+1).
//
// Algorithm.  Stockham autosort, radix R = E (16) except a smaller final
// radix, thread j of T = L/E holding elements j + m T (m < E) of its pair of
// lines in natural order in and out.  A radix-R pass of stride NS is computed
// in registers as two sub-passes: radix R1 = min(R, 4) with stride NS and
// twiddles W_{R1 NS}^{rA k}, then radix R2 = R/R1 with stride R1 NS and
// twiddles W_{R NS}^{i (k + jA NS)} (k = b mod NS).  Both twiddle sets come
// from the dithered tables (fft.cuh: step s reads copy s mod kDither), so no
// fixed rounded constant multiplies a large share of the values; only the
// first pass (NS = 1, where the sub-pass-B factors are the constants W_R^{i jA}
// common to every butterfly) multiplies by exact constants held as
// unevaluated FP32 pairs (hi + lo).  Pass outputs go through one padded
// shared-memory exchange of 16-byte pairs per pass boundary.
//
// Table entries hold one factor for both lanes, either as float2 (wx, wy),
// loaded with one 8-byte load and copied into both lanes (less L1 space and
// traffic, two register moves per operand), or as float4 (wx, wx, wy, wy),
// loaded as the two packed operands (no moves, more L1); the entry type is the
// table pointer's.  The pass of stride NS (NS > 1) owns (R1-1) NS
// entries W_{R1 NS}^{rA k} at (rA-1) NS + k, followed by (R2-1) R1 NS entries
// W_{R NS}^{i kB} at (i-1) R1 NS + kB.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fft.cuh"

namespace nlse {
namespace pr {

// ------------------------------------------------------------ packed lanes --

struct F2 {
    unsigned long long b;
};

__device__ __forceinline__ F2 pk(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.b) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up(F2 a, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.b));
}
__device__ __forceinline__ float lo(F2 a) {
    float x, y;
    up(a, x, y);
    return x;
}
__device__ __forceinline__ float hi(F2 a) {
    float x, y;
    up(a, x, y);
    return y;
}
__device__ __forceinline__ F2 bc(float x) { return pk(x, x); }
__device__ __forceinline__ F2 add(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(b.b));
    return r;
}
__device__ __forceinline__ F2 sub(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(b.b));
    return r;
}
__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(b.b));
    return r;
}
// a * b + c, fused, lane by lane
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.b) : "l"(a.b), "l"(b.b), "l"(c.b));
    return r;
}
// -a: both sign bits flipped by an integer operation (exact; it runs on the
// integer pipe, which the FP32 work leaves mostly idle)
__device__ __forceinline__ F2 neg(F2 a) {
    F2 r;
    asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(r.b) : "l"(a.b));
    return r;
}

// complex pair: (re0, re1), (im0, im1)
struct C2 {
    F2 re, im;
};
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return {sub(a.re, b.re), sub(a.im, b.im)}; }
// a * w for w = (wx + i wy) given as packed operands and nwy = -wy:
// re = ar wx - ai wy, im = ar wy + ai wx, each with its last add fused
__device__ __forceinline__ C2 cmulw(C2 a, F2 wx, F2 wy, F2 nwy) {
    return {fma(a.re, wx, mul(a.im, nwy)), fma(a.re, wy, mul(a.im, wx))};
}
// swap of the real and imaginary parts (a renaming)
__device__ __forceinline__ C2 swp(C2 a) { return {a.im, a.re}; }

// twiddle entry at a compile-time offset (in entries) from a per-pass base,
// through the read-only path, as the packed operands (wx, wx) and (wy, wy);
// volatile so that the loads stay where they are used (hoisted, they would
// hold registers through the passes)
template <int OFF> __device__ __forceinline__ void ldw(const float2* base, F2& wx, F2& wy) {
    float x, y;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2+%3];" : "=f"(x), "=f"(y) : "l"(base), "n"(OFF * 8));
    wx = bc(x);
    wy = bc(y);
}
template <int OFF> __device__ __forceinline__ void ldw(const float4* base, F2& wx, F2& wy) {
    asm volatile("ld.global.nc.v2.b64 {%0, %1}, [%2+%3];" : "=l"(wx.b), "=l"(wy.b) : "l"(base), "n"(OFF * 16));
}
// a 16-byte entry holding a different factor per lane, (x0, x1, y0, y1), as
// the packed operands (x0, x1) and (y0, y1)
__device__ __forceinline__ void ld_lanes(const float4* p, F2& x, F2& y) {
    asm volatile("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(x.b), "=l"(y.b) : "l"(p));
}
// one FP32 complex table entry (x, y) through the read-only path
__device__ __forceinline__ float2 ld1(const float2* p) {
    float2 r;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}

// ----------------------------------------------------------- exact factors --

// x * c with c given in double: an unevaluated FP32 pair hi + lo
__device__ __forceinline__ F2 mulc(F2 x, double c) {
    const float h = (float)c, l = (float)(c - (double)(float)c);
    return fma(x, bc(h), mul(x, bc(l)));
}
// x * c + y * d with constants c, d (hi + lo each)
__device__ __forceinline__ F2 dotc(F2 x, double c, F2 y, double d) {
    const float ch = (float)c, cl = (float)(c - (double)(float)c);
    const float dh = (float)d, dl = (float)(d - (double)(float)d);
    return fma(x, bc(ch), fma(y, bc(dh), fma(x, bc(cl), mul(y, bc(dl)))));
}

// a * W_16^J (forward: W_16 = exp(-2 pi i / 16))
template <int J> __device__ __forceinline__ C2 w16(C2 a) {
    constexpr int j = J & 15;
    constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, r2 = 0.70710678118654752440;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4) {  // -i
        return {a.im, neg(a.re)};
    } else if constexpr (j == 8) {
        return {neg(a.re), neg(a.im)};
    } else if constexpr (j == 12) {  // +i
        return {neg(a.im), a.re};
    } else if constexpr ((j & 1) == 0) {
        // W^j = r2 (cx - i sx), cx, sx = +-1: re = r2 (cx x + sx y), im = r2 (cx y - sx x)
        constexpr int cx = (j == 2 || j == 14) ? 1 : -1;
        constexpr int sx = (j == 2 || j == 6) ? 1 : -1;
        // x + y and y - x (or their negatives) carry the signs; the constant r2 or -r2
        const F2 s = add(a.re, a.im), d = sub(a.im, a.re);
        // re = r2 (cx x + sx y):  j = 2: s;  6: d;  10: -s;  14: -d
        // im = r2 (cx y - sx x):  j = 2: d;  6: -s; 10: -d;  14: s
        constexpr double re_c = (cx == sx) ? cx * r2 : sx * r2;  // coefficient of s (cx == sx) or d
        constexpr double im_c = (cx == sx) ? cx * r2 : -sx * r2;
        if constexpr (cx == sx) return {mulc(s, re_c), mulc(d, im_c)};
        else return {mulc(d, re_c), mulc(s, im_c)};
    } else {
        // W^j = c - i s: re = x c + y s, im = y c - x s
        constexpr double c = j == 1 ? c1 : j == 3 ? s1 : j == 5 ? -s1 : j == 7 ? -c1
                           : j == 9 ? -c1 : j == 11 ? -s1 : j == 13 ? s1 : c1;
        constexpr double s = j == 1 ? s1 : j == 3 ? c1 : j == 5 ? c1 : j == 7 ? s1
                           : j == 9 ? -s1 : j == 11 ? -c1 : j == 13 ? -c1 : -s1;
        return {dotc(a.re, c, a.im, s), dotc(a.im, c, a.re, -s)};
    }
}

// ---------------------------------------------------------------- DFT_R --

__device__ __forceinline__ void dft2(C2& a0, C2& a1) {
    const C2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}
// forward DFT_4; the products by -i and +i are renamings folded into the adds
__device__ __forceinline__ void dft4(C2& a0, C2& a1, C2& a2, C2& a3) {
    const C2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = {add(t1.re, d.im), sub(t1.im, d.re)};  // t1 - i d
    a3 = {sub(t1.re, d.im), add(t1.im, d.re)};  // t1 + i d
}

// --------------------------------------------------------- Stockham passes --

__host__ __device__ constexpr int split1(int r) { return r >= 4 ? 4 : r; }
__host__ __device__ constexpr int split2(int r) { return r / split1(r); }
// table entries of the pass with radix r and stride ns (none for ns = 1)
__host__ __device__ constexpr int pass_entries(int r, int ns) {
    return ns > 1 ? (split1(r) - 1) * ns + (split2(r) - 1) * split1(r) * ns : 0;
}
// first table entry of the pass with stride ns of an l-point transform with
// e elements per thread; pair_tab_offset(l, e, l) is the size of the table
__host__ __device__ constexpr int pair_tab_offset(int l, int e, int ns) {
    int off = 0, cur = 1;
    while (cur < ns) {
        const int rem = l / cur;
        const int r = rem >= e ? e : rem;
        off += pass_entries(r, cur);
        cur *= r;
    }
    return off;
}
__host__ __device__ constexpr int pair_tab_entries(int l, int e) { return pair_tab_offset(l, e, l); }

// padded shared-memory line (16-byte pairs): one spare slot every E elements
template <int L, int E> __host__ __device__ constexpr int pair_padded_len() { return L + L / E; }
// stride between the lines a block holds: a multiple of 8 slots (128 bytes:
// bulk-tensor copies land at line starts), plus a skew between lines
template <int L, int E, int LINES> __host__ __device__ constexpr int pair_line_stride() {
    constexpr int pl = pair_padded_len<L, E>();
    constexpr int base = (pl + 7) / 8 * 8;
    return LINES > 1 ? base + 8 : base;
}

template <int I, int END, typename F> __device__ __forceinline__ void sfor(F&& f) {
    if constexpr (I < END) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, END>(f);
    }
}

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Forward transform of a pair of lines of length L held in v (layout above).
// `sm` is this group's padded line (pair_padded_len<L, E>() slots); every
// thread of the block must call this (it contains __syncthreads()).  `hook`
// runs at the start of the last pass of a transform with more than one pass,
// when every thread has read the line for the last time: from there on the
// line is free until the transform returns.
template <int L, int E, int NS = 1, class H = NoHook, class TE>
__device__ __forceinline__ void fft_pair(C2 (&v)[E], C2* sm, const TE* __restrict__ tab, int j,
                                         const H& hook = H{}) {
    constexpr int REM = L / NS;
    constexpr int R = REM >= E ? E : REM;
    constexpr bool LAST = (NS * R == L);
    constexpr int T = L / E;
    constexpr int B = E / R;
    constexpr int R1 = split1(R), R2 = split2(R);
    static_assert(E % R == 0, "radix must divide the elements per thread");
    static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16, "radix");
    constexpr int TA = pair_tab_offset(L, E, NS);  // sub-pass A entries
    constexpr int TB = TA + (R1 - 1) * NS;         // sub-pass B entries
    if constexpr (LAST && NS > 1) hook();
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const int b = j + i * T;
        const int k = NS > 1 ? (b & (NS - 1)) : 0;
        C2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[i + r * B];
        // sub-pass A: radix R1 over rA on registers ip + R2 rA, for each ip < R2
        if constexpr (NS > 1 && R1 > 1) {
            const TE* ta = tab + TA + k;
            sfor<1, R1>([&](auto rc) {
                constexpr int rA = decltype(rc)::value;
                F2 wx, wy;
                ldw<(rA - 1) * NS>(ta, wx, wy);
                const F2 nwy = neg(wy);
#pragma unroll
                for (int ip = 0; ip < R2; ++ip) a[ip + R2 * rA] = cmulw(a[ip + R2 * rA], wx, wy, nwy);
            });
        }
#pragma unroll
        for (int ip = 0; ip < R2; ++ip) {
            if constexpr (R1 == 4) dft4(a[ip], a[ip + R2], a[ip + 2 * R2], a[ip + 3 * R2]);
            else if constexpr (R1 == 2) dft2(a[ip], a[ip + R2]);
        }
        // sub-pass B: radix R2 over ip on registers ip + R2 jA, for each jA < R1
        if constexpr (R2 > 1) {
            if constexpr (NS > 1) {
                const TE* tb = tab + TB + k;
                sfor<0, R1>([&](auto jc) {
                    constexpr int jA = decltype(jc)::value;
                    sfor<1, R2>([&](auto ic) {
                        constexpr int ip = decltype(ic)::value;
                        F2 wx, wy;
                        ldw<(ip - 1) * R1 * NS + jA * NS>(tb, wx, wy);
                        a[ip + R2 * jA] = cmulw(a[ip + R2 * jA], wx, wy, neg(wy));
                    });
                });
            } else {
                sfor<0, R1>([&](auto jc) {
                    constexpr int jA = decltype(jc)::value;
                    sfor<1, R2>([&](auto ic) {
                        constexpr int ip = decltype(ic)::value;
                        a[ip + R2 * jA] = w16<ip * jA * (16 / R)>(a[ip + R2 * jA]);
                    });
                });
            }
#pragma unroll
            for (int jA = 0; jA < R1; ++jA) {
                if constexpr (R2 == 4) dft4(a[R2 * jA], a[R2 * jA + 1], a[R2 * jA + 2], a[R2 * jA + 3]);
                else if constexpr (R2 == 2) dft2(a[R2 * jA], a[R2 * jA + 1]);
            }
        }
        // output r = jA + R1 q sits in slot q + R2 jA
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[i + r * B] = a[(r / R1) + R2 * (r % R1)];
        } else {
            const int base = ((b >> ilog2(NS)) << ilog2(NS * R)) + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[padix<E>(base + r * NS)] = a[(r / R1) + R2 * (r % R1)];
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = sm[padix<E>(j + m * T)];
        __syncthreads();
        fft_pair<L, E, NS * R>(v, sm, tab, j, hook);
    }
}

}  // namespace pr
}  // namespace nlse
