// fft.cuh -- register/shared-memory FFT engine for one-dimensional complex
// transforms of length N = 2^n, used by the row and column passes of the
// split-step march (arXiv 2306.15678, Eq. 2: the diffraction operator is
// applied in Fourier space).
//
// Data layout.  A group of T = N/E threads holds one transform; thread j holds
// E elements in registers, element m being x[j + m*T].  This layout is both the
// input layout (coalesced global loads: consecutive threads read consecutive
// addresses) and the output layout (natural frequency order, coalesced stores).
//
// Algorithm.  Stockham autosort, radix R <= E per pass (R = E except for a
// smaller final radix): for butterfly b (0 <= b < N/R) with stride NS (product
// of the earlier radices) and k = b mod NS,
//     a_r = x[b + r N/R] * W_{NS R}^{r k},   (a_0..a_{R-1}) <- DFT_R(a),
//     y[(b / NS) NS R + k + r NS] = a_r.
// The inputs of a thread's butterflies are exactly its registers; only the
// outputs of non-final passes go through shared memory (one padded exchange per
// pass boundary), and the final pass writes each result back into the register
// it came from, in natural order.  Forward is e^{-2 pi i nk/N}, unnormalised;
// the inverse uses conjugate twiddles, also unnormalised.
//
// Twiddles come from a pass-major table built in FP64 on the host: the pass
// with stride NS and radix R owns (R-1) NS consecutive entries, entry
// (r-1) NS + k holding W_{NS R}^{r k}.  A warp's loads for one r are then
// contiguous, and one base address per pass serves all r.
//
// Rounding of the table factors (FP32).  The same twiddles and propagator
// factors are applied at every z step, so a factor rounded to FP32 once would
// act as a fixed operator error that adds up linearly over thousands of steps.
// Instead each table exists in kDither copies whose entries are rounded up or
// down with a dither: entry e of copy d is rounded up when the fraction of an
// FP32 unit by which the exact value exceeds its lower FP32 neighbour is above
// (rev((d + o_e) mod kDither) + 1/2) / kDither, o_e a fixed pseudo-random
// offset per entry and component, rev the bit reversal of the 8-bit copy
// number, and step k uses copy k mod kDither.  The mean factor over every
// kDither (256) steps is then exact to 1/(2 kDither) of an FP32 unit, the rounding
// alternates up and down within a cycle (bit-reversed thresholds: its partial
// sums stay within about one unit), and each multiply stays a plain FP32
// complex product.  The three radix-16
// constants, applied to most values of every pass and all with the same
// rounding error, are kept exact to O(eps^2) as unevaluated FP32 pairs
// (hi + lo, FMA chains): rounded or dithered, their common magnitude error
// changes the power of the whole field every step.  In FP64 every factor is the
// rounded value itself.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace nlse {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };

template <typename V> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename V> __device__ __forceinline__ V mk(typename real_of<V>::type x,
                                                      typename real_of<V>::type y) {
    V r; r.x = x; r.y = y; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// FP32 complex sums and differences as packed FP32x2 operations (one
// instruction for both parts; each part rounds as a scalar add would)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// packed FP32x2 multiply and fused multiply-add, part by part
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
        "fma.rn.f32x2 pr, pa, pb, pc;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
    return mk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cscale(V a, typename real_of<V>::type s) {
    return mk<V>(a.x * s, a.y * s);
}

// copies of each FP32 table (step k uses copy k mod kDither; see above; a step
// reads one copy, so the copies cost memory, not cache)
constexpr int kDither = 256;

// table entry of twiddles and propagator factors: one complex value
template <typename T> struct tab_of;
template <> struct tab_of<float> { using type = float2; };
template <> struct tab_of<double> { using type = double2; };

// Table load through the read-only path at a compile-time byte offset from a
// per-pass base pointer.  Issued as volatile asm with the offset as an
// immediate: one base register serves every r of a pass, and the forward and
// inverse transforms of a kernel cannot share (and keep live) the loaded values.
template <int OFF> __device__ __forceinline__ float2 ldtab(const float2* base) {
    float2 r;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2+%3];" : "=f"(r.x), "=f"(r.y) : "l"(base), "n"(OFF * 8));
    return r;
}
template <int OFF> __device__ __forceinline__ double2 ldtab(const double2* base) {
    double2 r;
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2+%3];" : "=d"(r.x), "=d"(r.y) : "l"(base), "n"(OFF * 16));
    return r;
}

// Load of one table entry through the read-only path at its point in the
// program: volatile, so that the compiler does not hoist a kernel's table loads
// above the transforms (where they would hold registers throughout).
__device__ __forceinline__ float2 ldent(const float2* p) {
    float2 r;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ double2 ldent(const double2* p) {
    double2 r;
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    return r;
}

// compile-time loop helper
template <int I, int END, typename F> __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < END) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, END>(f);
    }
}

// a * w (CONJ = false) or a * conj(w) (CONJ = true)
template <bool CONJ, typename V> __device__ __forceinline__ V twmul(V a, V w) {
    return CONJ ? cmulc(a, w) : cmul(a, w);
}
// product of two table entries
template <typename V> __device__ __forceinline__ V tabmul(V a, V b) { return cmul(a, b); }

// multiply by W_4^1: -i in the forward transform, +i in the inverse
template <bool INV, typename V> __device__ __forceinline__ V rot4(V a) {
    return INV ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}

// x*c with c given in double: one rounding in FP64, hi/lo pair in FP32
__device__ __forceinline__ float mulc(float x, double c) {
    const float h = (float)c, l = (float)(c - (double)h);
    return fmaf(x, h, x * l);
}
__device__ __forceinline__ double mulc(double x, double c) { return x * c; }
// x*c + y*d with constants c, d
__device__ __forceinline__ float dotc(float x, double c, float y, double d) {
    const float ch = (float)c, cl = (float)(c - (double)ch);
    const float dh = (float)d, dl = (float)(d - (double)dh);
    return fmaf(x, ch, fmaf(y, dh, fmaf(x, cl, y * dl)));
}
__device__ __forceinline__ double dotc(double x, double c, double y, double d) { return x * c + y * d; }

// multiply by the constant W_16^J (forward) or its conjugate (inverse)
template <int J, bool INV, typename V> __device__ __forceinline__ V w16(V a) {
    constexpr int j = J & 15;
    constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173,
                     r2 = 0.70710678118654752440;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4) {
        return rot4<INV>(a);
    } else if constexpr (j == 8) {
        return mk<V>(-a.x, -a.y);
    } else if constexpr (j == 12) {
        return rot4<!INV>(a);
    } else if constexpr ((j & 1) == 0) {
        // W_16^j = r2 (cx - i sx) with cx, sx = +-1 (j = 2, 6, 10, 14)
        constexpr int cx = (j == 2 || j == 14) ? 1 : -1;
        constexpr int sx = (j == 2 || j == 6) ? 1 : -1;
        // forward: (x + i y)(cx - i sx) = (cx x + sx y) + i (cx y - sx x); inverse: sx -> -sx
        constexpr int ss = INV ? -sx : sx;
        const auto re = cx * a.x + ss * a.y;
        const auto im = cx * a.y - ss * a.x;
        return mk<V>(mulc(re, r2), mulc(im, r2));
    } else {
        // W_16^j = cos(2 pi j/16) - i sin(2 pi j/16)
        constexpr double c = j == 1 ? c1 : j == 3 ? s1 : j == 5 ? -s1 : j == 7 ? -c1
                           : j == 9 ? -c1 : j == 11 ? -s1 : j == 13 ? s1 : c1;
        constexpr double sn = j == 1 ? s1 : j == 3 ? c1 : j == 5 ? c1 : j == 7 ? s1
                            : j == 9 ? -s1 : j == 11 ? -c1 : j == 13 ? -c1 : -s1;
        // forward: (x + i y)(c - i s); inverse: (x + i y)(c + i s)
        if constexpr (INV) return mk<V>(dotc(a.x, c, a.y, -sn), dotc(a.x, sn, a.y, c));
        else return mk<V>(dotc(a.x, c, a.y, sn), dotc(a.y, c, a.x, -sn));
    }
}

// FP32 forward W_16^J with packed parts: the same fused operations, in the
// same order, as the scalar mulc / dotc forms above (the forward transforms
// of the single-line engine; the inverse takes the generic form).  Called by
// name through w16f, never picked by overload resolution.
template <int J> __device__ __forceinline__ float2 w16_packed(float2 a) {
    constexpr int j = J & 15;
    if constexpr (j == 0 || j == 4 || j == 8 || j == 12) {
        return w16<J, false, float2>(a);
    } else {
        constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173,
                         r2 = 0.70710678118654752440;
        if constexpr ((j & 1) == 0) {
            constexpr int cx = (j == 2 || j == 14) ? 1 : -1;
            constexpr int sx = (j == 2 || j == 6) ? 1 : -1;
            const float2 q = mk<float2>(cx * a.x + sx * a.y, cx * a.y - sx * a.x);
            constexpr float h = (float)r2, l = (float)(r2 - (double)(float)r2);
            return fma2(q, mk<float2>(h, h), mul2(q, mk<float2>(l, l)));
        } else {
            constexpr double c = j == 1 ? c1 : j == 3 ? s1 : j == 5 ? -s1 : j == 7 ? -c1
                               : j == 9 ? -c1 : j == 11 ? -s1 : j == 13 ? s1 : c1;
            constexpr double sn = j == 1 ? s1 : j == 3 ? c1 : j == 5 ? c1 : j == 7 ? s1
                                : j == 9 ? -s1 : j == 11 ? -c1 : j == 13 ? -c1 : -s1;
            constexpr float ch = (float)c, cl = (float)(c - (double)(float)c);
            constexpr float sh = (float)sn, sl = (float)(sn - (double)(float)sn);
            // re = dotc(x, c, y, sn), im = dotc(y, c, x, -sn): lanes (x, y) and (y, x)
            const float2 A = a, S = mk<float2>(a.y, a.x);
            float2 p = mul2(S, mk<float2>(sl, -sl));
            p = fma2(A, mk<float2>(cl, cl), p);
            p = fma2(S, mk<float2>(sh, -sh), p);
            return fma2(A, mk<float2>(ch, ch), p);
        }
    }
}

// W_16^J product used by the butterflies: the packed form for forward FP32
// transforms, the generic form otherwise
template <int J, bool INV, typename V> __device__ __forceinline__ V w16f(V a) {
    if constexpr (std::is_same<V, float2>::value && !INV) return w16_packed<J>(a);
    else return w16<J, INV, V>(a);
}

// ----------------------------------------------------------------- DFT_R --

template <bool INV, typename V> __device__ __forceinline__ void dft2(V& a0, V& a1) {
    V t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV, typename V> __device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
    V t0 = cadd(a0, a2), t1 = csub(a0, a2);
    V t2 = cadd(a1, a3), t3 = rot4<INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// FP32: the four sums and differences of equal sign packed; the two outputs
// that take the rotated difference mix sums and differences part by part and
// stay scalar (same operations, same results as the generic form)
template <bool INV> __device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    if constexpr (INV) {
        a1 = mk<float2>(t1.x - d.y, t1.y + d.x);
        a3 = mk<float2>(t1.x + d.y, t1.y - d.x);
    } else {
        a1 = mk<float2>(t1.x + d.y, t1.y - d.x);
        a3 = mk<float2>(t1.x - d.y, t1.y + d.x);
    }
}

template <int R, bool INV, typename V> __device__ __forceinline__ void dft(V (&a)[R]) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<INV>(a[0], a[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(a[0], a[1], a[2], a[3]);
    } else if constexpr (R == 8) {
        // 8 = 2 x 4: even/odd DFT4 then combine with W_8^k = W_16^(2k)
        dft4<INV>(a[0], a[2], a[4], a[6]);
        dft4<INV>(a[1], a[3], a[5], a[7]);
        V o1 = w16f<2, INV>(a[3]), o2 = w16f<4, INV>(a[5]), o3 = w16f<6, INV>(a[7]);
        V e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
        a[0] = cadd(e0, a[1]); a[4] = csub(e0, a[1]);
        a[1] = cadd(e1, o1);   a[5] = csub(e1, o1);
        a[2] = cadd(e2, o2);   a[6] = csub(e2, o2);
        a[3] = cadd(e3, o3);   a[7] = csub(e3, o3);
    } else if constexpr (R == 16) {
        // 16 = 4 x 4: Y[n2][k1] = DFT4_n1 x[4 n1 + n2]; Y *= W_16^(n2 k1);
        // X[k1 + 4 k2] = DFT4_n2 Y[n2][k1]
        dft4<INV>(a[0], a[4], a[8], a[12]);
        dft4<INV>(a[1], a[5], a[9], a[13]);
        dft4<INV>(a[2], a[6], a[10], a[14]);
        dft4<INV>(a[3], a[7], a[11], a[15]);
        // after these, a[n2 + 4 k1] holds Y[n2][k1]
        a[5] = w16f<1, INV>(a[5]);  a[9] = w16f<2, INV>(a[9]);  a[13] = w16f<3, INV>(a[13]);
        a[6] = w16f<2, INV>(a[6]);  a[10] = w16f<4, INV>(a[10]); a[14] = w16f<6, INV>(a[14]);
        a[7] = w16f<3, INV>(a[7]);  a[11] = w16f<6, INV>(a[11]); a[15] = w16f<9, INV>(a[15]);
        dft4<INV>(a[0], a[1], a[2], a[3]);     // k1 = 0 -> X[0], X[4], X[8], X[12]
        dft4<INV>(a[4], a[5], a[6], a[7]);     // k1 = 1 -> X[1], X[5], X[9], X[13]
        dft4<INV>(a[8], a[9], a[10], a[11]);   // k1 = 2
        dft4<INV>(a[12], a[13], a[14], a[15]); // k1 = 3
        // now a[4 k1 + k2] = X[k1 + 4 k2]; transpose the 4x4 index
        V t;
        t = a[1]; a[1] = a[4]; a[4] = t;
        t = a[2]; a[2] = a[8]; a[8] = t;
        t = a[3]; a[3] = a[12]; a[12] = t;
        t = a[6]; a[6] = a[9]; a[9] = t;
        t = a[7]; a[7] = a[13]; a[13] = t;
        t = a[11]; a[11] = a[14]; a[14] = t;
    } else {
        static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16, "radix");
    }
}

// --------------------------------------------------------- Stockham passes --

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// padded shared-memory index: one spare slot every E elements keeps the
// strided exchange writes free of bank conflicts
template <int E> __device__ __forceinline__ int padix(int p) { return p + (p >> ilog2(E)); }
template <int N, int E> __host__ __device__ constexpr int padded_len() { return N + N / E; }

// first entry of the twiddle block of the pass with stride ns (see above)
__host__ __device__ constexpr int twiddle_offset(int n, int e, int ns) {
    int off = 0, cur = 1;
    while (cur < ns) {
        const int rem = n / cur;
        const int r = rem >= e ? e : rem;
        if (cur > 1) off += (r - 1) * cur;
        cur *= r;
    }
    return off;
}

// Transform held in v (layout above).  `sm` points at this group's padded
// shared-memory line (padded_len<N,E>() elements); every thread of the block
// must call this function (it contains __syncthreads()).
template <typename V, int N, int E, bool INV, int NS = 1>
__device__ __forceinline__ void fft_stockham(
    V (&v)[E], V* sm, const typename tab_of<typename real_of<V>::type>::type* __restrict__ tw, int j) {
    constexpr int REM = N / NS;
    constexpr int R = REM >= E ? E : REM;
    constexpr bool LAST = (NS * R == N);
    constexpr int T = N / E;
    constexpr int B = E / R;
    static_assert(E % R == 0, "radix must divide the elements per thread");
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const int b = j + i * T;
        V a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[i + r * B];
        int k = 0;
        if constexpr (NS > 1) {
            k = b & (NS - 1);
            const auto* twp = tw + (twiddle_offset(N, E, NS) + k);
            static_for<1, R>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                a[r] = twmul<INV>(a[r], ldtab<(r - 1) * NS>(twp));
            });
        }
        dft<R, INV>(a);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[i + r * B] = a[r];
        } else {
            const int base = ((b >> ilog2(NS)) << ilog2(NS * R)) + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[padix<E>(base + r * NS)] = a[r];
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = sm[padix<E>(j + m * T)];
        __syncthreads();
        fft_stockham<V, N, E, INV, NS * R>(v, sm, tw, j);
    }
}

}  // namespace nlse
