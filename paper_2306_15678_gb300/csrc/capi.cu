// capi.cu -- host implementation of the C ABI declared in include/nlse.h:
// parameter validation, FP64 construction of the propagator, twiddle and
// screen tables (arXiv 2306.15678, Eq. 1-3), workspace carving, and the launch
// sequence of the split-step march (Eq. 2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/nlse.h"
#include "dispatch32.cuh"
#include "hot_areas.cuh"
#include "lens.cuh"
#include "moments.cuh"
#include "host_detail.h"

using namespace nlse;

namespace {

constexpr int kHistCap = 4096;
constexpr int kDiagBatch = 64;  // diagnostic steps whose per-block partials are finalised together
constexpr double kIref = 1.0e13;  // W/cm^2: scale of the screen's intensity variable
constexpr double kTwoPi = 6.283185307179586476925286766559;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// bytes of the device propagator tables: FP64 one copy of n 16-byte entries
// each; FP32 kDitherP dithered copies of P_x (n entries of 8 bytes) and of P_y
// with the cross-lane factors (pass32.cuh: py32_copy_bytes)
size_t px_bytes(int n, int precision) {
    return precision == NLSE_FP64 ? (size_t)n * 16 : (size_t)kDitherP * n * 8;
}
size_t py_bytes(int n, int precision) {
    return precision == NLSE_FP64 ? (size_t)n * 16 : (size_t)kDitherP * py32_copy_bytes(n);
}
// bytes of the twiddle region: FP64 one pass-major table of n 16-byte
// entries; FP32 kDither twiddle blocks (pass32.cuh: tw32_copy_bytes)
size_t tw_region_bytes(int n, int precision) {
    return precision == NLSE_FP64 ? (size_t)n * 16 : (size_t)kDither * tw32_copy_bytes(n);
}

int log2_exact(int n) {
    if (n <= 0 || (n & (n - 1))) return -1;
    int k = 0;
    while ((1 << k) < n) ++k;
    return k;
}

struct Layout {
    size_t state, aux, tw, px, py, partials, diag, hist, readout, status, total;
};

Layout layout_for(int n, int precision) {
    const size_t cs = precision == NLSE_FP64 ? 16 : 8;
    const size_t nn = (size_t)n * n;
    Layout L;
    size_t o = 0;
    L.state = o;    o = align256(o + nn * cs);
    L.aux = o;      o = align256(o + nn * cs);
    L.tw = o;       o = align256(o + tw_region_bytes(n, precision));
    L.px = o;       o = align256(o + px_bytes(n, precision));
    L.py = o;       o = align256(o + py_bytes(n, precision));
    L.partials = o; o = align256(o + (size_t)n * 2 * sizeof(double));
    L.diag = o;     o = align256(o + (size_t)kDiagBatch * n * 2 * sizeof(double));
    L.hist = o;     o = align256(o + (size_t)kHistCap * 2 * sizeof(double));
    L.readout = o;  o = align256(o + 2 * sizeof(double));
    L.status = o;   o = align256(o + sizeof(int));
    L.total = o;
    return L;
}

nlse_status validate(const nlse_params* p) {
    if (!p) return NLSE_EINVAL;
    const int k = log2_exact(p->n);
    if (k < 0) return NLSE_EINVAL;
    if (k < 3 || k > 13) return NLSE_EUNSUPPORTED;
    if (p->precision != NLSE_FP64 && p->precision != NLSE_FP32) return NLSE_EUNSUPPORTED;
    if (p->K < 1 || p->K > 16) return NLSE_EINVAL;
    if ((p->terms & ~15u) != 0) return NLSE_EINVAL;
    if (!(p->L > 0.0) || !std::isfinite(p->L)) return NLSE_EINVAL;
    if (p->dz == 0.0 || !std::isfinite(p->dz)) return NLSE_EINVAL;
    if (!(p->lambda0 > 0.0) || !(p->n0 > 0.0)) return NLSE_EINVAL;
    const double vals[] = {p->n2, p->sigmaK, p->rho_nt, p->rho_c, p->tau_pl, p->betaK};
    for (double v : vals)
        if (!std::isfinite(v)) return NLSE_EINVAL;
    if ((p->terms & NLSE_PLASMA) && !(p->rho_c > 0.0)) return NLSE_EINVAL;
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(p->theta[i])) return NLSE_EINVAL;
    if (p->diag_every < 0 || p->scheme < 0 || p->scheme > (NLSE_STRANG | NLSE_EXACT_SCREEN)) return NLSE_EINVAL;
    // the exact substep has a closed form for real gains and K >= 2 only
    if ((p->scheme & NLSE_EXACT_SCREEN) && (p->theta[1] != 0.0 || p->theta[3] != 0.0 || p->theta[5] != 0.0 || p->K < 2))
        return NLSE_EINVAL;
    return NLSE_OK;
}

// signed frequency index of FFT bin m
inline double signed_bin(int m, int n) { return (double)(m < n / 2 ? m : m - n); }

// Separable diffraction tables (Eq. 1-2, Lap_perp -> -(kx^2 + ky^2)):
// P_x(m) = exp(i k_m^2 dz / (2 k0)), P_y(m) = the same divided by n^2 (the
// normalisation of the inverse 2D transform).  Phases in FP64, reduced mod 2 pi.
// phase k_m^2 dz / (2 k0) of FFT bin m, reduced mod 2 pi (0 without diffraction)
double propagator_phase(const nlse_params* p, int m) {
    const double k0 = kTwoPi * p->n0 / p->lambda0;
    const double k = kTwoPi * signed_bin(m, p->n) / p->L;
    return (p->terms & NLSE_DIFFRACTION) ? std::fmod(k * k * p->dz / (2.0 * k0), kTwoPi) : 0.0;
}

void propagator_tables(const nlse_params* p, std::vector<double>& px, std::vector<double>& py) {
    const int n = p->n;
    const double inv_n2 = 1.0 / ((double)n * (double)n);
    px.resize(2 * (size_t)n);
    py.resize(2 * (size_t)n);
    for (int m = 0; m < n; ++m) {
        const double ph = propagator_phase(p, m);
        const double c = std::cos(ph), s = std::sin(ph);
        px[2 * m] = c;
        px[2 * m + 1] = s;
        py[2 * m] = c * inv_n2;
        py[2 * m + 1] = s * inv_n2;
    }
}

// Pass-major twiddle table in FP64 for transforms of length n done with e
// elements per thread (radix e, last pass possibly smaller): the pass with
// stride ns and radix r owns (r-1) ns entries, entry (rr-1) ns + k holding
// W_{ns r}^{rr k} = exp(-2 pi i rr k / (ns r)).  Angles are reduced exactly in
// integers before the FP64 cos/sin.
void twiddle_table(int n, int e, std::vector<double>& tw) {
    tw.assign(2 * (size_t)n, 0.0);
    int cur = 1, off = 0;
    while (cur < n) {
        const int rem = n / cur;
        const int r = rem >= e ? e : rem;
        if (cur > 1) {
            const long long period = (long long)cur * r;
            for (int rr = 1; rr < r; ++rr)
                for (int k = 0; k < cur; ++k) {
                    const long long m = ((long long)rr * k) % period;
                    const double a = kTwoPi * (double)m / (double)period;
                    const size_t i = (size_t)off + (size_t)(rr - 1) * cur + k;
                    const double c = std::cos(a), sn = std::sin(a);
                    tw[2 * i] = c;
                    tw[2 * i + 1] = -sn;
                }
            off += (r - 1) * cur;
        }
        cur *= r;
    }
}

// Screen coefficients (Eq. 2-3) in u = I / I_ref:
//   s = -i dz/(2 k0) [c_K eps_k I + c_P eps_m I^K + c_A i k0 alpha_m I^(K-1)]
//     = -i c_K a_K u + (-i c_P a_P) u^K + c_A a_A u^(K-1)
// with a_K = dz eps_k/(2 k0) I_ref, a_P = dz eps_m/(2 k0) I_ref^K,
// a_A = dz alpha_m/2 I_ref^(K-1).
template <typename T> ScreenCoef<T> screen_coef(const nlse_params* p) {
    const double k0 = kTwoPi * p->n0 / p->lambda0;
    const double eps_k = 2.0 * k0 * k0 * p->n2 / p->n0;
    const double eps_m = -k0 * k0 * p->sigmaK * p->rho_nt * p->tau_pl / p->rho_c;
    const double alpha_m = -p->betaK;
    const double aK = (p->terms & NLSE_KERR) ? p->dz * eps_k / (2.0 * k0) * kIref : 0.0;
    const double aP = (p->terms & NLSE_PLASMA)
                          ? p->dz * eps_m / (2.0 * k0) * std::pow(kIref, (double)p->K)
                          : 0.0;
    const double aA = (p->terms & NLSE_MPA)
                          ? p->dz * alpha_m / 2.0 * std::pow(kIref, (double)(p->K - 1))
                          : 0.0;
    const double* th = p->theta;
    ScreenCoef<T> c;
    c.inv_iref = (T)(1.0 / kIref);
    // -i (t0 + i t1) a = t1 a - i t0 a
    c.re_k = (T)(th[1] * aK);
    c.im_k = (T)(-th[0] * aK);
    c.re_p = (T)(th[3] * aP);
    c.im_p = (T)(-th[2] * aP);
    // (t4 + i t5) a
    c.re_a = (T)(th[4] * aA);
    c.im_a = (T)(th[5] * aA);
    c.K = p->K;
    c.active = (p->terms & (NLSE_KERR | NLSE_PLASMA | NLSE_MPA)) ? 1 : 0;
    c.has_gain = (c.re_k != (T)0 || c.re_p != (T)0 || c.re_a != (T)0) ? 1 : 0;
    c.real_gains = (c.re_k == (T)0 && c.re_p == (T)0 && c.im_a == (T)0) ? 1 : 0;
    c.reps = 1;
    c.scale = (T)1;
    c.exact = (p->scheme & NLSE_EXACT_SCREEN) ? 1 : 0;
    c.ka = (T)(-2.0 * (p->K - 1) * th[4] * aA);  // (K-1) c_A beta_K dz I_ref^(K-1)
    return c;
}

// Dithered rounding (fft.cuh, pass32.cuh): copy d of an FP32 table holds, for
// each component w of each entry, the FP32 neighbour of w above it when the
// fraction of an FP32 unit by which w exceeds its lower neighbour is above the
// copy's threshold, else the one below.  dsplit gives the two neighbours
// lo <= w <= hi and that fraction (0 when w is an FP32 value).
struct DSplit {
    float lo, hi;
    double frac;
};
DSplit dsplit(double w) {
    DSplit r;
    r.lo = (float)w;
    if ((double)r.lo > w) r.lo = std::nextafter(r.lo, -INFINITY);
    if ((double)r.lo == w) { r.hi = r.lo; r.frac = 0.0; return r; }
    r.hi = std::nextafter(r.lo, INFINITY);
    r.frac = (w - (double)r.lo) / ((double)r.hi - (double)r.lo);
    return r;
}
// fixed pseudo-random offset in [0, copies) of (table, entry, component)
int dither_offset(uint64_t table_id, uint64_t entry, int comp, int copies = kDither) {
    uint64_t z = table_id * 0x9E3779B97F4A7C15ull + entry * 2 + (uint64_t)comp + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (int)(z % (uint64_t)copies);
}
// identifiers of the dithered tables (distinct offsets per table)
enum : uint64_t {
    kTabTwiddle = 1, kTabPx = 2, kTabPy = 3, kTabRowPair = 4, kTabColPair = 5, kTabCross = 6, kTabRowPair8 = 7,
    kTabColPair8 = 8
};

// Threshold of copy d (of `copies`, a power of two) for an entry with offset
// o: the copies take the thresholds (q + 1/2) / copies in bit-reversed order
// of q = (d + o) mod copies, so that a run of consecutive steps rounds up and
// down in alternation (every partial sum of the rounding errors over a cycle
// stays within about one unit) instead of rounding the same way for half a
// cycle; over a whole cycle every threshold is used once, as before.
double dither_u(int d, int o, int copies = kDither) {
    const int q = (d + o) % copies;
    int r = 0;
    for (int b = 1, c = copies >> 1; b < copies; b <<= 1, c >>= 1)
        if (q & b) r |= c;
    return (r + 0.5) / copies;
}


// Twiddles of step k (0-based count of the steps taken before it): the start
// of twiddle block k mod kDither in FP32, the table itself in FP64.
template <typename T> const typename tab_of<T>::type* twiddles_at(const unsigned char* table, int n, int64_t k) {
    if (sizeof(T) == 4) table += (size_t)(k & (kDither - 1)) * tw32_copy_bytes(n);
    return reinterpret_cast<const typename tab_of<T>::type*>(table);
}
// twiddles of the one-off transforms (load prologue, readouts): copy 0
template <typename T> const typename tab_of<T>::type* twiddles_fixed(const unsigned char* table) {
    return reinterpret_cast<const typename tab_of<T>::type*>(table);
}
// copies of the propagator tables for step k
template <typename T> const typename tab_of<T>::type* px_at(const unsigned char* table, int n, int64_t k) {
    if (sizeof(T) == 4) table += (size_t)(k & (kDitherP - 1)) * n * 8;
    return reinterpret_cast<const typename tab_of<T>::type*>(table);
}
template <typename T> const typename tab_of<T>::type* py_at(const unsigned char* table, int n, int64_t k) {
    if (sizeof(T) == 4) table += (size_t)(k & (kDitherP - 1)) * py32_copy_bytes(n);
    return reinterpret_cast<const typename tab_of<T>::type*>(table);
}

void put_twiddle(std::vector<double>& out, size_t idx, long long m, long long period) {
    const double a = kTwoPi * (double)(m % period) / (double)period;
    out[2 * idx] = std::cos(a);
    out[2 * idx + 1] = -std::sin(a);
}
// FP64 pair table of an l-point transform of the pair engine (pair.cuh) with
// elements per thread e_max (16 or 8, at most l): per pass of stride ns > 1 and
// radix r = r1 r2, the entries W_{r1 ns}^{rA k} then W_{r ns}^{i kB}; angles
// reduced exactly in integers.
void pair_table(int l, int e_max, std::vector<double>& out) {
    const int e = std::min(e_max, l);
    out.assign(2 * (size_t)pr::pair_tab_entries(l, e), 0.0);
    size_t off = 0;
    for (int cur = 1; cur < l;) {
        const int r = std::min(e, l / cur);
        if (cur > 1) {
            const int r1 = pr::split1(r), r2 = pr::split2(r);
            for (int ra = 1; ra < r1; ++ra)
                for (int k = 0; k < cur; ++k) put_twiddle(out, off + (size_t)(ra - 1) * cur + k, (long long)ra * k, (long long)r1 * cur);
            off += (size_t)(r1 - 1) * cur;
            for (int i = 1; i < r2; ++i)
                for (int kb = 0; kb < r1 * cur; ++kb)
                    put_twiddle(out, off + (size_t)(i - 1) * r1 * cur + kb, (long long)i * kb, (long long)r * cur);
            off += (size_t)(r2 - 1) * r1 * cur;
        }
        cur *= r;
    }
}

// FP32 tables of one grid: kDither twiddle blocks (single-line table, row and
// column pair tables), P_x (kDitherP x n entries) and P_y with the cross-lane
// factors W_n^k (kDitherP x (n/2 pair entries (k, k + n/2), n/2 entries));
// every component of every entry dithered independently.  The cross-lane and propagator factors e^{i phi} are
// stored as (cos phi - 1, sin phi) (pass32.cuh), cos phi - 1 = -2 sin^2(phi/2)
// in FP64; P_y without its 1/n^2, which the kernel applies with P_x.
struct HostTables32 {
    std::vector<unsigned char> tw;
    std::vector<float> px, py;
};
void build_tables_f32(const nlse_params* p, HostTables32& t) {
    const int n = p->n, h = n / 2;
    std::vector<double> dp(2 * (size_t)n), single, cross(2 * (size_t)h);
    std::vector<double> pt[4];  // row E 16, row E 8, column E 16, column E 8
    for (int m = 0; m < n; ++m) {  // (cos phi - 1, sin phi) of P_x = P_y n^2
        const double ph = propagator_phase(p, m), sh = std::sin(0.5 * ph);
        dp[2 * m] = -2.0 * sh * sh;
        dp[2 * m + 1] = std::sin(ph);
    }
    twiddle_table(n, std::min(n, 16), single);
    pair_table(n, 16, pt[0]);
    pair_table(n, 8, pt[1]);
    pair_table(h, 16, pt[2]);
    pair_table(h, 8, pt[3]);
    for (int k = 0; k < h; ++k) {  // W_n^k = exp(-2 pi i k / n) as (cos - 1, sin)
        const double a = kTwoPi * (double)k / (double)n, sh = std::sin(0.5 * a);
        cross[2 * k] = -2.0 * sh * sh;
        cross[2 * k + 1] = -std::sin(a);
    }
    // the kDitherP thresholds in copy order for offset 0 (offset o: index d + o)
    std::vector<double> uq(2 * (size_t)kDitherP);
    for (int q = 0; q < 2 * kDitherP; ++q) uq[q] = dither_u(q % kDitherP, 0, kDitherP);
    auto dither_into = [&](double w, uint64_t table, uint64_t e, int c, float* dst, size_t stride) {
        const DSplit sp = dsplit(w);
        const int o = dither_offset(table, e, c, kDitherP);
        for (int d = 0; d < kDitherP; ++d) dst[(size_t)d * stride] = sp.frac > uq[d + o] ? sp.hi : sp.lo;
    };
    // P_x: kDitherP copies of n entries
    t.px.assign((size_t)kDitherP * 2 * n, 0.0f);
    for (int e = 0; e < n; ++e)
        for (int c = 0; c < 2; ++c) dither_into(dp[2 * e + c], kTabPx, e, c, t.px.data() + 2 * e + c, 2 * (size_t)n);
    // P_y pair entries and the cross-lane factors: kDitherP copies
    const size_t pyf = py32_copy_bytes(n) / 4;  // floats per copy
    t.py.assign((size_t)kDitherP * pyf, 0.0f);
    for (int k = 0; k < h; ++k)
        for (int c = 0; c < 2; ++c) {  // c = 0: cos - 1, 1: sin; lanes k and k + h
            dither_into(dp[2 * k + c], kTabPy, k, c, t.py.data() + 4 * k + 2 * c, pyf);
            dither_into(dp[2 * (k + h) + c], kTabPy, k + h, c, t.py.data() + 4 * k + 2 * c + 1, pyf);
            dither_into(cross[2 * k + c], kTabCross, k, c, t.py.data() + 4 * h + 2 * k + c, pyf);
        }
    // twiddle blocks: kDither copies (stride cb bytes)
    const size_t cb = tw32_copy_bytes(n), cbf = cb / 4;
    t.tw.assign((size_t)kDither * cb, 0);
    float* tw = reinterpret_cast<float*>(t.tw.data());
    for (size_t e = 0; e < single.size() / 2; ++e)
        for (int c = 0; c < 2; ++c) dither_into(single[2 * e + c], kTabTwiddle, e, c, tw + 2 * e + c, cbf);
    const uint64_t pid[4] = {kTabRowPair, kTabRowPair8, kTabColPair, kTabColPair8};
    const size_t poff[4] = {tw32_row_off(n, 16), tw32_row_off(n, 8), tw32_col_off(n, 16), tw32_col_off(n, 8)};
    for (int q = 0; q < 4; ++q)
        for (size_t e = 0; e < pt[q].size() / 2; ++e)
            for (int c = 0; c < 2; ++c) {
                if (q < 2) {  // row tables: (wx, wy)
                    dither_into(pt[q][2 * e + c], pid[q], e, c, tw + poff[q] / 4 + 2 * e + c, cbf);
                } else {      // column tables: (wx, wx, wy, wy)
                    float* f = tw + poff[q] / 4 + 4 * e + 2 * c;
                    dither_into(pt[q][2 * e + c], pid[q], e, c, f, cbf);
                    for (int d = 0; d < kDither; ++d) f[(size_t)d * cbf + 1] = f[(size_t)d * cbf];
                }
            }
}

}  // namespace


struct nlse_grid {
    nlse_params p;
    cudaStream_t stream;
    int device;
    unsigned char* ws;
    Layout lay;
    int64_t steps;
    int64_t hist_count;  // diagnostic steps finalised into the history ring
    int diag_pending;    // diagnostic steps recorded in the diag buffer, not yet finalised
    int loaded;
    int cols;  // column tile of the column pass
    int row_radix;  // radix of the row pass (FP32: 16 or 8)
    unsigned debug_extra_tx;  // test hook of the staged column pass (NLSE_DEBUG_COL_EXTRA_TX), 0 in use
    unsigned debug_row_extra_tx;  // test hook of the staged row pass (NLSE_DEBUG_ROW_EXTRA_TX), 0 in use
    double theta;  // accumulated global phase of the stored field, mod 2 pi
    const KernelSet<float>* k32;
    const KernelSet<double>* k64;
    ScreenCoef<float> sc32;
    ScreenCoef<double> sc64;
};

namespace {

inline nlse_status cuerr(cudaError_t e) { return e == cudaSuccess ? NLSE_OK : NLSE_ECUDA; }

template <typename T> struct Sel;
template <> struct Sel<float> {
    static const KernelSet<float>* ks(const nlse_grid* g) { return g->k32; }
    static const ScreenCoef<float>& sc(const nlse_grid* g) { return g->sc32; }
};
template <> struct Sel<double> {
    static const KernelSet<double>* ks(const nlse_grid* g) { return g->k64; }
    static const ScreenCoef<double>& sc(const nlse_grid* g) { return g->sc64; }
};

template <typename T> using VT = typename vec2<T>::type;
template <typename T> using WT = typename tab_of<T>::type;
template <typename T> const WT<T>* tab(nlse_grid* g, size_t off) {
    return reinterpret_cast<const WT<T>*>(g->ws + off);
}

template <typename T> VT<T>* at(nlse_grid* g, size_t off) { return reinterpret_cast<VT<T>*>(g->ws + off); }

// Global phase dither.  Eq. 1-3 are invariant under U -> U exp(i a), so each
// step may turn the whole field by a phase theta_s without changing the
// physics.  With theta_s = 2 pi frac(s (sqrt5 - 1)/2) (golden-ratio sequence)
// the spectral values, whose low-k part otherwise rotates by the same small
// angle every step, land at unrelated positions of the FP32 grid each step, so
// their rounding errors do not add up coherently.  The accumulated phase is
// kept here in FP64 and removed whenever the field is read out.
double step_phase(int64_t step) {
    return kTwoPi * std::fmod((double)step * 0.61803398874989484820, 1.0);
}
// Rotation factor of step k (0-based): exp(i theta_{k+1}) as the kernels
// apply it, and in *applied the angle it turns the field by.  In FP32 the
// factor is, among the FP32 pairs within 4 units of (cos, sin), the one whose
// squared modulus is closest to 1: a rounded factor would scale the power by
// 1 + O(2^-24) every step, a random walk over thousands of steps; the angle
// it applies instead is exact in FP64 and accumulated by the host.
template <typename T> WT<T> rot_for_step(int64_t k, double* applied);
template <> WT<double> rot_for_step<double>(int64_t k, double* applied) {
    const double th = step_phase(k + 1);
    if (applied) *applied = th;
    return make_double2(std::cos(th), std::sin(th));
}
template <> WT<float> rot_for_step<float>(int64_t k, double* applied) {
    const double th = step_phase(k + 1);
    const double c = std::cos(th), s = std::sin(th);
    float cs[9], ss[9];
    cs[4] = (float)c;
    ss[4] = (float)s;
    for (int i = 1; i <= 4; ++i) {
        cs[4 + i] = std::nextafter(cs[3 + i], INFINITY);
        cs[4 - i] = std::nextafter(cs[5 - i], -INFINITY);
        ss[4 + i] = std::nextafter(ss[3 + i], INFINITY);
        ss[4 - i] = std::nextafter(ss[5 - i], -INFINITY);
    }
    float bc = cs[4], bs = ss[4];
    double be = std::fabs((double)bc * bc + (double)bs * bs - 1.0);
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            const double e = std::fabs((double)cs[i] * cs[i] + (double)ss[j] * ss[j] - 1.0);
            if (e < be) { be = e; bc = cs[i]; bs = ss[j]; }
        }
    if (applied) *applied = std::atan2((double)bs, (double)bc);
    return make_float2(bc, bs);
}
template <typename V> V conj_of(V v) {
    v.y = -v.y;
    return v;
}
template <typename T> VT<T> unrot_value(double theta) {
    VT<T> v;
    v.x = (T)std::cos(theta);
    v.y = (T)(-std::sin(theta));
    return v;
}
inline double* dat(nlse_grid* g, size_t off) { return reinterpret_cast<double*>(g->ws + off); }

// per-block partials of a row pass of radix rad
template <typename T> int row_parts(const KernelSet<T>* ks, int rad) { return rad == 8 ? ks->row_blocks8 : ks->row_blocks; }

// Finalise the pending diagnostic steps into the history ring (one block per step).
template <typename T> nlse_status flush_diag(nlse_grid* g) {
    if (g->diag_pending == 0) return NLSE_OK;
    const double dx = g->p.L / g->p.n;
    k_finalize_batch<<<g->diag_pending, 256, 0, g->stream>>>(
        dat(g, g->lay.diag), row_parts(Sel<T>::ks(g), g->row_radix), dx * dx, dat(g, g->lay.hist),
        (long long)g->hist_count,
        kHistCap, reinterpret_cast<int*>(g->ws + g->lay.status));
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    g->hist_count += g->diag_pending;
    g->diag_pending = 0;
    return NLSE_OK;
}
nlse_status flush_diag_any(nlse_grid* g) {
    return g->p.precision == NLSE_FP64 ? flush_diag<double>(g) : flush_diag<float>(g);
}

// The march.  Lie: per step the column pass (diffraction) and the row pass
// (screen).  Strang: the screen coefficients are those of dz/2; a row pass
// with the screen alone opens the call (the first half screen), every step's
// row pass then applies its closing half screen, records the diagnostics and,
// except in the last step of the call, applies the opening half screen of the
// next step; so a call of m steps costs m + 1 row-pass sweeps and the state
// between calls is the field at a whole step, as in the Lie march.
template <typename T> nlse_status step_impl(nlse_grid* g, int nsteps, cudaEvent_t* ev = nullptr) {
    const KernelSet<T>* ks = Sel<T>::ks(g);
    VT<T>* field = at<T>(g, g->lay.state);
    const int n = g->p.n;
    double* partials = dat(g, g->lay.partials);
    const bool strang = (g->p.scheme & NLSE_STRANG) != 0;
    ScreenCoef<T> sc = Sel<T>::sc(g);
    for (int s = 0; s < nsteps; ++s) {
        if (ev && cudaEventRecord(ev[2 * s], g->stream) != cudaSuccess) return NLSE_ECUDA;
        const int64_t k = g->steps;
        if (strang && s == 0) {  // the opening half screen of the call: B_x S / n, screen, F_x
            sc.reps = 1;
            sc.scale = (T)1 / (T)n;
            if (ks->row_pass(field, field, twiddles_at<T>(g->ws + g->lay.tw, n, k), sc, partials, false,
                             g->row_radix, reinterpret_cast<int*>(g->ws + g->lay.status), g->debug_row_extra_tx,
                             g->stream) != cudaSuccess)
                return NLSE_ECUDA;
            sc.scale = (T)1;
        }
        const WT<T>* tw = twiddles_at<T>(g->ws + g->lay.tw, n, k);
        const WT<T>* px = px_at<T>(g->ws + g->lay.px, n, k);
        const WT<T>* py = py_at<T>(g->ws + g->lay.py, n, k);
        double th = 0.0;
        const WT<T> rot = rot_for_step<T>(k, &th);
        cudaError_t e = ks->col_pass(field, field, tw, px, py, rot, g->cols,
                                     reinterpret_cast<int*>(g->ws + g->lay.status), g->debug_extra_tx, g->stream);
        g->theta = std::fmod(g->theta + th, kTwoPi);
        if (e != cudaSuccess) return NLSE_ECUDA;
        if (ev && cudaEventRecord(ev[2 * s + 1], g->stream) != cudaSuccess) return NLSE_ECUDA;
        const bool diag = g->p.diag_every > 0 && ((g->steps + 1) % g->p.diag_every) == 0;
        // a diagnostic step leaves its per-block partials in the next slot of the
        // diag buffer; a full buffer is finalised into the history in one launch
        double* slot = dat(g, g->lay.diag) + 2 * (size_t)g->diag_pending * row_parts(ks, g->row_radix);
        sc.reps = strang && s + 1 < nsteps ? 2 : 1;
        e = ks->row_pass(field, field, tw, sc, diag ? slot : partials, diag, g->row_radix,
                         reinterpret_cast<int*>(g->ws + g->lay.status), g->debug_row_extra_tx, g->stream);
        if (e != cudaSuccess) return NLSE_ECUDA;
        if (diag && ++g->diag_pending == kDiagBatch && flush_diag<T>(g) != NLSE_OK) return NLSE_ECUDA;
        if (ev && cudaEventRecord(ev[2 * s + 2], g->stream) != cudaSuccess) return NLSE_ECUDA;
        ++g->steps;
    }
    return NLSE_OK;
}

// readout of the current field: optional field/fluence output; (power, peak)
// land in the readout slot
template <typename T> nlse_status readout_impl(nlse_grid* g, VT<T>* field_out, T* flu_out) {
    const KernelSet<T>* ks = Sel<T>::ks(g);
    double* partials = dat(g, g->lay.partials);
    cudaError_t e = ks->readout(at<T>(g, g->lay.state), twiddles_fixed<T>(g->ws + g->lay.tw), field_out, flu_out,
                                partials, unrot_value<T>(g->theta), g->stream);
    if (e != cudaSuccess) return NLSE_ECUDA;
    const double dx = g->p.L / g->p.n;
    k_finalize<<<1, 256, 0, g->stream>>>(partials, ks->row_blocks, dx * dx, dat(g, g->lay.readout),
                                         reinterpret_cast<int*>(g->ws + g->lay.status));
    return cuerr(cudaGetLastError());
}

nlse_status readout_any(nlse_grid* g, void* field_out, void* flu_out) {
    if (g->p.precision == NLSE_FP64)
        return readout_impl<double>(g, (double2*)field_out, (double*)flu_out);
    return readout_impl<float>(g, (float2*)field_out, (float*)flu_out);
}

nlse_status fetch_readout(nlse_grid* g, double out[2]) {
    cudaError_t e = cudaMemcpyAsync(out, g->ws + g->lay.readout, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, g->stream);
    if (e != cudaSuccess) return NLSE_ECUDA;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return NLSE_ECUDA;
    if (!std::isfinite(out[0]) || !std::isfinite(out[1])) return NLSE_ENONFINITE;
    return NLSE_OK;
}

template <typename T> nlse_status upload_tables(nlse_grid* g);
template <> nlse_status upload_tables<double>(nlse_grid* g) {
    std::vector<double> px, py, tw;
    propagator_tables(&g->p, px, py);
    // elements per thread of the FP64 kernels: 8 (at most n)
    twiddle_table(g->p.n, std::min(g->p.n, 8), tw);
    const size_t bytes = px.size() * sizeof(double);
    if (cudaMemcpyAsync(g->ws + g->lay.px, px.data(), bytes, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->ws + g->lay.py, py.data(), bytes, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->ws + g->lay.tw, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice,
                        g->stream) != cudaSuccess)
        return NLSE_ECUDA;
    // the host vectors die at return: make the copies complete first
    return cuerr(cudaStreamSynchronize(g->stream));
}
template <> nlse_status upload_tables<float>(nlse_grid* g) {
    HostTables32 t;
    build_tables_f32(&g->p, t);
    if (cudaMemcpyAsync(g->ws + g->lay.px, t.px.data(), t.px.size() * sizeof(float), cudaMemcpyHostToDevice,
                        g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->ws + g->lay.py, t.py.data(), t.py.size() * sizeof(float), cudaMemcpyHostToDevice,
                        g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->ws + g->lay.tw, t.tw.data(), t.tw.size(), cudaMemcpyHostToDevice, g->stream) !=
            cudaSuccess)
        return NLSE_ECUDA;
    return cuerr(cudaStreamSynchronize(g->stream));
}

}  // namespace

namespace nlse {
namespace detail {

nlse_status upload_tables_f32(const nlse_params* p, cudaStream_t s, unsigned char* px, unsigned char* py,
                              unsigned char* tw) {
    HostTables32 t;
    build_tables_f32(p, t);
    if (cudaMemcpyAsync(px, t.px.data(), t.px.size() * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(py, t.py.data(), t.py.size() * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return NLSE_ECUDA;
    if (tw && cudaMemcpyAsync(tw, t.tw.data(), t.tw.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return NLSE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}

ScreenCoef<float> screen_coef_f32(const nlse_params* p) { return screen_coef<float>(p); }

float2 rot_step_f32(long long k, double* applied) { return ::rot_for_step<float>(k, applied); }


cudaError_t finalize(const double* partials, int nparts, double scale, double* out, int* status,
                     cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(partials, nparts, scale, out, status);
    return cudaGetLastError();
}

}  // namespace detail
}  // namespace nlse

// ------------------------------------------------------------------ C ABI --

namespace {

// scratch of the effective lens: counters, the separable low-pass factors,
// complex work array (w, its spectrum, w_dif), labels, per-root maximum keys
// (then the centre list), per-root centres
struct LensScratch {
    size_t ctr, tab, wbuf, lab, key, cen, total;
};

LensScratch lens_scratch_layout(int n, int precision) {
    const size_t nn = (size_t)n * n;
    LensScratch L;
    size_t o = 0;
    L.ctr = o;  o = align256(o + 2 * sizeof(int));
    L.tab = o;  o = align256(o + 2 * (size_t)n * sizeof(double));
    L.wbuf = o; o = align256(o + nn * (precision == NLSE_FP64 ? 16 : 8));
    L.lab = o;  o = align256(o + nn * sizeof(int));
    L.key = o;  o = align256(o + nn * sizeof(unsigned long long));
    L.cen = o;  o = align256(o + nn * sizeof(int));
    L.total = o;
    return L;
}

bool lens_part_ok(int count, const double* r, const double* amp, const double* freq, const double* phase) {
    if (count < 0 || count > NLSE_LENS_SEGMENTS) return false;
    double prev = 0.0;
    for (int j = 0; j < count; ++j) {
        if (!std::isfinite(r[j]) || !(r[j] > prev)) return false;
        if (!std::isfinite(amp[j]) || !std::isfinite(freq[j]) || !std::isfinite(phase[j])) return false;
        prev = r[j];
    }
    return true;
}

template <typename T>
nlse_status lens_impl(nlse_grid* g, const nlse_lens* ls, unsigned char* sc, int32_t* count, int32_t* centres,
                      int32_t capacity, T* w_dif_out) {
    using V = VT<T>;
    const KernelSet<T>* ks = Sel<T>::ks(g);
    const int n = g->p.n;
    const size_t nn = (size_t)n * n;
    const LensScratch SL = lens_scratch_layout(n, g->p.precision);
    int* ctr = reinterpret_cast<int*>(sc + SL.ctr);
    V* wbuf = reinterpret_cast<V*>(sc + SL.wbuf);
    int* lab = reinterpret_cast<int*>(sc + SL.lab);
    unsigned long long* key = reinterpret_cast<unsigned long long*>(sc + SL.key);
    int* cen = reinterpret_cast<int*>(sc + SL.cen);
    int* list = reinterpret_cast<int*>(sc + SL.key);  // the keys are done with when the list is gathered
    V* field = at<T>(g, g->lay.aux);
    const auto* tw = twiddles_fixed<T>(g->ws + g->lay.tw);
    cudaStream_t st = g->stream;
    const int blocks = (int)std::min<size_t>((nn + 255) / 256, 152 * 8);

    // the field leaves the state for the scratch half of the grid (row-major,
    // global phase removed) and comes back after the screen
    nlse_status s = readout_any(g, field, nullptr);
    if (s != NLSE_OK) return s;
    if (cudaMemsetAsync(ctr, 0, 2 * sizeof(int), st) != cudaSuccess) return NLSE_ECUDA;
    k_lens_fluence<T><<<blocks, 256, 0, st>>>(field, wbuf, nn);
    // separable low-pass factors: fx[p] = exp(-l_dif kx_p^2), fy[q] = exp(-l_dif ky_q^2) / n^2
    std::vector<T> htab(2 * (size_t)n);
    const double kunit = kTwoPi / g->p.L;
    for (int m = 0; m < n; ++m) {
        const double k = kunit * (m < n / 2 ? m : m - n);
        const double f = std::exp(-ls->l_dif * k * k);
        htab[m] = (T)f;
        htab[n + m] = (T)(f / ((double)n * n));
    }
    T* tab = reinterpret_cast<T*>(sc + SL.tab);
    if (cudaMemcpyAsync(tab, htab.data(), htab.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return NLSE_ECUDA;
    cudaError_t e = ks->dft2(wbuf, tw, false, st);
    if (e != cudaSuccess) return NLSE_ECUDA;
    k_lens_filter<T><<<blocks, 256, 0, st>>>(wbuf, n, tab, tab + n);
    e = ks->dft2(wbuf, tw, true, st);
    if (e != cudaSuccess) return NLSE_ECUDA;

    // lenses: regions of Re(wbuf) >= w_l, labelled by their smallest index
    const int rt = n < 256 ? n : 256;
    k_hot_runs<T><<<n, rt, 0, st>>>(reinterpret_cast<const T*>(wbuf), n, 2, (T)ls->w_l, lab);
    k_hot_merge<<<blocks, 256, 0, st>>>(lab, n, ls->connectivity, ctr + 1);
    k_hot_roots<<<blocks, 256, 0, st>>>(lab, n, ctr);
    k_hot_spread<<<blocks, 256, 0, st>>>(lab, (int)nn);
    // centres: per lens the smallest index of its largest value
    if (cudaMemsetAsync(key, 0, nn * sizeof(unsigned long long), st) != cudaSuccess) return NLSE_ECUDA;
    if (cudaMemsetAsync(cen, 0x7f, nn * sizeof(int), st) != cudaSuccess) return NLSE_ECUDA;
    k_lens_keymax<T><<<blocks, 256, 0, st>>>(wbuf, lab, key, nn);
    k_lens_argmax<T><<<blocks, 256, 0, st>>>(wbuf, lab, key, cen, nn);
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    int hc[2] = {0, 0};
    if (cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st) != cudaSuccess) return NLSE_ECUDA;
    if (cudaMemsetAsync(ctr, 0, sizeof(int), st) != cudaSuccess) return NLSE_ECUDA;
    k_lens_gather<<<blocks, 256, 0, st>>>(lab, cen, list, ctr, nn);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return NLSE_ECUDA;
    if (hc[1] & kHotStatusGaveUp) return NLSE_ETIMEOUT;
    const int nl = hc[0];
    // the list in increasing index order: the order the screen sums the lenses in
    std::vector<int32_t> hl((size_t)nl);
    if (nl > 0) {
        if (cudaMemcpyAsync(hl.data(), list, (size_t)nl * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return NLSE_ECUDA;
        std::sort(hl.begin(), hl.end());
        if (cudaMemcpyAsync(list, hl.data(), (size_t)nl * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return NLSE_ECUDA;
    }
    if (w_dif_out) k_lens_real<T><<<blocks, 256, 0, st>>>(wbuf, w_dif_out, nn);

    // Eqs. 5-6 and the screen of Eq. 2
    const double dx = g->p.L / n;
    LensCoef c;
    c.n_re = ls->n_re;
    c.n_im = ls->n_im;
    double reach = 0.0;
    for (int j = 0; j < kLensSeg; ++j) {
        c.r_re[j] = ls->r_re[j]; c.a[j] = ls->a[j]; c.omega[j] = ls->omega[j]; c.psi[j] = ls->psi[j];
        c.r_im[j] = ls->r_im[j]; c.b[j] = ls->b[j]; c.nu[j] = ls->nu[j]; c.eta[j] = ls->eta[j];
    }
    if (ls->n_re > 0) reach = std::max(reach, ls->r_re[ls->n_re - 1]);
    if (ls->n_im > 0) reach = std::max(reach, ls->r_im[ls->n_im - 1]);
    c.reach2 = (reach / dx + 1.0) * (reach / dx + 1.0);
    if (nl > 0 && (ls->n_re > 0 || ls->n_im > 0)) {
        const int ts = n < 16 ? n : 16;
        k_lens_apply<T><<<dim3(n / ts, n / ts), dim3(ts, ts), 0, st>>>(field, n, dx, list, nl, c);
    }
    e = ks->row_forward(field, at<T>(g, g->lay.state), tw, st);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    g->theta = 0.0;  // the readout removed the accumulated global phase
    if (cudaStreamSynchronize(st) != cudaSuccess) return NLSE_ECUDA;
    *count = nl;
    if (centres)
        for (int i = 0; i < nl && i < capacity; ++i) centres[i] = hl[(size_t)i];
    return NLSE_OK;
}

}  // namespace

extern "C" {

const char* nlse_status_string(nlse_status s) {
    switch (s) {
        case NLSE_OK: return "NLSE_OK";
        case NLSE_EINVAL: return "NLSE_EINVAL: invalid argument";
        case NLSE_EUNSUPPORTED: return "NLSE_EUNSUPPORTED: unsupported size or precision";
        case NLSE_ENOMEM: return "NLSE_ENOMEM: workspace too small";
        case NLSE_ECUDA: return "NLSE_ECUDA: CUDA error";
        case NLSE_ENONFINITE: return "NLSE_ENONFINITE: non-finite value in the field";
        case NLSE_ETIMEOUT: return "NLSE_ETIMEOUT: device-side wait timed out";
        case NLSE_ESTATE: return "NLSE_ESTATE: call out of order";
    }
    return "NLSE: unknown status";
}

int32_t nlse_version(void) { return 10000; }

nlse_status nlse_workspace_size(const nlse_params* p, size_t* bytes) {
    if (!bytes) return NLSE_EINVAL;
    nlse_status st = validate(p);
    if (st != NLSE_OK) return st;
    *bytes = layout_for(p->n, p->precision).total;
    return NLSE_OK;
}

nlse_status nlse_create(const nlse_params* p, void* cuda_stream, void* dev_workspace,
                        size_t workspace_bytes, nlse_grid** out) {
    if (!out || !dev_workspace) return NLSE_EINVAL;
    *out = nullptr;
    nlse_status st = validate(p);
    if (st != NLSE_OK) return st;
    if (reinterpret_cast<uintptr_t>(dev_workspace) & 255) return NLSE_EINVAL;
    Layout lay = layout_for(p->n, p->precision);
    if (workspace_bytes < lay.total) return NLSE_ENOMEM;
    nlse_grid* g = new (std::nothrow) nlse_grid();
    if (!g) return NLSE_ENOMEM;
    g->p = *p;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    g->ws = static_cast<unsigned char*>(dev_workspace);
    g->lay = lay;
    const int k = log2_exact(p->n);
    if (cudaGetDevice(&g->device) != cudaSuccess) { delete g; return NLSE_ECUDA; }
    nlse_params screen_p = *p;  // the screen of one Lie step, or half of a symmetric step
    if (p->scheme & NLSE_STRANG) screen_p.dz = 0.5 * p->dz;
    if (p->precision == NLSE_FP64) {
        g->k64 = kernels_f64(k);
        g->cols = g->k64->col_default;
        g->row_radix = g->k64->row_radix_default;
        g->sc64 = screen_coef<double>(&screen_p);
    } else {
        g->k32 = kernels_f32(k);
        g->cols = g->k32->col_default;
        g->row_radix = g->k32->row_radix_default;
        g->sc32 = screen_coef<float>(&screen_p);
    }
    if (const char* env = std::getenv("NLSE_DEBUG_COL_EXTRA_TX")) g->debug_extra_tx = (unsigned)std::atoi(env);
    if (const char* env = std::getenv("NLSE_DEBUG_ROW_EXTRA_TX")) g->debug_row_extra_tx = (unsigned)std::atoi(env);
    if (const char* env = std::getenv("NLSE_COL_TILE")) {
        const int c = std::atoi(env);
        const int mask = p->precision == NLSE_FP64 ? g->k64->col_mask : g->k32->col_mask;
        for (int i = 0; i < kColOptionCount; ++i)
            if (kColOptions[i] == c && ((mask >> i) & 1)) g->cols = c;
    }
    st = p->precision == NLSE_FP64 ? upload_tables<double>(g) : upload_tables<float>(g);
    if (st == NLSE_OK)
        st = cuerr(cudaMemsetAsync(g->ws + lay.status, 0, sizeof(int), g->stream));
    if (st != NLSE_OK) { delete g; return st; }
    *out = g;
    return NLSE_OK;
}

nlse_status nlse_load_field(nlse_grid* g, const void* src, int src_on_device) {
    if (!g || !src) return NLSE_EINVAL;
    const size_t cs = g->p.precision == NLSE_FP64 ? 16 : 8;
    const size_t bytes = (size_t)g->p.n * g->p.n * cs;
    void* state = g->ws + g->lay.state;
    // the forward row transform reads the row-major field (the caller's device
    // buffer, or the host field staged in the scratch buffer) and writes the
    // state, whose layout differs: never in place
    const void* rows = src;
    cudaError_t e = cudaSuccess;
    if (!src_on_device) {
        rows = g->ws + g->lay.aux;
        e = cudaMemcpyAsync(g->ws + g->lay.aux, src, bytes, cudaMemcpyHostToDevice, g->stream);
    }
    if (e == cudaSuccess) {
        if (g->p.precision == NLSE_FP64)
            e = g->k64->row_forward((const double2*)rows, (double2*)state, twiddles_fixed<double>(g->ws + g->lay.tw),
                                    g->stream);
        else
            e = g->k32->row_forward((const float2*)rows, (float2*)state, twiddles_fixed<float>(g->ws + g->lay.tw),
                                    g->stream);
    }
    if (e != cudaSuccess) return NLSE_ECUDA;
    g->steps = 0;
    g->hist_count = 0;
    g->diag_pending = 0;
    g->theta = 0.0;
    g->loaded = 1;
    return NLSE_OK;
}

nlse_status nlse_step(nlse_grid* g, int32_t nsteps) {
    if (!g || nsteps < 0) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    return g->p.precision == NLSE_FP64 ? step_impl<double>(g, nsteps) : step_impl<float>(g, nsteps);
}

nlse_status nlse_step_timed(nlse_grid* g, int32_t nsteps, double* col_ms, double* row_ms) {
    if (!g || nsteps < 0) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    std::vector<cudaEvent_t> ev(2 * (size_t)nsteps + 1, nullptr);
    nlse_status st = NLSE_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; st = NLSE_ECUDA; break; }
    if (st == NLSE_OK)
        st = g->p.precision == NLSE_FP64 ? step_impl<double>(g, nsteps, ev.data())
                                         : step_impl<float>(g, nsteps, ev.data());
    double c = 0.0, r = 0.0;
    if (st == NLSE_OK && nsteps > 0) {
        if (cudaEventSynchronize(ev[2 * (size_t)nsteps]) != cudaSuccess) st = NLSE_ECUDA;
        for (int s = 0; st == NLSE_OK && s < nsteps; ++s) {
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, ev[2 * s], ev[2 * s + 1]) != cudaSuccess ||
                cudaEventElapsedTime(&b, ev[2 * s + 1], ev[2 * s + 2]) != cudaSuccess)
                st = NLSE_ECUDA;
            c += a;
            r += b;
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (st == NLSE_OK) {
        if (col_ms) *col_ms += c;
        if (row_ms) *row_ms += r;
    }
    return st;
}

nlse_status nlse_set_column_tile(nlse_grid* g, int32_t cols) {
    if (!g) return NLSE_EINVAL;
    const int mask = g->p.precision == NLSE_FP64 ? g->k64->col_mask : g->k32->col_mask;
    for (int i = 0; i < kColOptionCount; ++i)
        if (kColOptions[i] == cols && ((mask >> i) & 1)) {
            g->cols = cols;
            return NLSE_OK;
        }
    return NLSE_EUNSUPPORTED;
}

nlse_status nlse_set_row_radix(nlse_grid* g, int32_t radix) {
    if (!g) return NLSE_EINVAL;
    const int mask = g->p.precision == NLSE_FP64 ? g->k64->row_radix_mask : g->k32->row_radix_mask;
    const int bit = radix == 16 ? 1 : radix == 8 ? 2 : radix == (kRowStaged | 16) ? 4 : 0;
    if (!(mask & bit)) return NLSE_EUNSUPPORTED;
    // recorded partials carry the block count of the radix they were made with
    if (flush_diag_any(g) != NLSE_OK) return NLSE_ECUDA;
    g->row_radix = radix;
    return NLSE_OK;
}

nlse_status nlse_steps_taken(nlse_grid* g, int64_t* steps) {
    if (!g || !steps) return NLSE_EINVAL;
    *steps = g->steps;
    return NLSE_OK;
}

nlse_status nlse_power(nlse_grid* g, double* watts) {
    if (!g || !watts) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    nlse_status st = readout_any(g, nullptr, nullptr);
    if (st != NLSE_OK) return st;
    double r[2];
    st = fetch_readout(g, r);
    *watts = r[0];
    return st;
}

nlse_status nlse_peak(nlse_grid* g, double* w_per_cm2) {
    if (!g || !w_per_cm2) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    nlse_status st = readout_any(g, nullptr, nullptr);
    if (st != NLSE_OK) return st;
    double r[2];
    st = fetch_readout(g, r);
    *w_per_cm2 = r[1];
    return st;
}

nlse_status nlse_fluence(nlse_grid* g, void* dst, int dst_on_device, int downsample) {
    if (!g || !dst) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    const int n = g->p.n;
    if (downsample < 1 || (downsample & (downsample - 1)) || downsample > n) return NLSE_EINVAL;
    const bool f64 = g->p.precision == NLSE_FP64;
    const size_t rs = f64 ? 8 : 4;
    unsigned char* flu = g->ws + g->lay.aux;          // n^2 reals
    unsigned char* box = flu + (size_t)n * n * rs;    // (n/ds)^2 reals (second half of aux)
    const bool direct = dst_on_device && downsample == 1;
    nlse_status st = readout_any(g, nullptr, direct ? dst : flu);
    if (st != NLSE_OK) return st;
    const int m = n / downsample;
    const size_t out_bytes = (size_t)m * m * rs;
    if (downsample > 1) {
        void* target = dst_on_device ? dst : box;
        const int blocks = (int)(((size_t)m * m + 255) / 256) < 4096 ? (int)(((size_t)m * m + 255) / 256) : 4096;
        if (f64) k_box_mean<double><<<blocks, 256, 0, g->stream>>>((const double*)flu, (double*)target, n, downsample);
        else k_box_mean<float><<<blocks, 256, 0, g->stream>>>((const float*)flu, (float*)target, n, downsample);
        if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
        if (!dst_on_device) {
            if (cudaMemcpyAsync(dst, box, out_bytes, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
                return NLSE_ECUDA;
            return cuerr(cudaStreamSynchronize(g->stream));
        }
        return NLSE_OK;
    }
    if (!dst_on_device) {
        if (cudaMemcpyAsync(dst, flu, out_bytes, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
            return NLSE_ECUDA;
        return cuerr(cudaStreamSynchronize(g->stream));
    }
    return NLSE_OK;
}

nlse_status nlse_read_field(nlse_grid* g, void* dst, int dst_on_device) {
    if (!g || !dst) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    const size_t cs = g->p.precision == NLSE_FP64 ? 16 : 8;
    const size_t bytes = (size_t)g->p.n * g->p.n * cs;
    void* target = dst_on_device ? dst : (void*)(g->ws + g->lay.aux);
    nlse_status st = readout_any(g, target, nullptr);
    if (st != NLSE_OK) return st;
    if (!dst_on_device) {
        if (cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
            return NLSE_ECUDA;
        return cuerr(cudaStreamSynchronize(g->stream));
    }
    return NLSE_OK;
}

nlse_status nlse_hot_areas(nlse_grid* g, double w_p, int32_t connectivity, int32_t* count, int32_t* labels,
                           int labels_on_device) {
    if (!g || !count || !std::isfinite(w_p) || (connectivity != 4 && connectivity != 8)) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    const int n = g->p.n;
    const int nn = n * n;
    const bool f64 = g->p.precision == NLSE_FP64;
    unsigned char* flu = g->ws + g->lay.aux;  // n^2 reals; the labels use the second half of aux
    int* lab = labels && labels_on_device ? labels : reinterpret_cast<int*>(flu + (size_t)nn * (f64 ? 8 : 4));
    nlse_status st = readout_any(g, nullptr, flu);
    if (st != NLSE_OK) return st;
    // the readout's finalisation has consumed the partials: they hold {count, status} now
    int* word = reinterpret_cast<int*>(dat(g, g->lay.partials));
    if (cudaMemsetAsync(word, 0, 2 * sizeof(int), g->stream) != cudaSuccess) return NLSE_ECUDA;
    const int rt = n < 256 ? n : 256;
    if (f64) k_hot_runs<double><<<n, rt, 0, g->stream>>>((const double*)flu, n, 1, w_p, lab);
    else k_hot_runs<float><<<n, rt, 0, g->stream>>>((const float*)flu, n, 1, (float)w_p, lab);
    const int blocks = std::min((nn + 255) / 256, 152 * 8);
    k_hot_merge<<<blocks, 256, 0, g->stream>>>(lab, n, connectivity, word + 1);
    k_hot_roots<<<blocks, 256, 0, g->stream>>>(lab, n, word);
    k_hot_spread<<<blocks, 256, 0, g->stream>>>(lab, nn);
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    int host_word[2] = {0, 0};
    if (cudaMemcpyAsync(host_word, word, sizeof(host_word), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        return NLSE_ECUDA;
    if (labels && !labels_on_device &&
        cudaMemcpyAsync(labels, lab, (size_t)nn * sizeof(int), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        return NLSE_ECUDA;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return NLSE_ECUDA;
    if (host_word[1] & kHotStatusGaveUp) return NLSE_ETIMEOUT;
    *count = host_word[0];
    return NLSE_OK;
}

nlse_status nlse_turbulent_screen(nlse_grid* g, const void* xi, int xi_on_device, double tau, double k_h,
                                  double thickness) {
    if (!g || !xi || !std::isfinite(tau) || !std::isfinite(k_h) || !(k_h >= 0.0) || !std::isfinite(thickness))
        return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    const int n = g->p.n;
    const bool f64 = g->p.precision == NLSE_FP64;
    const size_t nn = (size_t)n * n;
    const size_t bytes = nn * (f64 ? 16 : 8);
    unsigned char* field = g->ws + g->lay.aux;
    unsigned char* spec = g->ws + g->lay.state;
    // the field leaves the state for the scratch buffer (row-major, global
    // phase removed); the state buffer then holds the screen while it is built
    nlse_status st = readout_any(g, field, nullptr);
    if (st != NLSE_OK) return st;
    const void* src = xi;
    if (!xi_on_device) {
        if (cudaMemcpyAsync(spec, xi, bytes, cudaMemcpyHostToDevice, g->stream) != cudaSuccess) return NLSE_ECUDA;
        src = spec;
    }
    const double rc = k_h * g->p.L / kTwoPi;
    const double r2 = rc * rc;
    // largest integer p~^2 + q~^2 inside the cut-off (none above 2 (n/2)^2)
    const long long m2max = r2 >= 2.0 * (double)(n / 2) * (n / 2) ? 2LL * (n / 2) * (n / 2) : (long long)std::floor(r2);
    const double c = thickness / (2.0 * (kTwoPi * g->p.n0 / g->p.lambda0));
    const int blocks = (int)std::min<size_t>((nn + 255) / 256, 152 * 8);
    cudaError_t e;
    if (f64) {
        k_turb_spectrum<double><<<blocks, 256, 0, g->stream>>>((const double2*)src, (double2*)spec, n, tau, m2max);
        e = g->k64->dft2((double2*)spec, twiddles_fixed<double>(g->ws + g->lay.tw), true, g->stream);
        if (e == cudaSuccess) {
            k_turb_apply<double><<<blocks, 256, 0, g->stream>>>((double2*)field, (const double2*)spec, c, nn);
            e = g->k64->row_forward((const double2*)field, (double2*)spec, twiddles_fixed<double>(g->ws + g->lay.tw),
                                    g->stream);
        }
    } else {
        k_turb_spectrum<float><<<blocks, 256, 0, g->stream>>>((const float2*)src, (float2*)spec, n, (float)tau, m2max);
        e = g->k32->dft2((float2*)spec, twiddles_fixed<float>(g->ws + g->lay.tw), true, g->stream);
        if (e == cudaSuccess) {
            k_turb_apply<float><<<blocks, 256, 0, g->stream>>>((float2*)field, (const float2*)spec, (float)c, nn);
            e = g->k32->row_forward((const float2*)field, (float2*)spec, twiddles_fixed<float>(g->ws + g->lay.tw),
                                    g->stream);
        }
    }
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    g->theta = 0.0;  // the readout removed the accumulated global phase
    return NLSE_OK;
}


nlse_status nlse_lens_scratch_size(const nlse_params* p, size_t* bytes) {
    if (!bytes) return NLSE_EINVAL;
    nlse_status s = validate(p);
    if (s != NLSE_OK) return s;
    *bytes = lens_scratch_layout(p->n, p->precision).total;
    return NLSE_OK;
}

nlse_status nlse_effective_lens(nlse_grid* g, const nlse_lens* lens, void* scratch, size_t scratch_bytes,
                                int32_t* count, int32_t* centres, int32_t capacity, void* w_dif_out) {
    if (!g || !lens || !scratch || !count || (centres && capacity < 0)) return NLSE_EINVAL;
    if (reinterpret_cast<uintptr_t>(scratch) & 255) return NLSE_EINVAL;
    if (!std::isfinite(lens->l_dif) || lens->l_dif < 0.0 || !std::isfinite(lens->w_l) || !(lens->w_l > 0.0))
        return NLSE_EINVAL;
    if ((lens->connectivity != 4 && lens->connectivity != 8) || lens->reserved != 0) return NLSE_EINVAL;
    if (!lens_part_ok(lens->n_re, lens->r_re, lens->a, lens->omega, lens->psi) ||
        !lens_part_ok(lens->n_im, lens->r_im, lens->b, lens->nu, lens->eta))
        return NLSE_EINVAL;
    if (scratch_bytes < lens_scratch_layout(g->p.n, g->p.precision).total) return NLSE_ENOMEM;
    if (!g->loaded) return NLSE_ESTATE;
    unsigned char* sc = static_cast<unsigned char*>(scratch);
    if (g->p.precision == NLSE_FP64)
        return lens_impl<double>(g, lens, sc, count, centres, capacity, static_cast<double*>(w_dif_out));
    return lens_impl<float>(g, lens, sc, count, centres, capacity, static_cast<float*>(w_dif_out));
}

nlse_status nlse_moments(nlse_grid* g, int32_t count, const int32_t* p, const int32_t* q, double* out) {
    if (!g || !p || !q || !out || count < 1 || count > kMomMax) return NLSE_EINVAL;
    for (int k = 0; k < count; ++k)
        if (p[k] < 1 || p[k] > 16 || q[k] < 0 || q[k] > 16) return NLSE_EINVAL;
    if (!g->loaded) return NLSE_ESTATE;
    // the per-block partials use the diagnostic slots: finalise pending records first
    if (flush_diag_any(g) != NLSE_OK) return NLSE_ECUDA;
    const int n = g->p.n;
    const size_t nn = (size_t)n * n;
    const bool f64 = g->p.precision == NLSE_FP64;
    unsigned char* flu = g->ws + g->lay.aux;
    nlse_status st = readout_any(g, nullptr, flu);
    if (st != NLSE_OK) return st;
    MomentSpec ms;
    ms.count = count;
    for (int k = 0; k < kMomMax; ++k) {
        ms.p[k] = k < count ? p[k] : 1;
        ms.q[k] = k < count ? q[k] : 0;
    }
    const int blocks = (int)std::min<size_t>((nn + 255) / 256, 152 * 4);
    double* part = dat(g, g->lay.diag);
    const double dx = g->p.L / n;
    if (f64) k_moments<double><<<blocks, 256, 0, g->stream>>>((const double*)flu, n, dx, ms, part);
    else k_moments<float><<<blocks, 256, 0, g->stream>>>((const float*)flu, n, dx, ms, part);
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    std::vector<double> h((size_t)blocks * kMomMax);
    if (cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, g->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
        return NLSE_ECUDA;
    for (int k = 0; k < count; ++k) {
        double s = 0.0;
        for (int b = 0; b < blocks; ++b) s += h[(size_t)b * kMomMax + k];
        out[k] = s * dx * dx;
    }
    return NLSE_OK;
}

nlse_status nlse_history(nlse_grid* g, double* power, double* peak, int32_t capacity, int32_t* count) {
    if (!g || !count || capacity < 0) return NLSE_EINVAL;
    if (flush_diag_any(g) != NLSE_OK) return NLSE_ECUDA;
    const int64_t have = g->hist_count < kHistCap ? g->hist_count : kHistCap;
    const int64_t first = g->hist_count - have;
    std::vector<double> buf(2 * (size_t)kHistCap);
    if (have > 0) {
        if (cudaMemcpyAsync(buf.data(), g->ws + g->lay.hist, buf.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
            return NLSE_ECUDA;
        if (cudaStreamSynchronize(g->stream) != cudaSuccess) return NLSE_ECUDA;
    }
    const int64_t ncopy = have < capacity ? have : capacity;
    for (int64_t i = 0; i < ncopy; ++i) {
        const int64_t slot = (first + i) % kHistCap;
        if (power) power[i] = buf[2 * slot];
        if (peak) peak[i] = buf[2 * slot + 1];
    }
    *count = (int32_t)ncopy;
    return NLSE_OK;
}

nlse_status nlse_device_status(nlse_grid* g) {
    if (!g) return NLSE_EINVAL;
    int word = 0;
    if (cudaMemcpyAsync(&word, g->ws + g->lay.status, sizeof(int), cudaMemcpyDeviceToHost, g->stream) !=
        cudaSuccess)
        return NLSE_ECUDA;
    if (cudaMemsetAsync(g->ws + g->lay.status, 0, sizeof(int), g->stream) != cudaSuccess) return NLSE_ECUDA;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return NLSE_ECUDA;
    if (word & 6) return NLSE_ETIMEOUT;
    if (word & 1) return NLSE_ENONFINITE;
    return NLSE_OK;
}

nlse_status nlse_destroy(nlse_grid* g) {
    if (!g) return NLSE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    delete g;
    return cuerr(e);
}

}  // extern "C"

// ================================================================ adjoint ==
// Reverse-mode gradient of J = sum (|U_M|^2 - D)^2 / sum D^2 after M steps
// (kernels in adjoint.cuh).  The forward run stores the x-spectral state S
// every `ckpt` steps; the backward sweep recomputes each segment from its
// checkpoint, keeping the column-pass outputs T_n of the segment, and then
// runs the backward row and column passes from the last step of the segment
// to its first.  All kernels are deterministic, so the recomputed states are
// bit-identical to the forward ones.

namespace {

struct AdjLayout {
    size_t state, gam, tw, px, py, pxc, pyc, seg, ckpt, target, partials, acc, result, total;
    int nck;
};

AdjLayout adj_layout_for(int n, int precision, int nsteps, int ckpt) {
    const size_t cs = precision == NLSE_FP64 ? 16 : 8;
    const size_t field = (size_t)n * n * cs;
    AdjLayout L;
    L.nck = (nsteps + ckpt - 1) / ckpt;
    if (L.nck < 1) L.nck = 1;
    size_t o = 0;
    L.state = o;    o = align256(o + field);
    L.gam = o;      o = align256(o + field);
    L.tw = o;       o = align256(o + tw_region_bytes(n, precision));
    L.px = o;       o = align256(o + px_bytes(n, precision));
    L.py = o;       o = align256(o + py_bytes(n, precision));
    L.pxc = o;      o = align256(o + px_bytes(n, precision));
    L.pyc = o;      o = align256(o + py_bytes(n, precision));
    L.seg = o;      o = align256(o + field * (size_t)ckpt);
    L.ckpt = o;     o = align256(o + field * (size_t)L.nck);
    L.target = o;   o = align256(o + (size_t)n * n * sizeof(double));
    L.partials = o; o = align256(o + (size_t)n * 2 * sizeof(double));
    L.acc = o;      o = align256(o + (size_t)n * 6 * sizeof(double));
    L.result = o;   o = align256(o + 4 * sizeof(double) + sizeof(int));
    L.total = o;
    return L;
}

template <typename T> AdjCoef<T> adj_coef(const nlse_params* p) {
    AdjCoef<T> a;
    a.sc = screen_coef<T>(p);
    const double k0 = kTwoPi * p->n0 / p->lambda0;
    const double eps_k = 2.0 * k0 * k0 * p->n2 / p->n0;
    const double eps_m = -k0 * k0 * p->sigmaK * p->rho_nt * p->tau_pl / p->rho_c;
    a.aK = (T)((p->terms & NLSE_KERR) ? p->dz * eps_k / (2.0 * k0) * kIref : 0.0);
    a.aP = (T)((p->terms & NLSE_PLASMA) ? p->dz * eps_m / (2.0 * k0) * std::pow(kIref, (double)p->K) : 0.0);
    a.aA = (T)((p->terms & NLSE_MPA) ? p->dz * (-p->betaK) / 2.0 * std::pow(kIref, (double)(p->K - 1)) : 0.0);
    return a;
}

}  // namespace

struct nlse_adjoint {
    nlse_params p;
    int32_t nsteps, ckpt;
    cudaStream_t stream;
    unsigned char* ws;
    AdjLayout lay;
    int cols;
    int row_radix;
    const KernelSet<float>* k32;
    const KernelSet<double>* k64;
    AdjCoef<float> ac32;
    AdjCoef<double> ac64;
    double sum_d2;
    int have_target, have_forward;
};

namespace {

template <typename T> struct ASel;
template <> struct ASel<float> {
    static const KernelSet<float>* ks(const nlse_adjoint* a) { return a->k32; }
    static const AdjCoef<float>& ac(const nlse_adjoint* a) { return a->ac32; }
};
template <> struct ASel<double> {
    static const KernelSet<double>* ks(const nlse_adjoint* a) { return a->k64; }
    static const AdjCoef<double>& ac(const nlse_adjoint* a) { return a->ac64; }
};

template <typename T> VT<T>* aat(nlse_adjoint* a, size_t off) { return reinterpret_cast<VT<T>*>(a->ws + off); }
template <typename T> const WT<T>* atab(nlse_adjoint* a, size_t off) {
    return reinterpret_cast<const WT<T>*>(a->ws + off);
}
inline size_t adj_field_bytes(const nlse_adjoint* a) {
    return (size_t)a->p.n * a->p.n * (a->p.precision == NLSE_FP64 ? 16 : 8);
}

template <typename T> nlse_status adj_upload(nlse_adjoint* a);
template <> nlse_status adj_upload<double>(nlse_adjoint* a) {
    std::vector<double> px, py, tw;
    propagator_tables(&a->p, px, py);
    twiddle_table(a->p.n, std::min(a->p.n, 8), tw);
    // conjugated propagator tables: the conjugates of the same values
    std::vector<double> pxc = px, pyc = py;
    for (size_t i = 1; i < pxc.size(); i += 2) { pxc[i] = -pxc[i]; pyc[i] = -pyc[i]; }
    const std::vector<double>* src[5] = {&tw, &px, &py, &pxc, &pyc};
    const size_t off[5] = {a->lay.tw, a->lay.px, a->lay.py, a->lay.pxc, a->lay.pyc};
    for (int t = 0; t < 5; ++t)
        if (cudaMemcpyAsync(a->ws + off[t], src[t]->data(), src[t]->size() * sizeof(double), cudaMemcpyHostToDevice,
                            a->stream) != cudaSuccess)
            return NLSE_ECUDA;
    return cudaStreamSynchronize(a->stream) == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}
template <> nlse_status adj_upload<float>(nlse_adjoint* a) {
    HostTables32 t;
    build_tables_f32(&a->p, t);
    // conjugated propagator tables: the conjugates of the same rounded values
    // (P_x entries (d, s); P_y entries (d, d', s, s'))
    std::vector<float> pxc = t.px, pyc = t.py;
    for (size_t i = 1; i < pxc.size(); i += 2) pxc[i] = -pxc[i];
    // in every copy the n/2 P_y entries (d, d', s, s') are conjugated; the
    // cross-lane factors that follow belong to the transform and stay as they are
    const int hn = a->p.n / 2;
    const size_t pyf = py32_copy_bytes(a->p.n) / 4;
    for (size_t c0 = 0; c0 < pyc.size(); c0 += pyf)
        for (int k = 0; k < hn; ++k) {
            pyc[c0 + 4 * k + 2] = -pyc[c0 + 4 * k + 2];
            pyc[c0 + 4 * k + 3] = -pyc[c0 + 4 * k + 3];
        }
    const void* src[5] = {t.tw.data(), t.px.data(), t.py.data(), pxc.data(), pyc.data()};
    const size_t bytes[5] = {t.tw.size(), t.px.size() * 4, t.py.size() * 4, pxc.size() * 4, pyc.size() * 4};
    const size_t off[5] = {a->lay.tw, a->lay.px, a->lay.py, a->lay.pxc, a->lay.pyc};
    for (int q = 0; q < 5; ++q)
        if (cudaMemcpyAsync(a->ws + off[q], src[q], bytes[q], cudaMemcpyHostToDevice, a->stream) != cudaSuccess)
            return NLSE_ECUDA;
    return cudaStreamSynchronize(a->stream) == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}

template <typename T> nlse_status adj_forward_impl(nlse_adjoint* a, const void* src, int on_device, double* loss) {
    const KernelSet<T>* ks = ASel<T>::ks(a);
    VT<T>* state = aat<T>(a, a->lay.state);
    const WT<T>* tw = twiddles_fixed<T>(a->ws + a->lay.tw);
    const int n = a->p.n;
    const size_t fb = adj_field_bytes(a);
    cudaError_t e;
    if (on_device) {
        e = ks->row_forward((const VT<T>*)src, state, tw, a->stream);
    } else {  // the host field is staged in gam (free until the backward sweep)
        VT<T>* rows = aat<T>(a, a->lay.gam);
        e = cudaMemcpyAsync(rows, src, fb, cudaMemcpyHostToDevice, a->stream);
        if (e == cudaSuccess) e = ks->row_forward(rows, state, tw, a->stream);
    }
    if (e != cudaSuccess) return NLSE_ECUDA;
    const ScreenCoef<T>& sc = ASel<T>::ac(a).sc;
    double* partials = reinterpret_cast<double*>(a->ws + a->lay.partials);
    for (int s = 0; s < a->nsteps; ++s) {
        if (s % a->ckpt == 0 &&
            cudaMemcpyAsync(a->ws + a->lay.ckpt + fb * (size_t)(s / a->ckpt), state, fb,
                            cudaMemcpyDeviceToDevice, a->stream) != cudaSuccess)
            return NLSE_ECUDA;
        const WT<T>* tws = twiddles_at<T>(a->ws + a->lay.tw, n, s);
        if (ks->col_pass(state, state, tws, px_at<T>(a->ws + a->lay.px, n, s),
                         py_at<T>(a->ws + a->lay.py, n, s), rot_for_step<T>(s, nullptr), a->cols, nullptr,
                         0u, a->stream) != cudaSuccess)
            return NLSE_ECUDA;
        if (ks->row_pass(state, state, tws, sc, partials, false, a->row_radix, nullptr, 0u, a->stream) !=
            cudaSuccess)
            return NLSE_ECUDA;
    }
    double* result = reinterpret_cast<double*>(a->ws + a->lay.result);
    if (ks->loss_seed(state, aat<T>(a, a->lay.gam), reinterpret_cast<const double*>(a->ws + a->lay.target),
                      tw, 1.0 / a->sum_d2, partials, a->stream) != cudaSuccess)
        return NLSE_ECUDA;
    k_finalize<<<1, 256, 0, a->stream>>>(partials, ks->adj_blocks, 1.0 / a->sum_d2, result,
                                         reinterpret_cast<int*>(result + 4));
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    double r[2];
    if (cudaMemcpyAsync(r, result, sizeof(r), cudaMemcpyDeviceToHost, a->stream) != cudaSuccess)
        return NLSE_ECUDA;
    if (cudaStreamSynchronize(a->stream) != cudaSuccess) return NLSE_ECUDA;
    *loss = r[0];
    return std::isfinite(r[0]) ? NLSE_OK : NLSE_ENONFINITE;
}

template <typename T> nlse_status adj_backward_impl(nlse_adjoint* a, double* dtheta, void* dU0, int on_device) {
    const KernelSet<T>* ks = ASel<T>::ks(a);
    const AdjCoef<T>& ac = ASel<T>::ac(a);
    VT<T>* state = aat<T>(a, a->lay.state);
    VT<T>* gam = aat<T>(a, a->lay.gam);
    const WT<T>* tw = twiddles_fixed<T>(a->ws + a->lay.tw);
    const int n = a->p.n;
    const size_t fb = adj_field_bytes(a);
    double* partials = reinterpret_cast<double*>(a->ws + a->lay.partials);
    double* acc = reinterpret_cast<double*>(a->ws + a->lay.acc);
    if (cudaMemsetAsync(acc, 0, (size_t)a->p.n * 6 * sizeof(double), a->stream) != cudaSuccess)
        return NLSE_ECUDA;
    auto seg = [&](int i) { return reinterpret_cast<VT<T>*>(a->ws + a->lay.seg + fb * (size_t)i); };
    for (int c = (a->nsteps - 1) / a->ckpt; c >= 0; --c) {
        const int c0 = c * a->ckpt, c1 = std::min(c0 + a->ckpt, (int)a->nsteps);
        if (cudaMemcpyAsync(state, a->ws + a->lay.ckpt + fb * (size_t)c, fb, cudaMemcpyDeviceToDevice,
                            a->stream) != cudaSuccess)
            return NLSE_ECUDA;
        for (int s = c0; s < c1; ++s) {  // recompute the segment, keeping T_s
            const WT<T>* tws = twiddles_at<T>(a->ws + a->lay.tw, n, s);
            if (ks->col_pass(state, seg(s - c0), tws, px_at<T>(a->ws + a->lay.px, n, s),
                             py_at<T>(a->ws + a->lay.py, n, s), rot_for_step<T>(s, nullptr), a->cols,
                             nullptr, 0u, a->stream) != cudaSuccess)
                return NLSE_ECUDA;
            if (s + 1 < c1 &&
                ks->row_pass(seg(s - c0), state, tws, ac.sc, partials, false, a->row_radix, nullptr, 0u, a->stream) !=
                    cudaSuccess)
                return NLSE_ECUDA;
        }
        for (int s = c1 - 1; s >= c0; --s) {  // reverse the segment with the forward step's constants
            const WT<T>* tws = twiddles_at<T>(a->ws + a->lay.tw, n, s);
            if (ks->adj_row(gam, seg(s - c0), tws, ac, acc, a->stream) != cudaSuccess) return NLSE_ECUDA;
            if (ks->col_pass(gam, gam, tws, px_at<T>(a->ws + a->lay.pxc, n, s),
                             py_at<T>(a->ws + a->lay.pyc, n, s), conj_of(rot_for_step<T>(s, nullptr)), a->cols,
                             nullptr, 0u, a->stream) != cudaSuccess)
                return NLSE_ECUDA;
        }
    }
    // dJ/dU0 = B_x G_S0 (the readout applies 1/n, undone by the factor n)
    VT<T> scale;
    scale.x = (T)a->p.n;
    scale.y = (T)0;
    VT<T>* out = on_device ? (VT<T>*)dU0 : seg(0);
    if (ks->readout(gam, tw, out, nullptr, partials, scale, a->stream) != cudaSuccess) return NLSE_ECUDA;
    std::vector<double> h((size_t)a->p.n * 6);
    if (cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, a->stream) !=
        cudaSuccess)
        return NLSE_ECUDA;
    if (!on_device &&
        cudaMemcpyAsync(dU0, out, fb, cudaMemcpyDeviceToHost, a->stream) != cudaSuccess)
        return NLSE_ECUDA;
    if (cudaStreamSynchronize(a->stream) != cudaSuccess) return NLSE_ECUDA;
    for (int q = 0; q < 6; ++q) dtheta[q] = 0.0;
    for (int b = 0; b < ks->adj_blocks; ++b)  // fixed order: deterministic
        for (int q = 0; q < 6; ++q) dtheta[q] += h[6 * (size_t)b + q];
    return NLSE_OK;
}

}  // namespace

extern "C" {

nlse_status nlse_adjoint_workspace_size(const nlse_params* p, int32_t nsteps, int32_t ckpt_every,
                                        size_t* bytes) {
    if (!bytes || nsteps < 1 || ckpt_every < 1) return NLSE_EINVAL;
    nlse_status st = validate(p);
    if (st != NLSE_OK) return st;
    if (p->scheme != NLSE_LIE) return NLSE_EUNSUPPORTED;  // the adjoint differentiates the Lie march
    *bytes = adj_layout_for(p->n, p->precision, nsteps, std::min(ckpt_every, nsteps)).total;
    return NLSE_OK;
}

nlse_status nlse_adjoint_create(const nlse_params* p, int32_t nsteps, int32_t ckpt_every, void* cuda_stream,
                                void* dev_workspace, size_t workspace_bytes, nlse_adjoint** out) {
    if (!out || !dev_workspace || nsteps < 1 || ckpt_every < 1) return NLSE_EINVAL;
    *out = nullptr;
    nlse_status st = validate(p);
    if (st != NLSE_OK) return st;
    if (p->scheme != NLSE_LIE) return NLSE_EUNSUPPORTED;
    if (reinterpret_cast<uintptr_t>(dev_workspace) & 255) return NLSE_EINVAL;
    const int ck = std::min(ckpt_every, nsteps);
    AdjLayout lay = adj_layout_for(p->n, p->precision, nsteps, ck);
    if (workspace_bytes < lay.total) return NLSE_ENOMEM;
    nlse_adjoint* a = new (std::nothrow) nlse_adjoint();
    if (!a) return NLSE_ENOMEM;
    a->p = *p;
    a->nsteps = nsteps;
    a->ckpt = ck;
    a->stream = static_cast<cudaStream_t>(cuda_stream);
    a->ws = static_cast<unsigned char*>(dev_workspace);
    a->lay = lay;
    const int k = log2_exact(p->n);
    if (p->precision == NLSE_FP64) {
        a->k64 = kernels_f64(k);
        a->cols = a->k64->col_default;
        a->row_radix = a->k64->row_radix_default;
        a->ac64 = adj_coef<double>(p);
        st = adj_upload<double>(a);
    } else {
        a->k32 = kernels_f32(k);
        a->cols = a->k32->col_default;
        a->row_radix = a->k32->row_radix_default;
        a->ac32 = adj_coef<float>(p);
        st = adj_upload<float>(a);
    }
    if (st != NLSE_OK) { delete a; return st; }
    *out = a;
    return NLSE_OK;
}

nlse_status nlse_adjoint_set_launch(nlse_adjoint* a, int32_t cols, int32_t row_radix) {
    if (!a) return NLSE_EINVAL;
    const bool f64 = a->p.precision == NLSE_FP64;
    const int cmask = f64 ? a->k64->col_mask : a->k32->col_mask;
    const int rmask = f64 ? a->k64->row_radix_mask : a->k32->row_radix_mask;
    bool col_ok = false;
    for (int i = 0; i < kColOptionCount; ++i) col_ok |= kColOptions[i] == cols && ((cmask >> i) & 1);
    const int bit = row_radix == 16 ? 1 : row_radix == 8 ? 2 : row_radix == (kRowStaged | 16) ? 4 : 0;
    if (!col_ok || !(rmask & bit)) return NLSE_EUNSUPPORTED;
    a->cols = cols;
    a->row_radix = row_radix;
    a->have_forward = 0;
    return NLSE_OK;
}

nlse_status nlse_adjoint_set_theta(nlse_adjoint* a, const double* theta) {
    if (!a || !theta) return NLSE_EINVAL;
    nlse_params q = a->p;
    for (int i = 0; i < 6; ++i) q.theta[i] = theta[i];
    nlse_status st = validate(&q);
    if (st != NLSE_OK) return st;
    a->p = q;
    if (a->p.precision == NLSE_FP64) a->ac64 = adj_coef<double>(&a->p);
    else a->ac32 = adj_coef<float>(&a->p);
    a->have_forward = 0;
    return NLSE_OK;
}

nlse_status nlse_adjoint_set_target(nlse_adjoint* a, const double* target, int on_device) {
    if (!a || !target) return NLSE_EINVAL;
    const int n = a->p.n;
    const size_t bytes = (size_t)n * n * sizeof(double);
    double* d = reinterpret_cast<double*>(a->ws + a->lay.target);
    if (cudaMemcpyAsync(d, target, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        a->stream) != cudaSuccess)
        return NLSE_ECUDA;
    double* partials = reinterpret_cast<double*>(a->ws + a->lay.partials);
    double* result = reinterpret_cast<double*>(a->ws + a->lay.result);
    k_sumsq_rows<<<n, 256, 0, a->stream>>>(d, n, partials);
    k_finalize<<<1, 256, 0, a->stream>>>(partials, n, 1.0, result, reinterpret_cast<int*>(result + 4));
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    double r[2];
    if (cudaMemcpyAsync(r, result, sizeof(r), cudaMemcpyDeviceToHost, a->stream) != cudaSuccess)
        return NLSE_ECUDA;
    if (cudaStreamSynchronize(a->stream) != cudaSuccess) return NLSE_ECUDA;
    if (!(r[0] > 0.0) || !std::isfinite(r[0])) return NLSE_EINVAL;  // an all-zero target has no loss scale
    a->sum_d2 = r[0];
    a->have_target = 1;
    a->have_forward = 0;
    return NLSE_OK;
}

nlse_status nlse_adjoint_forward(nlse_adjoint* a, const void* U0, int on_device, double* loss) {
    if (!a || !U0 || !loss) return NLSE_EINVAL;
    if (!a->have_target) return NLSE_ESTATE;
    nlse_status st = a->p.precision == NLSE_FP64 ? adj_forward_impl<double>(a, U0, on_device, loss)
                                                 : adj_forward_impl<float>(a, U0, on_device, loss);
    a->have_forward = st == NLSE_OK;
    return st;
}

nlse_status nlse_adjoint_backward(nlse_adjoint* a, double* dtheta, void* dU0, int dU0_on_device) {
    if (!a || !dtheta || !dU0) return NLSE_EINVAL;
    if (!a->have_forward) return NLSE_ESTATE;
    a->have_forward = 0;  // the backward sweep consumes the seeded adjoint state
    return a->p.precision == NLSE_FP64 ? adj_backward_impl<double>(a, dtheta, dU0, dU0_on_device)
                                       : adj_backward_impl<float>(a, dtheta, dU0, dU0_on_device);
}

nlse_status nlse_adjoint_destroy(nlse_adjoint* a) {
    if (!a) return NLSE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(a->stream);
    delete a;
    return cuerr(e);
}

}  // extern "C"
