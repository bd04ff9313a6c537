/*
 * nlse_oracle.c -- plain, slow FP64 CPU oracle for the split-step (phase-screen)
 * z-march of the stationary transverse NLSE of Bulygin & Geints,
 * "Toward high-speed effective numerical simulation of multiple filamentation
 * of high-power femtosecond laser radiation in transparent medium" (arXiv 2306.15678).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle for the CUDA path.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA library: every quantity below is recomputed here from the physical inputs.
 *
 * What it computes (all in double precision, physical CGS-optical units:
 * lengths in cm, intensity I = |U|^2 in W/cm^2, power in W):
 *
 *   Eq. 1  2 i k0 dU/dz = (Lap_perp + eps_k |U|^2 + eps_h[U]) U
 *   Eq. 3  eps_h U = (eps_m I^K + i k0 alpha_m I^(K-1)) U   (exponents read as
 *          I^m and I^(m-1) with m = K, the multiphoton order; the printed
 *          (UU*)^(2m) is taken as a typesetting slip)
 *   Eq. 2  one step over dz is the operator exponential split into a linear
 *          diffraction part and a nonlinear screen that is evaluated on the
 *          field entering the screen (U_in) and held fixed over the step.
 *
 * One z step (Lie order, diffraction first, then the screen):
 *   U_hat = FFT2(U);  U_hat *= exp(+i (kx^2 + ky^2) dz / (2 k0));
 *   v = IFFT2(U_hat) (1/N^2 normalisation);
 *   U = v * exp(s(|v|^2)),
 *   s(I) = -i dz/(2 k0) [c_K eps_k I + c_P eps_m I^K + c_A i k0 alpha_m I^(K-1)],
 *   c_K = theta0 + i theta1, c_P = theta2 + i theta3, c_A = theta4 + i theta5.
 *
 * Coefficient readings (the paper prints no values; both sides read them from
 * the same parameter record):
 *   k0 = 2 pi n0 / lambda0, eps_k = 2 k0^2 n2 / n0 (Kerr),
 *   eps_m = -k0^2 sigma_K rho_nt tau_pl / rho_c (plasma defocusing),
 *   alpha_m = -beta_K (multiphoton absorption, dI/dz = -beta_K I^K).
 *
 * The FFT is an iterative radix-2 Cooley-Tukey transform with a twiddle table
 * built from cos/sin of the exact angle; forward is unnormalised, inverse
 * carries 1/N per dimension.  Spatial frequencies k_m = 2 pi m~/L with
 * m~ = m for m < N/2 and m - N otherwise.
 *
 * Pins (tests/test_oracle_pins.py): brute-force DFT and numpy.fft.fft2 for the
 * FFT; the closed-form Gaussian beam for diffraction; the exact pointwise Kerr,
 * plasma and absorption identities for the screen; power conservation, time
 * reversal, the discrete energy balance and mirror/transpose symmetry for the
 * march; central finite differences for the adjoint; math.fsum / brute force
 * for the readouts and the loss; hand-counted patterns and scipy.ndimage.label
 * for the hot areas; single spectral lines and the Kerr screen for the
 * turbulent layer; the heat-kernel closed form, hand-made lenses and the
 * single-centre screen for the effective lens.
 */
#define _POSIX_C_SOURCE 200809L
#define _DEFAULT_SOURCE 1
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Parameter record of the oracle (its own layout; mirrored only by the
 * oracle's Python wrapper). */
typedef struct {
    int32_t n;        /* grid points per side, power of two */
    int32_t K;        /* multiphoton order m of Eq. 3 */
    uint32_t terms;   /* bit 0 Kerr, bit 1 plasma, bit 2 absorption, bit 3 diffraction */
    int32_t reserved; /* screen: 0 frozen at the entering intensity (Eq. 2), 1 exact substep */
    double L;         /* transverse window, cm */
    double dz;        /* z step, cm */
    double lambda0;   /* carrier wavelength, cm */
    double n0;        /* linear refractive index */
    double n2;        /* Kerr index, cm^2/W */
    double sigmaK;    /* K-photon ionisation rate coefficient, s^-1 cm^2K W^-K */
    double rho_nt;    /* neutral density, cm^-3 */
    double rho_c;     /* critical plasma density, cm^-3 */
    double tau_pl;    /* effective pulse duration, s */
    double betaK;     /* K-photon absorption coefficient, cm^(2K-3) W^(1-K) */
    double theta[6];  /* complex gains (re, im) on Kerr, plasma, absorption */
} orc_params;

enum { ORC_KERR = 1u, ORC_PLASMA = 2u, ORC_MPA = 4u, ORC_DIFFRACTION = 8u };

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops of the calling thread (timing of
 * the oracle on fewer cores; the arithmetic and its order do not depend on it:
 * every parallel loop writes disjoint outputs and the sums are serial). */
void orc_set_num_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/* ------------------------------------------------------------------ FFT -- */

/* twiddle table tw[j] = exp(-2 pi i j / n), j < n/2 */
static cplx *make_twiddles(int n) {
    cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)(n / 2 > 0 ? n / 2 : 1));
    for (int j = 0; j < n / 2; ++j) {
        double a = -2.0 * M_PI * (double)j / (double)n;
        tw[j] = cos(a) + I * sin(a);
    }
    return tw;
}

/* in-place radix-2 transform of a contiguous array of length n */
static void fft1d_contig(cplx *a, int n, int inverse, const cplx *tw) {
    for (int i = 1, j = 0; i < n; ++i) {  /* bit-reversal permutation */
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2, step = n / len;
        for (int i = 0; i < n; i += len) {
            for (int j = 0; j < half; ++j) {
                cplx w = tw[j * step];
                if (inverse) w = conj(w);
                cplx u = a[i + j], v = a[i + j + half] * w;
                a[i + j] = u + v;
                a[i + j + half] = u - v;
            }
        }
    }
    if (inverse) {
        double s = 1.0 / (double)n;
        for (int i = 0; i < n; ++i) a[i] *= s;
    }
}

/* 1D transform of a length-n vector with a stride (used by the tests) */
void orc_fft1d(cplx *a, int n, int stride, int inverse) {
    cplx *tw = make_twiddles(n);
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int i = 0; i < n; ++i) buf[i] = a[(size_t)i * stride];
    fft1d_contig(buf, n, inverse, tw);
    for (int i = 0; i < n; ++i) a[(size_t)i * stride] = buf[i];
    free(buf);
    free(tw);
}

/* 2D transform of a row-major n x n array: rows (x), then columns (y) */
void orc_fft2d(cplx *a, int n, int inverse) {
    cplx *tw = make_twiddles(n);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) fft1d_contig(a + (size_t)r * n, n, inverse, tw);
#pragma omp parallel
    {
        cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
        for (int c = 0; c < n; ++c) {
            for (int r = 0; r < n; ++r) col[r] = a[(size_t)r * n + c];
            fft1d_contig(col, n, inverse, tw);
            for (int r = 0; r < n; ++r) a[(size_t)r * n + c] = col[r];
        }
        free(col);
    }
    free(tw);
}

/* ---------------------------------------------------------- diffraction -- */

static double wavenumber(const orc_params *p) { return 2.0 * M_PI * p->n0 / p->lambda0; }

/* signed spatial frequency of FFT bin m: 2 pi m~ / L */
static double kfreq(int m, int n, double L) {
    int mm = (m < n / 2) ? m : m - n;
    return 2.0 * M_PI * (double)mm / L;
}

/* Diffraction propagator of Eq. 1-2: Lap_perp -> -k_perp^2 in Fourier space,
 * so dU_hat/dz = +i k_perp^2/(2 k0) U_hat and P = exp(+i k_perp^2 dz/(2 k0)).
 * Written as a full 2D table (no separable shortcut). */
void orc_propagator(const orc_params *p, cplx *P) {
    int n = p->n;
    double k0 = wavenumber(p);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) {
        double ky = kfreq(r, n, p->L);
        for (int c = 0; c < n; ++c) {
            double kx = kfreq(c, n, p->L);
            double phase = (kx * kx + ky * ky) * p->dz / (2.0 * k0);
            P[(size_t)r * n + c] = cexp(I * phase);
        }
    }
}

/* linear half of the step: U <- IFFT2(P * FFT2(U)) */
void orc_linear(const orc_params *p, cplx *U) {
    if (!(p->terms & ORC_DIFFRACTION)) return;
    size_t nn = (size_t)p->n * p->n;
    cplx *P = (cplx *)malloc(sizeof(cplx) * nn);
    orc_propagator(p, P);
    orc_fft2d(U, p->n, 0);
    for (size_t i = 0; i < nn; ++i) U[i] *= P[i];
    orc_fft2d(U, p->n, 1);
    free(P);
}

/* adjoint of the linear half: U <- IFFT2(conj(P) * FFT2(U)) */
static void orc_linear_adjoint(const orc_params *p, cplx *U) {
    if (!(p->terms & ORC_DIFFRACTION)) return;
    size_t nn = (size_t)p->n * p->n;
    cplx *P = (cplx *)malloc(sizeof(cplx) * nn);
    orc_propagator(p, P);
    orc_fft2d(U, p->n, 0);
    for (size_t i = 0; i < nn; ++i) U[i] *= conj(P[i]);
    orc_fft2d(U, p->n, 1);
    free(P);
}

/* --------------------------------------------------------------- screen -- */

typedef struct {
    double k0, eps_k, eps_m, alpha_m;
    cplx cK, cP, cA;
    int useK, useP, useA;
} screen_coef;

static screen_coef make_coef(const orc_params *p) {
    screen_coef c;
    c.k0 = wavenumber(p);
    c.eps_k = 2.0 * c.k0 * c.k0 * p->n2 / p->n0;
    c.eps_m = -c.k0 * c.k0 * p->sigmaK * p->rho_nt * p->tau_pl / p->rho_c;
    c.alpha_m = -p->betaK;
    c.cK = p->theta[0] + I * p->theta[1];
    c.cP = p->theta[2] + I * p->theta[3];
    c.cA = p->theta[4] + I * p->theta[5];
    c.useK = (p->terms & ORC_KERR) != 0;
    c.useP = (p->terms & ORC_PLASMA) != 0;
    c.useA = (p->terms & ORC_MPA) != 0;
    return c;
}

/* exponent s(I) of the pointwise screen (Eq. 2 with the terms of Eq. 3) */
static cplx screen_exponent(const screen_coef *c, const orc_params *p, double In) {
    cplx bracket = 0.0;
    if (c->useK) bracket += c->cK * c->eps_k * In;
    if (c->useP) bracket += c->cP * c->eps_m * pow(In, (double)p->K);
    if (c->useA) bracket += c->cA * I * c->k0 * c->alpha_m * pow(In, (double)(p->K - 1));
    return -I * p->dz / (2.0 * c->k0) * bracket;
}

/* dS/dI, used by the adjoint */
static cplx screen_exponent_dI(const screen_coef *c, const orc_params *p, double In) {
    cplx bracket = 0.0;
    if (c->useK) bracket += c->cK * c->eps_k;
    if (c->useP) bracket += c->cP * c->eps_m * (double)p->K * pow(In, (double)(p->K - 1));
    if (c->useA && p->K >= 2)
        bracket += c->cA * I * c->k0 * c->alpha_m * (double)(p->K - 1) * pow(In, (double)(p->K - 2));
    return -I * p->dz / (2.0 * c->k0) * bracket;
}

/* dS/dtheta_j for j = 0..5 */
static void screen_exponent_dtheta(const screen_coef *c, const orc_params *p, double In, cplx out[6]) {
    cplx base[3];
    base[0] = c->useK ? c->eps_k * In : 0.0;
    base[1] = c->useP ? c->eps_m * pow(In, (double)p->K) : 0.0;
    base[2] = c->useA ? I * c->k0 * c->alpha_m * pow(In, (double)(p->K - 1)) : 0.0;
    for (int t = 0; t < 3; ++t) {
        cplx pre = -I * p->dz / (2.0 * c->k0) * base[t];
        out[2 * t] = pre;          /* d/d(real part of the gain) */
        out[2 * t + 1] = I * pre;  /* d/d(imaginary part of the gain) */
    }
}

/* Exact pointwise substep (p->reserved == 1): the nonlinear part of Eq. 1-3
 * over dz solved exactly instead of frozen at the entering intensity, for
 * real gains (theta[1] = theta[3] = theta[5] = 0, K >= 2).  Pointwise the
 * equation is dU/dz = -(i/(2 k0)) (c_K eps_k I + c_P eps_m I^K) U
 * - (c_A beta_K / 2) I^(K-1) U, so the intensity obeys dI/dz = -b I^K
 * (b = c_A beta_K) and the phase integrates the intensity:
 *   I(z) = I0 (1 + a z/dz)^(-1/(K-1)),  a = (K-1) b I0^(K-1) dz,
 *   int_0^dz I   = I0 dz [(1+a)^((K-2)/(K-1)) - 1] / (a (K-2)/(K-1))   (K = 2: ln(1+a)/a),
 *   int_0^dz I^K = I0^K dz (K-1) [1 - (1+a)^(-1/(K-1))] / a,
 * each factor 1 when a = 0; written with log1p / expm1 so small a loses nothing. */
static void screen_exact_point(const orc_params *p, const screen_coef *c, cplx *u) {
    cplx v = *u;
    double I0 = creal(v) * creal(v) + cimag(v) * cimag(v);
    int K = p->K;
    double b = c->useA ? creal(c->cA) * p->betaK : 0.0;
    double a = (double)(K - 1) * b * pow(I0, (double)(K - 1)) * p->dz;
    double amp = 1.0, f1 = 1.0, fk = 1.0;
    if (a != 0.0) {
        double l = log1p(a);
        amp = exp(-l / (2.0 * (K - 1)));
        if (K == 2) f1 = l / a;
        else {
            double e = (double)(K - 2) / (double)(K - 1);
            f1 = expm1(e * l) / (a * e);
        }
        fk = -(double)(K - 1) * expm1(-l / (double)(K - 1)) / a;
    }
    double bracket = 0.0;
    if (c->useK) bracket += creal(c->cK) * c->eps_k * I0 * f1;
    if (c->useP) bracket += creal(c->cP) * c->eps_m * pow(I0, (double)K) * fk;
    double phase = -p->dz / (2.0 * c->k0) * bracket;
    *u = v * amp * cexp(I * phase);
}

/* nonlinear half of the step: U <- v * exp(s(|v|^2)), screen held at |v|^2
 * (or the exact substep above when p->reserved == 1) */
void orc_screen(const orc_params *p, cplx *U) {
    if (!(p->terms & (ORC_KERR | ORC_PLASMA | ORC_MPA))) return;
    screen_coef c = make_coef(p);
    if (p->reserved == 1) {
        size_t nn0 = (size_t)p->n * p->n;
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < nn0; ++i) screen_exact_point(p, &c, &U[i]);
        return;
    }
    size_t nn = (size_t)p->n * p->n;
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < nn; ++i) {
        cplx v = U[i];
        double In = creal(v) * creal(v) + cimag(v) * cimag(v);
        U[i] = v * cexp(screen_exponent(&c, p, In));
    }
}

/* ------------------------------------------------------------- readouts -- */

/* Neumaier-compensated sum, fixed row-major order */
static double nsum_abs2(const cplx *U, size_t nn) {
    double s = 0.0, comp = 0.0;
    for (size_t i = 0; i < nn; ++i) {
        double x = creal(U[i]) * creal(U[i]) + cimag(U[i]) * cimag(U[i]);
        double t = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - t) + x; else comp += (x - t) + s;
        s = t;
    }
    return s + comp;
}

/* beam power P = sum |U|^2 dx^2 (rectangle rule), W */
double orc_power(const cplx *U, int n, double L) {
    double dx = L / (double)n;
    return nsum_abs2(U, (size_t)n * n) * dx * dx;
}

/* Spatial moment of Eq. 8, M(p, q) = integral of I^p (x^2 + y^2)^q dx dy with
 * I = U U*, by the rectangle rule on the cell centres x_j = (j - n/2 + 1/2) dx.
 * The printed Q^{mn} = int (U_n U_n*)^{2m} (x^2+y^2)^m is read, as Eq. 3's
 * exponents are, with (UU*)^{2m} standing for |U|^{2m} = I^m: Q^m = M(m, m)
 * for beam n.  M(1, 0) is the power. */
double orc_moment(const cplx *U, int n, double L, int p, int q) {
    double dx = L / (double)n;
    double sum = 0.0;
    for (int y = 0; y < n; ++y) {
        double yc = ((double)y - n / 2 + 0.5) * dx;
        for (int x = 0; x < n; ++x) {
            double xc = ((double)x - n / 2 + 0.5) * dx;
            cplx u = U[(size_t)y * n + x];
            double inten = creal(u) * creal(u) + cimag(u) * cimag(u);
            sum += pow(inten, (double)p) * pow(xc * xc + yc * yc, (double)q);
        }
    }
    return sum * dx * dx;
}

/* peak intensity max |U|^2, W/cm^2 */
double orc_peak(const cplx *U, int n) {
    double m = 0.0;
    size_t nn = (size_t)n * n;
    for (size_t i = 0; i < nn; ++i) {
        double x = creal(U[i]) * creal(U[i]) + cimag(U[i]) * cimag(U[i]);
        if (x > m) m = x;
    }
    return m;
}

/* fluence w = U U^* (stationary model), averaged over aligned ds x ds blocks */
void orc_fluence(const cplx *U, int n, int ds, double *out) {
    int m = n / ds;
    for (int R = 0; R < m; ++R)
        for (int C = 0; C < m; ++C) {
            double s = 0.0;
            for (int r = 0; r < ds; ++r)
                for (int c = 0; c < ds; ++c) {
                    cplx v = U[(size_t)(R * ds + r) * n + (C * ds + c)];
                    s += creal(v) * creal(v) + cimag(v) * cimag(v);
                }
            out[(size_t)R * m + C] = s / (double)(ds * ds);
        }
}

/* fluence-mismatch loss J = sum (|U|^2 - D)^2 / sum D^2 */
double orc_loss(const cplx *U, const double *D, int n) {
    size_t nn = (size_t)n * n;
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < nn; ++i) {
        double F = creal(U[i]) * creal(U[i]) + cimag(U[i]) * cimag(U[i]);
        num += (F - D[i]) * (F - D[i]);
        den += D[i] * D[i];
    }
    return num / den;
}

/* ---------------------------------------------------------------- march -- */

/* nsteps Lie steps in place; power[k], peak[k] after k steps (k = 0..nsteps)
 * when the arrays are non-NULL */
void orc_march(const orc_params *p, cplx *U, int nsteps, double *power, double *peak) {
    if (power) power[0] = orc_power(U, p->n, p->L);
    if (peak) peak[0] = orc_peak(U, p->n);
    for (int s = 0; s < nsteps; ++s) {
        orc_linear(p, U);
        orc_screen(p, U);
        if (power) power[s + 1] = orc_power(U, p->n, p->L);
        if (peak) peak[s + 1] = orc_peak(U, p->n);
    }
}

/* nsteps symmetric (Strang) steps in place: half a screen step, the full
 * diffraction step, half a screen step (the phase-screen operator exponential
 * of Eq. 2 split symmetrically; each half-screen is the frozen-intensity
 * screen of orc_screen over dz/2).  power[k], peak[k] after k steps. */
void orc_march_strang(const orc_params *p, cplx *U, int nsteps, double *power, double *peak) {
    orc_params half = *p;
    half.dz = 0.5 * p->dz;
    if (power) power[0] = orc_power(U, p->n, p->L);
    if (peak) peak[0] = orc_peak(U, p->n);
    for (int s = 0; s < nsteps; ++s) {
        orc_screen(&half, U);
        orc_linear(p, U);
        orc_screen(&half, U);
        if (power) power[s + 1] = orc_power(U, p->n, p->L);
        if (peak) peak[s + 1] = orc_peak(U, p->n);
    }
}

/* ------------------------------------------------------------ hot areas -- */

/* "Hot areas" (Sec. 3.3): the closed regions of the beam cross-section where the
 * fluence w >= w_p, counted as the connected components of the thresholded
 * grid.  conn = 4 (edge neighbours) or 8 (edge and corner neighbours); the
 * window is not periodic.  labels[i] = -1 outside the regions, else the
 * smallest row-major index of the pixel's region (row-major scan order makes
 * the first pixel met the smallest).  Returns the number of regions, or -1 for
 * a bad argument.  Plain flood fill with an explicit stack. */
int orc_hot_areas(const double *w, int n, double wp, int conn, int32_t *labels) {
    if (n < 1 || (conn != 4 && conn != 8)) return -1;
    size_t nn = (size_t)n * n;
    for (size_t i = 0; i < nn; ++i) labels[i] = -2;  /* -2: unvisited */
    size_t *stack = malloc(nn * sizeof(size_t));
    if (!stack) return -1;
    int count = 0;
    for (size_t i = 0; i < nn; ++i) {
        if (labels[i] != -2) continue;
        if (!(w[i] >= wp)) { labels[i] = -1; continue; }
        ++count;
        size_t top = 0;
        stack[top++] = i;
        labels[i] = (int32_t)i;
        while (top > 0) {
            size_t q = stack[--top];
            int r = (int)(q / (size_t)n), c = (int)(q % (size_t)n);
            for (int dr = -1; dr <= 1; ++dr)
                for (int dc = -1; dc <= 1; ++dc) {
                    if (dr == 0 && dc == 0) continue;
                    if (conn == 4 && dr != 0 && dc != 0) continue;
                    int rr = r + dr, cc = c + dc;
                    if (rr < 0 || rr >= n || cc < 0 || cc >= n) continue;
                    size_t t = (size_t)rr * n + cc;
                    if (labels[t] != -2) continue;
                    if (w[t] >= wp) {
                        labels[t] = (int32_t)i;
                        stack[top++] = t;
                    } else {
                        labels[t] = -1;
                    }
                }
        }
    }
    free(stack);
    return count;
}

/* ---------------------------------------------------- turbulent screen -- */

/* Turbulent phase screen of Sec. 3.3 (Eqs. 9-10), built by the spectral method:
 * its spectral amplitude is a step, tau for spatial frequencies |k| <= k_h (k_h
 * read as the upper cut-off, so the step is theta(k_h - |k|)) and 0 above, and
 * the screen is the real part of the unnormalised inverse 2D DFT of that
 * amplitude times the caller's complex random draws xi (FFT bin order, rows =
 * k_y, columns = k_x):
 *   eps_t(y_l, x_j) = Re sum_{q,p} tau [p~^2 + q~^2 <= (k_h L / 2 pi)^2]
 *                     xi[q][p] exp(+2 pi i (p j + q l) / n),
 * with p~, q~ the signed bin numbers.  eps_t is written to eps (n*n). */
void orc_turbulent_eps(const orc_params *p, const cplx *xi, double tau, double kh, double *eps) {
    int n = p->n;
    size_t nn = (size_t)n * n;
    double rc = kh * p->L / (2.0 * M_PI);
    double r2 = rc * rc;
    cplx *S = (cplx *)malloc(sizeof(cplx) * nn);
    for (int q = 0; q < n; ++q) {
        int qq = (q < n / 2) ? q : q - n;
        for (int c = 0; c < n; ++c) {
            int pp = (c < n / 2) ? c : c - n;
            double m2 = (double)pp * pp + (double)qq * qq;
            S[(size_t)q * n + c] = (m2 <= r2) ? tau * xi[(size_t)q * n + c] : 0.0;
        }
    }
    orc_fft2d(S, n, 1); /* carries 1/n^2 */
    for (size_t i = 0; i < nn; ++i) eps[i] = creal(S[i]) * (double)nn;
    free(S);
}

/* The screen acts on the field like the other permittivity terms of Eq. 9 over
 * a layer of the given thickness: U <- U exp(-i thickness eps_t / (2 k0)), the
 * same form as the nonlinear screen's exp(-i dz/(2 k0) [...]). */
void orc_turbulent_screen(const orc_params *p, cplx *U, const cplx *xi, double tau, double kh,
                          double thickness) {
    size_t nn = (size_t)p->n * p->n;
    double *eps = (double *)malloc(sizeof(double) * nn);
    orc_turbulent_eps(p, xi, tau, kh, eps);
    double c = thickness / (2.0 * wavenumber(p));
    for (size_t i = 0; i < nn; ++i) U[i] *= cexp(-I * c * eps[i]);
    free(eps);
}

/* ------------------------------------------------------ effective lens -- */

/* Effective-lens screen of Sec. 2 (Eqs. 4-6).  Its parameters: the low-pass
 * length l_dif (cm^2) of Eq. 4, the trimming level w_l (W/cm^2), the neighbours
 * that join lens pixels (4 or 8), and the radial ansatz of Eq. 6: n_re
 * segments of the real part, segment j covering r_re[j-1] <= r < r_re[j]
 * (r_re[-1] = 0) with value a[j] cos(omega[j] r + psi[j]), and n_im segments of
 * the imaginary part with b, nu, eta; zero beyond the last joint. */
#define ORC_LENS_SEG 8
typedef struct {
    double l_dif, w_l;
    int32_t conn, n_re, n_im, reserved;
    double r_re[ORC_LENS_SEG], a[ORC_LENS_SEG], omega[ORC_LENS_SEG], psi[ORC_LENS_SEG];
    double r_im[ORC_LENS_SEG], b[ORC_LENS_SEG], nu[ORC_LENS_SEG], eta[ORC_LENS_SEG];
} orc_lens;

/* Eq. 4: w_dif = F^-1 exp(-l_dif k^2) F w, read with k^2 = kx^2 + ky^2 (the
 * printed exp(-l_dif) lacks its argument; a Gaussian low-pass is the operator
 * that widens every maximum and keeps w_dif decreasing away from it). */
void orc_lens_lowpass(int n, double L, const double *w, double l_dif, double *out) {
    size_t nn = (size_t)n * n;
    cplx *W = (cplx *)malloc(sizeof(cplx) * nn);
    for (size_t i = 0; i < nn; ++i) W[i] = w[i];
    orc_fft2d(W, n, 0);
    for (int r = 0; r < n; ++r) {
        double ky = kfreq(r, n, L);
        for (int c = 0; c < n; ++c) {
            double kx = kfreq(c, n, L);
            W[(size_t)r * n + c] *= exp(-l_dif * (kx * kx + ky * ky));
        }
    }
    orc_fft2d(W, n, 1);
    for (size_t i = 0; i < nn; ++i) out[i] = creal(W[i]);
    free(W);
}

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* Lens centres: the regions of w_dif >= w_l (trimming, Fig. 1) are the
 * disconnected lenses; the centre of each is its pixel of largest w_dif (the
 * first in row-major order on a tie).  Writes the centres' row-major indices
 * in increasing order to centres (room for n*n) and returns their number, or
 * -1 for a bad argument. */
int orc_lens_centres(const double *wd, int n, double w_l, int conn, int32_t *centres) {
    size_t nn = (size_t)n * n;
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * nn);
    int count = orc_hot_areas(wd, n, w_l, conn, lab);
    if (count < 0) { free(lab); return -1; }
    int32_t *best = (int32_t *)malloc(sizeof(int32_t) * nn);  /* per region root: pixel of the maximum */
    for (size_t i = 0; i < nn; ++i) best[i] = -1;
    for (size_t i = 0; i < nn; ++i) {
        int32_t root = lab[i];
        if (root < 0) continue;
        if (best[root] < 0 || wd[i] > wd[best[root]]) best[root] = (int32_t)i;
    }
    int k = 0;
    for (size_t i = 0; i < nn; ++i)
        if (lab[i] == (int32_t)i) centres[k++] = best[i];
    qsort(centres, (size_t)k, sizeof(int32_t), cmp_i32);
    free(best);
    free(lab);
    return k;
}

/* Eq. 6: the radial ansatz at distance r (cm) from a lens centre */
void orc_lens_value(const orc_lens *ls, double r, double *re, double *im) {
    *re = 0.0;
    *im = 0.0;
    for (int j = 0; j < ls->n_re; ++j)
        if (r < ls->r_re[j]) { *re = ls->a[j] * cos(ls->omega[j] * r + ls->psi[j]); break; }
    for (int j = 0; j < ls->n_im; ++j)
        if (r < ls->r_im[j]) { *im = ls->b[j] * cos(ls->nu[j] * r + ls->eta[j]); break; }
}

/* Eq. 5 and the screen of Eq. 2: D_f(r) = sum over the centres (in the given
 * order) of f_lens(|r - r_c|), the distance taken across the window (not
 * periodic); the screen enters Eq. 2 as exp(-i(h l_f/(2 k0) - f_lens)), so the
 * field is multiplied by exp(+i D_f): U <- U exp(i Re D_f - Im D_f). */
void orc_lens_apply(int n, double L, cplx *U, const int32_t *centres, int count, const orc_lens *ls) {
    double dx = L / n;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double dre = 0.0, dim = 0.0;
            for (int c = 0; c < count; ++c) {
                int xc = centres[c] % n, yc = centres[c] / n;
                double r = dx * sqrt((double)(x - xc) * (x - xc) + (double)(y - yc) * (y - yc));
                double fr, fi;
                orc_lens_value(ls, r, &fr, &fi);
                dre += fr;
                dim += fi;
            }
            U[(size_t)y * n + x] *= cexp(I * (dre + I * dim));
        }
}

/* The whole effective-lens screen on U: fluence, Eq. 4 low-pass, trimming and
 * centres, Eqs. 5-6.  Returns the number of lenses and writes their centres
 * (room for n*n), or -1 for a bad argument. */
int orc_effective_lens(const orc_params *p, cplx *U, const orc_lens *ls, int32_t *centres) {
    int n = p->n;
    size_t nn = (size_t)n * n;
    double *w = (double *)malloc(sizeof(double) * nn);
    for (size_t i = 0; i < nn; ++i) w[i] = creal(U[i] * conj(U[i]));
    orc_lens_lowpass(n, p->L, w, ls->l_dif, w);
    int count = orc_lens_centres(w, n, ls->w_l, ls->conn, centres);
    if (count >= 0) orc_lens_apply(n, p->L, U, centres, count, ls);
    free(w);
    return count;
}

/* -------------------------------------------------------------- adjoint -- */

/* Reverse-mode derivative of J(theta, U0) = loss(march(U0, nsteps), D).
 * Gradients use the convention G = dJ/dRe + i dJ/dIm.  For a complex-linear
 * map the gradient pulls back with the Hermitian adjoint; for the pointwise
 * screen w = v exp(s(|v|^2)):
 *   G_v = conj(exp(s)) G_w + 2 Re(conj(G_w) w s'(I)) v,
 *   dJ/dtheta_j += sum Re(conj(G_w) w ds/dtheta_j).
 * The forward states are stored every ckpt steps and each segment is
 * recomputed from its checkpoint in the backward sweep.
 * Returns J; writes dtheta[6] and dU0[n*n]. */
double orc_adjoint(const orc_params *p, const cplx *U0, const double *D, int nsteps, int ckpt,
                   double *dtheta, cplx *dU0) {
    int n = p->n;
    size_t nn = (size_t)n * n;
    if (ckpt < 1) ckpt = 1;
    int nck = (nsteps + ckpt - 1) / ckpt + 1;
    cplx *ck = (cplx *)malloc(sizeof(cplx) * nn * (size_t)nck);
    cplx *U = (cplx *)malloc(sizeof(cplx) * nn);
    memcpy(U, U0, sizeof(cplx) * nn);
    for (int s = 0; s < nsteps; ++s) {
        if (s % ckpt == 0) memcpy(ck + nn * (size_t)(s / ckpt), U, sizeof(cplx) * nn);
        orc_linear(p, U);
        orc_screen(p, U);
    }
    double J = orc_loss(U, D, n);
    double den = 0.0;
    for (size_t i = 0; i < nn; ++i) den += D[i] * D[i];
    /* seed: dJ/dU_M = 4 (|U|^2 - D) U / sum D^2 */
    cplx *G = dU0;
    for (size_t i = 0; i < nn; ++i) {
        double F = creal(U[i]) * creal(U[i]) + cimag(U[i]) * cimag(U[i]);
        G[i] = 4.0 * (F - D[i]) * U[i] / den;
    }
    for (int j = 0; j < 6; ++j) dtheta[j] = 0.0;
    screen_coef c = make_coef(p);
    cplx *seg = (cplx *)malloc(sizeof(cplx) * nn * (size_t)ckpt); /* v of each step */
    for (int c0 = ((nsteps - 1) / ckpt) * ckpt; c0 >= 0; c0 -= ckpt) {
        int c1 = c0 + ckpt < nsteps ? c0 + ckpt : nsteps;
        memcpy(U, ck + nn * (size_t)(c0 / ckpt), sizeof(cplx) * nn);
        for (int s = c0; s < c1; ++s) {
            orc_linear(p, U);
            memcpy(seg + nn * (size_t)(s - c0), U, sizeof(cplx) * nn);
            orc_screen(p, U);
        }
        for (int s = c1 - 1; s >= c0; --s) {
            const cplx *v = seg + nn * (size_t)(s - c0);
            double acc[6] = {0, 0, 0, 0, 0, 0};
            for (size_t i = 0; i < nn; ++i) {
                double In = creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
                cplx e = cexp(screen_exponent(&c, p, In));
                cplx w = v[i] * e;
                cplx gw = G[i];
                cplx ds[6];
                screen_exponent_dtheta(&c, p, In, ds);
                for (int j = 0; j < 6; ++j) acc[j] += creal(conj(gw) * w * ds[j]);
                cplx sp = screen_exponent_dI(&c, p, In);
                G[i] = conj(e) * gw + 2.0 * creal(conj(gw) * w * sp) * v[i];
            }
            for (int j = 0; j < 6; ++j) dtheta[j] += acc[j];
            orc_linear_adjoint(p, G);
        }
    }
    free(seg);
    free(U);
    free(ck);
    return J;
}
