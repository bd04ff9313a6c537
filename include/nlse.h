/*
 * nlse.h -- C ABI of the GB300 (sm_103a) split-step Fourier march of the
 * stationary transverse nonlinear Schroedinger equation (NLSE) of
 * Bulygin & Geints, arXiv 2306.15678.
 *
 * The method (Sec. 2):
 *   Eq. 1   2 i k0 dU/dz = (Lap_perp + eps_k U U* + eps_h[U]) U
 *   Eq. 3   eps_h U = (eps_m (UU*)^K + i k0 alpha_m (UU*)^(K-1)) U
 *           (the printed exponents 2m and 2(m-1) are read as m = K and K-1:
 *           plasma refraction ~ I^K, K-photon absorption ~ I^(K-1) in the field
 *           equation, i.e. dI/dz = -beta_K I^K)
 *   Eq. 2   one z step is the operator exponential split into diffraction
 *           exp(i k_perp^2 dz / (2 k0)) applied in Fourier space and a pointwise
 *           complex phase screen evaluated on the field entering the screen.
 *
 * One call of nlse_step(g, n) advances the field by n Lie steps
 *   U <- v exp(s(|v|^2)),   v = IFFT2( exp(i (kx^2+ky^2) dz/(2 k0)) FFT2(U) ),
 *   s(I) = -i dz/(2 k0) [c_K eps_k I + c_P eps_m I^K + c_A i k0 alpha_m I^(K-1)],
 * with eps_k = 2 k0^2 n2/n0, eps_m = -k0^2 sigma_K rho_nt tau_pl / rho_c,
 * alpha_m = -beta_K, k0 = 2 pi n0 / lambda0 and complex gains
 * c_K = theta[0] + i theta[1], c_P = theta[2] + i theta[3],
 * c_A = theta[4] + i theta[5] (nominal 1, 0, 1, 0, 1, 0).
 *
 * Units: CGS-optical.  Lengths in cm, |U|^2 in W/cm^2, power in W.
 * Field layout everywhere: row-major n x n (row = y, column = x), complex
 * values interleaved (re, im); complex128 for NLSE_FP64 grids, complex64 for
 * NLSE_FP32 grids.  Grid points sit on cell centres x_j = (j - n/2 + 1/2) L/n.
 *
 * Memory ownership: the caller owns every device buffer (the workspace holds
 * the field, the propagator and twiddle tables, reduction partials, the
 * diagnostics history and the adjoint's checkpoints) and the CUDA stream.  The
 * library owns only the opaque host structures it allocates in *_create and
 * frees in *_destroy.  A workspace must outlive its handle and must not be
 * shared by two live handles.
 *
 * Errors: every call returns an nlse_status and never aborts, traps or exits.
 * Arguments are validated before any launch (NLSE_EINVAL, NLSE_EUNSUPPORTED,
 * NLSE_ENOMEM for a workspace that is too small).  Launch failures and
 * asynchronous faults surface as NLSE_ECUDA at the next call that checks
 * them.  A device status word records non-finite readouts (NLSE_ENONFINITE)
 * and bounded waits that ran out (NLSE_ETIMEOUT); calls that synchronise
 * report it.
 *
 * Threading: a handle is bound to the stream given at creation and is not
 * thread-safe; use one handle per host thread.  Calls that do not say
 * "synchronises" only enqueue work on the stream.
 */
#ifndef NLSE_H
#define NLSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nlse_status {
    NLSE_OK = 0,
    NLSE_EINVAL = 1,        /* bad argument (null pointer, bad size, bad value) */
    NLSE_EUNSUPPORTED = 2,  /* valid request outside what this build supports */
    NLSE_ENOMEM = 3,        /* caller's workspace is smaller than required */
    NLSE_ECUDA = 4,         /* a CUDA call or kernel launch failed */
    NLSE_ENONFINITE = 5,    /* a readout found NaN or Inf in the field */
    NLSE_ETIMEOUT = 6,      /* a bounded device-side wait ran out */
    NLSE_ESTATE = 7         /* call out of order (e.g. step before load) */
} nlse_status;

/* terms of Eq. 1-3 (bit mask) */
enum {
    NLSE_KERR = 1u,         /* eps_k |U|^2: Kerr self-focusing */
    NLSE_PLASMA = 2u,       /* eps_m |U|^(2K): plasma defocusing */
    NLSE_MPA = 4u,          /* i k0 alpha_m |U|^(2K-2): multiphoton absorption */
    NLSE_DIFFRACTION = 8u,  /* Lap_perp */
    NLSE_ALL_TERMS = 15u
};

/* arithmetic of the field march; reductions, tables and losses are FP64 in both */
enum { NLSE_FP64 = 0, NLSE_FP32 = 1 };

/* Physical description of one grid (Eq. 1-3, Eq. 7).  Plain old data. */
typedef struct nlse_params {
    int32_t n;            /* points per side: power of two, 8 <= n <= 8192 */
    int32_t K;            /* multiphoton order (Eq. 3 "m"), 1 <= K <= 16 */
    uint32_t terms;       /* NLSE_KERR | NLSE_PLASMA | NLSE_MPA | NLSE_DIFFRACTION */
    int32_t precision;    /* NLSE_FP64 or NLSE_FP32 */
    double L;             /* transverse window side, cm (> 0) */
    double dz;            /* z step, cm (non-zero; negative marches backwards) */
    double lambda0;       /* carrier wavelength, cm */
    double n0;            /* linear refractive index */
    double n2;            /* Kerr index, cm^2/W */
    double sigmaK;        /* K-photon ionisation coefficient, s^-1 cm^(2K) W^-K */
    double rho_nt;        /* neutral density, cm^-3 */
    double rho_c;         /* critical plasma density, cm^-3 */
    double tau_pl;        /* effective pulse duration, s */
    double betaK;         /* K-photon absorption coefficient, cm^(2K-3) W^(1-K) */
    double theta[6];      /* complex screen gains (re, im) for Kerr, plasma, absorption */
    int32_t diag_every;   /* record power and peak every this many steps (0 = never) */
    int32_t scheme;       /* NLSE_LIE or NLSE_STRANG, optionally | NLSE_EXACT_SCREEN */
} nlse_params;

/* Splitting of a step (Eq. 2): NLSE_LIE -- diffraction over dz, then the screen
 * over dz; NLSE_STRANG -- the screen over dz/2, diffraction over dz, the screen
 * over dz/2 (symmetric, second order in dz).  OR NLSE_EXACT_SCREEN in to
 * replace the screen frozen at the entering intensity by the exact pointwise
 * substep of the nonlinear part of Eqs. 1-3: for real gains (theta[1] =
 * theta[3] = theta[5] = 0) and K >= 2 the intensity obeys dI/dz = -c_A beta_K
 * I^K, so I(z) = I0 (1 + (K-1) c_A beta_K I0^(K-1) z)^(-1/(K-1)), and the Kerr
 * and plasma phases are the closed-form integrals of I and I^K over the step
 * (NLSE_EINVAL for complex gains or K < 2).  The batched march and the adjoint
 * take NLSE_LIE only (NLSE_EUNSUPPORTED otherwise). */
enum { NLSE_LIE = 0, NLSE_STRANG = 1, NLSE_EXACT_SCREEN = 2 };

typedef struct nlse_grid nlse_grid;

/* Human-readable name of a status code (static storage, never NULL). */
const char* nlse_status_string(nlse_status s);

/* Library version as major*10000 + minor*100 + patch. */
int32_t nlse_version(void);

/* Bytes of device workspace nlse_create needs for these parameters
 * (field, scratch field, tables, partials, history).  No CUDA call. */
nlse_status nlse_workspace_size(const nlse_params* p, size_t* bytes);

/* Create a grid on the current CUDA device.  `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream); `dev_workspace` is a device pointer of at
 * least nlse_workspace_size() bytes, 256-byte aligned.  Builds the propagator
 * tables P(kx), P(ky) (phase k^2 dz/(2 k0) in FP64, reduced mod 2 pi, then
 * rounded to the grid precision) and the FFT twiddles on the host and copies
 * them into the workspace (asynchronously, on the stream).  *out receives the
 * handle.  Eq. 1-2 (propagator), Eq. 3 (screen coefficients). */
nlse_status nlse_create(const nlse_params* p, void* cuda_stream, void* dev_workspace,
                        size_t workspace_bytes, nlse_grid** out);

/* Load the field U (n x n interleaved complex of the grid precision; host
 * memory if src_on_device == 0, device memory otherwise) and reset the step
 * counter and the diagnostics history.  Eq. 7 supplies the usual initial
 * beams (see the Python helper paper_2306_15678_gb300.beams). */
nlse_status nlse_load_field(nlse_grid* g, const void* src, int src_on_device);

/* Advance the field by nsteps >= 0 Lie steps (Eq. 2), asynchronously on the
 * grid's stream: per step one column pass (FFT_y, multiply by
 * exp(i (kx^2+ky^2) dz/(2k0))/n^2, inverse FFT_y) and one row pass (inverse
 * FFT_x, nonlinear screen, forward FFT_x).  Every diag_every steps the row pass
 * also reduces power and peak into the history. */
nlse_status nlse_step(nlse_grid* g, int32_t nsteps);

/* Same work as nlse_step, with CUDA events recorded on the grid's stream
 * around every launch: adds the summed durations (milliseconds) of the column
 * passes to *col_ms and of the row passes (with their diagnostics reduction)
 * to *row_ms.  Either pointer may be NULL.  Synchronises.  Measurement aid
 * for the per-kernel roofline; the paper has no counterpart. */
nlse_status nlse_step_timed(nlse_grid* g, int32_t nsteps, double* col_ms, double* row_ms);

/* Arithmetic-rate probe: enqueue on cuda_stream one launch of `blocks` blocks
 * of 256 threads, every thread running 8 independent fused multiply-add
 * chains for `iters` rounds (rounded up to a multiple of 16): kind 0 = FP32
 * FMA, 1 = FP64 FMA, 2 = packed FP32x2 FMA (fma.rn.f32x2, two FMAs per
 * instruction).  The caller times the
 * launch (CUDA events on the same stream) to get the peak FMA rate, the
 * denominator of the ALU roofline of the FP64 march.  sink_dev: device
 * buffer of `blocks` 8-byte slots (8-byte aligned) that the kernel may write.
 * NLSE_EINVAL for iters < 1, blocks < 1, a null or misaligned sink or an
 * unknown kind.  Measurement aid; the paper has no counterpart. */
nlse_status nlse_alu_probe(int32_t kind, int32_t iters, int32_t blocks, void* cuda_stream, void* sink_dev);

/* Column tile of the column pass: a width of 1, 2, 4, 8 or 16 columns per
 * block, or'ed with NLSE_COL_TMA for the variant that moves the tile between
 * global and shared memory with bulk tensor copies (cp.async.bulk.tensor,
 * boxes of 512 rows) instead of per-thread loads and stores (n >= 512), and
 * in FP32 with NLSE_COL_R8 for the radix-8 column transform (8 elements per
 * thread, more threads in flight, one more shared-memory exchange; radix 16
 * without it).  The field between the passes is stored in 16-byte units that
 * hold one column's values at two adjacent rows, so a column is a sequence of
 * units.  NLSE_EUNSUPPORTED for a tile this size or precision cannot use.
 * Chosen by the autotuner (default FP32: the narrowest radix-16 staged tile
 * of at least 128 threads); for a given radix the results do not depend on
 * the tile, bit for bit, while the radix changes the rounding (both stay
 * within the stated tolerances).  A bounded wait (1 s) of the staged variant
 * that runs out makes the block skip its tile and sets NLSE_ETIMEOUT in the
 * device status word (nlse_device_status).  The block then waits once more
 * (1 s) for the copy it started; if that copy still has not landed, it may
 * land later in shared memory of another block, so after an NLSE_ETIMEOUT the
 * field of the grid and the results of later kernels on its stream are not to
 * be trusted: destroy the grid and reload. */
enum { NLSE_COL_TMA = 0x100, NLSE_COL_R8 = 0x200 };
nlse_status nlse_set_column_tile(nlse_grid* g, int32_t cols);

/* Radix of the row pass's transforms: 16 (16 elements per thread, the default
 * in FP32) or 8 (8 elements per thread: twice the threads in flight, one more
 * shared-memory exchange per transform); FP64 grids take 8 only.
 * NLSE_ROW_STAGED | 16 (FP32, n >= 2048): radix 16 with persistent blocks, each
 * moving its next row pair into shared memory with one bulk copy while it
 * finishes the current one; bit-identical to radix 16, its wait for a copy
 * bounded as the staged column pass's (NLSE_ETIMEOUT, see
 * nlse_set_column_tile).  NLSE_EUNSUPPORTED otherwise.  Chosen by the
 * autotuner with the column tile; the radix changes the rounding, not the
 * tolerances met.  Finalises pending diagnostics first (enqueued on the grid's
 * stream). */
enum { NLSE_ROW_STAGED = 0x100 };
nlse_status nlse_set_row_radix(nlse_grid* g, int32_t radix);

/* Number of z steps taken since the last load. */
nlse_status nlse_steps_taken(nlse_grid* g, int64_t* steps);

/* Beam power P = sum |U|^2 dx^2 in W, summed in FP64 in a fixed order
 * (deterministic).  Synchronises the stream.  Sec. 3.1 "total pulse energy". */
nlse_status nlse_power(nlse_grid* g, double* watts);

/* Peak intensity max |U|^2 in W/cm^2.  Synchronises.  Sec. 3.1 "I_m". */
nlse_status nlse_peak(nlse_grid* g, double* w_per_cm2);

/* Fluence w = U U* (Sec. 2, before Eq. 4; stationary model), averaged over
 * aligned downsample x downsample blocks (downsample = 1, 2, 4, ... <= n),
 * written as (n/downsample)^2 reals of the grid precision (float for FP32,
 * double for FP64) to dst (host if dst_on_device == 0).  Synchronises when dst
 * is on the host. */
nlse_status nlse_fluence(nlse_grid* g, void* dst, int dst_on_device, int downsample);

/* Copy the current field U (n x n interleaved complex of the grid precision)
 * to dst (host if dst_on_device == 0).  Synchronises when dst is on the host. */
nlse_status nlse_read_field(nlse_grid* g, void* dst, int dst_on_device);

/* Hot areas of the current cross-section (Sec. 3.3: the closed regions where
 * the fluence w = U U* reaches the cut-off w_p, whose number the paper tracks
 * against distance).  A pixel belongs to a region when w >= w_p, both taken in
 * the grid precision (w_p rounded to float for FP32 grids); regions are the
 * connected components of those pixels with `connectivity` = 4 (edge
 * neighbours) or 8 (edges and corners); the window is not periodic.
 *   count   host int32: the number of regions.
 *   labels  NULL, or n*n int32 in row-major order (host if labels_on_device ==
 *           0, else device memory on the grid's stream): -1 outside every
 *           region, else the smallest row-major index (y*n + x) of the pixel's
 *           region, so that labels are unique and independent of the order in
 *           which the device joins pixels.
 * NLSE_EINVAL for a bad argument (w_p not finite, connectivity not 4 or 8);
 * NLSE_ESTATE before a field is loaded.  Synchronises. */
nlse_status nlse_hot_areas(nlse_grid* g, double w_p, int32_t connectivity, int32_t* count,
                           int32_t* labels, int labels_on_device);

/* Pass the current field through a turbulent layer (Sec. 3.3, Eqs. 9-10): the
 * random permittivity screen eps_t enters Eq. 9 beside the other terms, so a
 * layer of the given thickness (cm) multiplies the field by
 * exp(-i thickness eps_t / (2 k0)), k0 = 2 pi n0 / lambda0.  eps_t is built by
 * the spectral method with the step spectrum of Eq. 10, read as amplitude tau
 * for |k| <= k_h (k_h the upper cut-off, rad/cm) and 0 above:
 *   eps_t(y_l, x_j) = Re sum_{q,p} tau [p~^2 + q~^2 <= (k_h L / 2 pi)^2]
 *                     xi[q][p] exp(+2 pi i (p j + q l) / n),
 * p~, q~ the signed bin numbers (p~ = p for p < n/2, else p - n).
 *   xi  n*n complex of the grid precision (interleaved re, im), row q = k_y
 *       bin, column p = k_x bin: the caller's random draws (e.g. complex unit
 *       Gaussians), host if xi_on_device == 0, else device memory that is
 *       only read.
 * Between z steps only; the step count and the recorded history are kept.
 * NLSE_EINVAL for a bad argument (tau, thickness not finite, k_h negative or
 * not finite); NLSE_ESTATE before a field is loaded.  Asynchronous when xi is
 * on the device. */
nlse_status nlse_turbulent_screen(nlse_grid* g, const void* xi, int xi_on_device, double tau,
                                  double k_h, double thickness);

/* Effective lens (Sec. 2, Eqs. 4-6; Fig. 1): the screen that replaces the
 * filamentation region on a sparse grid once the intensity reaches the
 * pre-filamentation level.  Built from the current field:
 *   1. w = U U*; Eq. 4 low-pass w_dif = F^-1 exp(-l_dif k^2) F w (k^2 = kx^2 + ky^2);
 *   2. trimming: the lenses are the connected regions of w_dif >= w_l
 *      (4 or 8 neighbours, window not periodic, compared in grid precision);
 *   3. each lens is centred on its pixel of largest w_dif (first in row-major
 *      order on a tie);
 *   4. Eqs. 5-6: D_f(r) = sum over the centres, in increasing row-major index,
 *      of f_lens(|r - r_c|), with the piecewise radial ansatz of Eq. 6: real
 *      part a_j cos(omega_j r + psi_j) on r_re[j-1] <= r < r_re[j] (r_re[-1] = 0,
 *      j < n_re), imaginary part b_l cos(nu_l r + eta_l) on its own joints r_im,
 *      zero beyond the last joint; distances in cm across the window;
 *   5. the screen enters Eq. 2 as exp(-i(h l_f/(2 k0) - f_lens)): the field is
 *      multiplied by exp(+i D_f) = exp(i Re D_f) exp(-Im D_f).
 * The diffraction over the lens length l_f is the caller's (a diffraction-only
 * grid marched over l_f, or the ordinary march).  FP64 for the ansatz and the
 * phase factor; the low-pass in the grid precision. */
#define NLSE_LENS_SEGMENTS 8
typedef struct {
    double l_dif;          /* cm^2, >= 0 */
    double w_l;            /* W/cm^2, > 0 */
    int32_t connectivity;  /* 4 or 8 */
    int32_t n_re, n_im;    /* segments of the real / imaginary part, 0..8 */
    int32_t reserved;      /* 0 */
    double r_re[NLSE_LENS_SEGMENTS], a[NLSE_LENS_SEGMENTS], omega[NLSE_LENS_SEGMENTS],
        psi[NLSE_LENS_SEGMENTS];
    double r_im[NLSE_LENS_SEGMENTS], b[NLSE_LENS_SEGMENTS], nu[NLSE_LENS_SEGMENTS],
        eta[NLSE_LENS_SEGMENTS];
} nlse_lens;

/* Device scratch the effective lens needs for a grid of these parameters
 * (256-byte aligned by the caller).  Host-only. */
nlse_status nlse_lens_scratch_size(const nlse_params* p, size_t* bytes);

/* Apply the effective lens to the current field (steps 1-5 above).
 *   scratch   caller's device buffer of at least nlse_lens_scratch_size bytes,
 *             256-byte aligned, overwritten; free again when the call returns.
 *   count     host int32: the number of lenses.
 *   centres   NULL, or host int32[capacity]: the centres' row-major indices
 *             (y*n + x), increasing; the first min(count, capacity) are written.
 *   w_dif_out NULL, or device memory for n*n reals of the grid precision: w_dif.
 * The step count and history are kept.  NLSE_EINVAL for a bad argument (joints
 * not positive and increasing, a coefficient not finite, w_l <= 0, ...);
 * NLSE_ENOMEM for a scratch smaller than required; NLSE_ESTATE before a field
 * is loaded.  Synchronises. */
nlse_status nlse_effective_lens(nlse_grid* g, const nlse_lens* lens, void* scratch, size_t scratch_bytes,
                                int32_t* count, int32_t* centres, int32_t capacity, void* w_dif_out);

/* Spatial moments of the current fluence (Eq. 8, the moment measure of the
 * fit): out[k] = sum over the grid of I^p[k] (x^2 + y^2)^q[k] dx^2, I = U U*,
 * on the cell centres x_j = (j - n/2 + 1/2) dx, y likewise (the window centre
 * is the origin).  Eq. 8's Q^m of a beam is M(m, m) (its (UU*)^{2m} read as
 * I^m); M(1, 0) is the power.  count = 1..8, 1 <= p <= 16, 0 <= q <= 16
 * (NLSE_EINVAL otherwise); FP64 sums in a fixed order.  Synchronises. */
nlse_status nlse_moments(nlse_grid* g, int32_t count, const int32_t* p, const int32_t* q, double* out);

/* Copy up to `capacity` recorded (power, peak) pairs, oldest first, into
 * power[] and peak[] (host arrays; either may be NULL) and their count into
 * *count.  Entry i was recorded after (i+1)*diag_every steps.  The history
 * keeps the last 4096 records.  Synchronises. */
nlse_status nlse_history(nlse_grid* g, double* power, double* peak, int32_t capacity,
                         int32_t* count);

/* Read and clear the device status word (synchronises): NLSE_OK,
 * NLSE_ENONFINITE or NLSE_ETIMEOUT. */
nlse_status nlse_device_status(nlse_grid* g);

/* Power P = sum |U|^2 dx^2 (dx = L/n) and peak max |U|^2 of a caller's field,
 * computed without allocating any device memory.  The paper has no
 * counterpart: this serves callers that may not allocate device memory once
 * they are running, such as a service that hands all device memory to its own
 * pool at start-up, or a loop that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree can cause.
 *   field_dev: device pointer, n x n interleaved complex of `precision`
 *              (physical field U, row-major), read only; aligned to one
 *              complex value (16 bytes in FP64, 8 in FP32), else NLSE_EINVAL;
 *   n:         1 <= n <= 8192 rows and columns; larger n returns
 *              NLSE_EUNSUPPORTED before any launch;
 *   out_dev:   device pointer to 2 doubles (8-byte aligned, else NLSE_EINVAL),
 *              receives (power, peak).
 * Enqueued on cuda_stream (a cudaStream_t, NULL = legacy default stream);
 * does not synchronise.  The per-row partial sums live in one 128 KiB
 * __device__ array that every device loading the library keeps until exit and
 * that every call on a device shares: calls that overlap on the GPU (e.g. on
 * two streams) race on it, so serialise them.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
nlse_status nlse_power_peak_noalloc(const void* field_dev, int32_t n, int32_t precision, double L,
                                    void* cuda_stream, double* out_dev);

/* Release the handle (not the caller's workspace).  Synchronises. */
nlse_status nlse_destroy(nlse_grid* g);

/* ------------------------------------------------------------------ batch --
 * Many independent beams (the paper's statistical realisations, Sec. 3.3, and
 * test beams, Sec. 2) of different grid sizes (n = 256..4096, FP32 only)
 * marched together: every z step of every beam runs inside one persistent
 * kernel launch whose blocks pull (step, pass, beam, tile) work items in
 * dependency order.  Waits between items are bounded (timeout_ms); when one
 * runs out the launch stops and nlse_batch_status reports NLSE_ETIMEOUT.  A
 * batched beam is bit-identical to the same beam on its own nlse_grid. */
typedef struct nlse_batch nlse_batch;

/* Launch shape of the persistent kernel (chosen by an autotuner; see the
 * Python package).  threads: 128, 256 or 512 threads per block (sets the rows
 * and columns per tile; 128 needs n <= 2048 and radix 16, NLSE_EUNSUPPORTED
 * otherwise); ctas_per_sm: resident blocks per SM (0 = as many as fit);
 * timeout_ms: bound on every wait; debug_skip_item: test hook -- the work item
 * with this index never reports completion (-1 = none); radix: transform
 * radix of every pass, 16 (or 0: the default; 128 registers per thread) or 8
 * (64 registers, twice the resident warps; a beam of n = 4096 then needs 512
 * threads); per_thread_columns: 0 (default) stages the column tiles of beams
 * with n >= 512 in shared memory with bulk tensor copies, 1 moves every column
 * tile with per-thread loads and stores.  A batched beam is bit-identical to
 * the same beam on its own grid with the same radix for its rows and columns
 * (nlse_set_row_radix, NLSE_COL_R8); the column staging does not change a bit. */
typedef struct nlse_batch_tuning {
    int32_t threads;
    int32_t ctas_per_sm;
    int32_t timeout_ms;
    int64_t debug_skip_item;
    int32_t radix;
    int32_t per_thread_columns;
} nlse_batch_tuning;

/* Device bytes for `count` beams with parameters params[0..count-1].  No CUDA call. */
nlse_status nlse_batch_workspace_size(int32_t count, const nlse_params* params, size_t* bytes);

/* Create (tuning may be NULL for the defaults 256, 0, 2000, -1, 16, 0).  Builds every
 * beam's tables exactly as nlse_create does.  Synchronises. */
nlse_status nlse_batch_create(int32_t count, const nlse_params* params, const nlse_batch_tuning* tuning,
                              void* cuda_stream, void* dev_workspace, size_t workspace_bytes,
                              nlse_batch** out);

/* Load beam `beam`'s field (n x n complex64, host or device) before any step. */
nlse_status nlse_batch_load_field(nlse_batch* b, int32_t beam, const void* src, int src_on_device);

/* Advance every beam nsteps Lie steps in one persistent launch (async). */
nlse_status nlse_batch_step(nlse_batch* b, int32_t nsteps);

/* Capture the launch of nsteps steps into a CUDA graph (counter resets,
 * persistent kernel, step-base update) for nlse_batch_replay. */
nlse_status nlse_batch_capture(nlse_batch* b, int32_t nsteps);

/* Launch the captured graph: every beam advances the captured step count. */
nlse_status nlse_batch_replay(nlse_batch* b);

/* Read and clear the status word (synchronises): NLSE_OK or NLSE_ETIMEOUT. */
nlse_status nlse_batch_status(nlse_batch* b);

/* Steps taken by every beam since creation. */
nlse_status nlse_batch_steps_taken(nlse_batch* b, int64_t* steps);

/* Field of one beam (n x n complex64) to dst (host if dst_on_device == 0). */
nlse_status nlse_batch_read_field(nlse_batch* b, int32_t beam, void* dst, int dst_on_device);

/* Power sum |U|^2 dx^2 of one beam, FP64, deterministic.  Synchronises. */
nlse_status nlse_batch_power(nlse_batch* b, int32_t beam, double* watts);

/* Release the handle (not the workspace).  Synchronises. */
nlse_status nlse_batch_destroy(nlse_batch* b);

/* ---------------------------------------------------------------- adjoint --
 * Gradient of the fluence-mismatch loss of an M-step march,
 *     J(theta, U0) = sum (|U_M|^2 - D)^2 / sum D^2,
 * with respect to the six screen gains theta (Eq. 3 terms; see nlse_params)
 * and the input field U0, by the exact discrete adjoint of the march (the
 * paper fits its effective-lens ansatz with a genetic algorithm, Sec. 2 and
 * Fig. 2; this makes the fit gradient-based).  Gradients follow the convention
 * G = dJ/dRe + i dJ/dIm (PyTorch's for complex leaves).  The forward run keeps
 * the state every ckpt_every steps; the backward sweep recomputes each segment
 * from its checkpoint.  Memory: (2 + ckpt_every + ceil(M/ckpt_every)) fields
 * plus one n x n double target (nlse_adjoint_workspace_size). */
typedef struct nlse_adjoint nlse_adjoint;

/* Device bytes for an adjoint of nsteps >= 1 steps checkpointed every
 * ckpt_every >= 1 steps (values above nsteps act as nsteps).  No CUDA call. */
nlse_status nlse_adjoint_workspace_size(const nlse_params* p, int32_t nsteps, int32_t ckpt_every,
                                        size_t* bytes);

/* Create on the current device; workspace as for nlse_create (256-byte aligned,
 * caller-owned).  Uploads the propagator tables and their conjugates.  Synchronises. */
nlse_status nlse_adjoint_create(const nlse_params* p, int32_t nsteps, int32_t ckpt_every, void* cuda_stream,
                                void* dev_workspace, size_t workspace_bytes, nlse_adjoint** out);

/* Replace the six screen gains (invalidates a pending forward run). */
nlse_status nlse_adjoint_set_theta(nlse_adjoint* a, const double* theta);

/* Launch shape of the forward and backward sweeps: a column-tile code and a
 * row-pass code as for nlse_set_column_tile / nlse_set_row_radix (the radices
 * change the rounding within the stated tolerances; tiles of one radix and the
 * staged row pass do not change a bit).  NLSE_EUNSUPPORTED for a code the grid
 * size or precision does not offer; nothing is changed then.  Invalidates a
 * pending forward run. */
nlse_status nlse_adjoint_set_launch(nlse_adjoint* a, int32_t cols, int32_t row_radix);

/* Target fluence D: n x n doubles (host or device), copied in; sum D^2 must be
 * positive (NLSE_EINVAL otherwise).  Synchronises. */
nlse_status nlse_adjoint_set_target(nlse_adjoint* a, const double* target, int on_device);

/* March U0 (n x n interleaved complex of the grid precision, host or device)
 * M steps with checkpoints, then evaluate J (FP64) into *loss and seed the
 * adjoint.  NLSE_ESTATE without a target.  Synchronises. */
nlse_status nlse_adjoint_forward(nlse_adjoint* a, const void* U0, int on_device, double* loss);

/* Backward sweep after nlse_adjoint_forward: dtheta[6] (host) receives dJ/dtheta
 * summed in FP64 in a fixed order; dU0 (n x n complex of the grid precision,
 * host or device) receives dJ/dU0.  Consumes the forward run (NLSE_ESTATE if
 * there is none).  Synchronises. */
nlse_status nlse_adjoint_backward(nlse_adjoint* a, double* dtheta, void* dU0, int dU0_on_device);

/* Release the handle (not the workspace).  Synchronises. */
nlse_status nlse_adjoint_destroy(nlse_adjoint* a);

#ifdef __cplusplus
}
#endif

#endif /* NLSE_H */
