"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the passage of arXiv 2306.15678 (or the mathematical fact) it
checks.  None of them compares the oracle with itself: the expected values come
from brute force, a library routine, a closed form, an exact identity or a
conservation law.  The last group plants a mistake in a copy of the oracle and
checks that a pin fails.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2306_15678_gb300 import beams, configs

RNG = np.random.default_rng(12345)


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def crand(shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# --------------------------------------------------------------- FFT (Eq. 2)

@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_fft2_matches_brute_force_dft(n):
    """O(N^4) DFT written from its definition X[ky,kx] = sum a[y,x] e^{-2pi i (ky y + kx x)/N}."""
    a = crand((n, n))
    idx = np.arange(n)
    expected = np.zeros((n, n), dtype=np.complex128)
    for ky in range(n):
        for kx in range(n):
            ph = np.exp(-2j * np.pi * (ky * idx[:, None] + kx * idx[None, :]) / n)
            expected[ky, kx] = np.sum(a * ph)
    assert rel_max(oracle.fft2(a), expected) < 1e-13
    # inverse: e^{+2pi i ...} / N^2
    back = np.zeros_like(expected)
    for y in range(n):
        for x in range(n):
            ph = np.exp(2j * np.pi * (y * idx[:, None] + x * idx[None, :]) / n)
            back[y, x] = np.sum(a * ph) / (n * n)
    assert rel_max(oracle.fft2(a, inverse=True), back) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 8, 32, 64])
def test_fft1_matches_brute_force_dft(n):
    a = crand(n)
    k = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(k, k) / n)
    assert rel_max(oracle.fft1(a), W @ a) < 1e-13
    assert rel_max(oracle.fft1(a, inverse=True), np.conj(W) @ a / n) < 1e-13


def test_fft2_matches_numpy_at_256():
    a = crand((256, 256))
    assert rel_max(oracle.fft2(a), np.fft.fft2(a)) < 1e-13
    assert rel_max(oracle.fft2(a, inverse=True), np.fft.ifft2(a)) < 1e-13


def test_fft2_parseval_and_roundtrip():
    a = crand((128, 128))
    A = oracle.fft2(a)
    lhs = math.fsum(np.abs(A).ravel() ** 2)
    rhs = 128 * 128 * math.fsum(np.abs(a).ravel() ** 2)
    assert abs(lhs / rhs - 1) < 1e-14
    assert rel_max(oracle.fft2(A, inverse=True), a) < 1e-14


# ------------------------------------------------- diffraction (Eq. 1-2)

def gaussian_closed_form(n, L, w0, A, k0, z):
    """Gaussian beam of 2 i k0 dU/dz = Lap U (the paper's sign convention):
    U = A/(1 - i z/zR) exp(-r^2 / (w0^2 (1 - i z/zR))), zR = k0 w0^2 / 2."""
    x = beams.cell_centres(n, L)
    r2 = x[:, None] ** 2 + x[None, :] ** 2
    zR = k0 * w0 * w0 / 2.0
    q = 1.0 - 1j * z / zR
    return A / q * np.exp(-r2 / (w0 * w0 * q))


def test_linear_march_matches_closed_form_gaussian():
    """256^2, 25.6 mm window, w0 = 2 mm, 200 steps of 1 cm with diffraction only."""
    cfg = configs.cfg_plain_fp64()
    cfg = dict(cfg, terms=configs.DIFFRACTION)
    b = cfg["beam"]
    U0 = beams.gaussian_beam(cfg["n"], cfg["L"], b["w0"], b["P"])
    U, pw, _ = oracle.march(U0, cfg, 200)
    k0 = 2 * math.pi / cfg["lambda0"]
    A = math.sqrt(2 * b["P"] / (math.pi * b["w0"] ** 2))
    ref = gaussian_closed_form(cfg["n"], cfg["L"], b["w0"], A, k0, 200 * cfg["dz"])
    assert rel_l2(U, ref) < 1e-12
    # the opposite propagator sign gives the conjugate-convention beam, far off
    bad = gaussian_closed_form(cfg["n"], cfg["L"], b["w0"], A, -k0, 200 * cfg["dz"])
    assert rel_l2(U, bad) > 1e-2
    assert np.max(np.abs(pw / pw[0] - 1)) < 1e-13


def test_propagator_is_unimodular_and_even():
    cfg = configs.physics(32, 1.0, 3.0, configs.DIFFRACTION)
    P = oracle.propagator(cfg)
    assert np.max(np.abs(np.abs(P) - 1)) < 1e-15
    # k -> -k symmetry (index m -> N - m) in both dimensions
    m = (-np.arange(32)) % 32
    assert rel_max(P[m][:, m], P) < 1e-15
    assert rel_max(P.T, P) < 1e-15
    # phase at bin (0, 1): (2 pi / L)^2 dz / (2 k0)
    k0 = 2 * math.pi / cfg["lambda0"]
    expect = (2 * math.pi / cfg["L"]) ** 2 * cfg["dz"] / (2 * k0)
    assert abs(np.angle(P[0, 1]) - (expect % (2 * math.pi) if expect < math.pi else
                                    math.remainder(expect, 2 * math.pi))) < 1e-12


# -------------------------------------------------- screen (Eq. 2 and Eq. 3)

def field_with_intensity(n, Imax, rng):
    return np.sqrt(Imax) * (rng.uniform(0.05, 1.0, (n, n)) *
                            np.exp(1j * rng.uniform(-np.pi, np.pi, (n, n))))


def test_kerr_screen_exact_phase_identity():
    """Kerr only, no diffraction: |U_out| = |v| and arg(U_out/v) = -k0 n2 |v|^2 dz."""
    cfg = configs.physics(32, 1.0, 0.5, configs.KERR)
    v = field_with_intensity(32, 3e12, np.random.default_rng(1))
    U = oracle.screen(v, cfg)
    I = np.abs(v) ** 2
    k0 = 2 * math.pi / cfg["lambda0"]
    assert rel_max(np.abs(U), np.abs(v)) < 1e-15
    phase = np.angle(U / v)
    expect = np.angle(np.exp(-1j * k0 * cfg["n2"] * I * cfg["dz"]))
    assert np.max(np.abs(phase - expect)) < 1e-12


def test_screen_gain_convention_on_kerr():
    """Complex gain c_K = theta0 + i theta1 on the Kerr screen: the imaginary part
    turns the phase into an amplitude factor exp(theta1 k0 n2 I dz)."""
    th = (0.7, 0.3, 1.0, 0.0, 1.0, 0.0)
    cfg = configs.physics(16, 1.0, 0.5, configs.KERR, theta=th)
    v = field_with_intensity(16, 1e12, np.random.default_rng(2))
    U = oracle.screen(v, cfg)
    I = np.abs(v) ** 2
    a = 2 * math.pi / cfg["lambda0"] * cfg["n2"] * cfg["dz"] * I
    assert rel_max(np.abs(U) / np.abs(v), np.exp(0.3 * a)) < 1e-14
    assert np.max(np.abs(np.angle(U / v) - np.angle(np.exp(-1j * 0.7 * a)))) < 1e-12


def test_plasma_screen_pure_defocusing_phase():
    """Plasma only: |U| kept, phase +(k0 sigma_K rho_nt tau_pl / (2 rho_c)) I^K dz."""
    cfg = configs.physics(16, 1.0, 0.5, configs.PLASMA)
    v = field_with_intensity(16, 6e13, np.random.default_rng(3))
    U = oracle.screen(v, cfg)
    I = np.abs(v) ** 2
    k0 = 2 * math.pi / cfg["lambda0"]
    ph = k0 * cfg["sigmaK"] * cfg["rho_nt"] * cfg["tau_pl"] / (2 * cfg["rho_c"]) * I ** 8 * cfg["dz"]
    assert ph.max() > 0.5  # the test exercises a sizeable phase
    assert rel_max(np.abs(U), np.abs(v)) < 1e-15
    assert np.max(np.abs(np.angle(U / v) - np.angle(np.exp(1j * ph)))) < 1e-11


def test_mpa_screen_exact_attenuation():
    """Absorption only: I_out = I exp(-beta_K I^(K-1) dz), phase kept."""
    cfg = configs.physics(16, 1.0, 5.0, configs.MPA)
    v = field_with_intensity(16, 6e13, np.random.default_rng(4))
    U = oracle.screen(v, cfg)
    I = np.abs(v) ** 2
    expect = I * np.exp(-cfg["betaK"] * I ** 7 * cfg["dz"])
    assert (expect / I).min() < 0.9
    assert rel_max(np.abs(U) ** 2, expect) < 1e-14
    assert np.max(np.abs(np.angle(U / v))) < 1e-14


def test_mpa_march_converges_to_ode_closed_form():
    """dI/dz = -beta I^K has I(z) = I0 (1 + (K-1) beta I0^(K-1) z)^(-1/(K-1)); the
    frozen-intensity screen converges to it at first order in dz."""
    I0, z = 1e14, 2.0
    v = np.full((4, 4), math.sqrt(I0), dtype=np.complex128)
    exact = I0 * (1 + 7 * configs.BETA_K * I0 ** 7 * z) ** (-1 / 7)
    errs = []
    for m in (40, 80, 160, 320):
        cfg = configs.physics(4, 1.0, z / m, configs.MPA)
        U, _, _ = oracle.march(v, cfg, m)
        errs.append(abs(np.abs(U[0, 0]) ** 2 / exact - 1))
    assert exact / I0 < 0.6
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)
    assert errs[-1] < 2e-2


# ------------------------------------------------------ march invariants

def small_cfg(n, terms, nsteps, power_pcr=10.0, L=2.56, w0=0.2, dz=1.0, noise=True):
    cfg = configs.physics(n, L, dz, terms)
    b = dict(w0=w0, P=power_pcr * configs.critical_power(), amp=0.05 if noise else 0.0,
             ell_cells=3.0, seed=7 if noise else None, phase=0.0, phase_seed=None)
    cfg.update(beam=b, nsteps=nsteps)
    return cfg


def test_lossless_march_conserves_power():
    """Kerr + diffraction (Eq. 1 with eps_h = 0) conserves power to rounding."""
    cfg = small_cfg(128, configs.KERR | configs.DIFFRACTION, 100)
    U0 = beams.make_field(cfg)
    U, pw, pk = oracle.march(U0, cfg, 100)
    assert pk[-1] > 1.2 * pk[0]  # self-focusing is active
    assert np.max(np.abs(pw / pw[0] - 1)) < 1e-12


def test_time_reversal_recovers_input():
    """Lossless step N(dz) L(dz) is undone by L(-dz) N(-dz)."""
    cfg = small_cfg(64, configs.KERR | configs.PLASMA | configs.DIFFRACTION, 30,
                    power_pcr=60.0, w0=0.25)
    U0 = beams.make_field(cfg)
    U, _, pk = oracle.march(U0, cfg, 30)
    back = dict(cfg, dz=-cfg["dz"])
    for _ in range(30):
        U = oracle.screen(U, back)
        U = oracle.linear(U, back)
    assert rel_l2(U, U0) < 1e-11


def strang_case(M, Z=10.0, terms=configs.KERR | configs.DIFFRACTION):
    cfg = configs.physics(64, 0.64, Z / M, terms)
    cfg["beam"] = dict(w0=0.05, P=10.0 * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=3,
                       phase=0.0, phase_seed=None)
    return cfg


def test_strang_is_second_order_and_lie_first_order():
    """Symmetric splitting of the step (Eq. 2: half screen, diffraction, half
    screen) has a global error O(dz^2), the Lie step O(dz): halving dz over a
    fixed 10 cm divides the error by ~4 and ~2 (Kerr + diffraction, the peak
    doubles over the distance)."""
    U0 = beams.make_field(strang_case(1))
    ref, _, _ = oracle.march(U0, strang_case(640), 640, scheme="strang")
    for scheme, ratio in (("strang", 4.0), ("lie", 2.0)):
        err = [rel_l2(oracle.march(U0, strang_case(M), M, scheme=scheme)[0], ref) for M in (10, 20, 40)]
        for a, b in zip(err, err[1:]):
            assert abs(a / b / ratio - 1) < 0.1, (scheme, err)
    assert rel_l2(oracle.march(U0, strang_case(10), 10, scheme="strang")[0], ref) < \
        0.2 * rel_l2(oracle.march(U0, strang_case(10), 10, scheme="lie")[0], ref)


def test_strang_step_is_time_symmetric():
    """Lossless symmetric step: S(-dz) S(dz) is the identity (the half screens
    keep |U| and the diffraction step is unitary), to rounding."""
    cfg = strang_case(30, terms=configs.KERR | configs.PLASMA | configs.DIFFRACTION)
    U0 = beams.make_field(cfg)
    U, _, _ = oracle.march(U0, cfg, 30, scheme="strang")
    back, _, _ = oracle.march(U, dict(cfg, dz=-cfg["dz"]), 30, scheme="strang")
    assert rel_l2(U, U0) > 1e-3
    assert rel_l2(back, U0) < 1e-11


def test_mpa_discrete_energy_balance():
    """With absorption the power after a step is sum I_v exp(-beta I_v^(K-1) dz) dx^2
    where v is the diffracted field (the linear step is unitary)."""
    cfg = small_cfg(64, configs.ALL_TERMS, 1, power_pcr=400.0, w0=0.12, dz=2.0)
    U = beams.make_field(cfg)
    dx2 = (cfg["L"] / cfg["n"]) ** 2
    lost = 0.0
    for _ in range(6):
        v = oracle.linear(U, cfg)
        assert abs(oracle.power(v, cfg["L"]) / oracle.power(U, cfg["L"]) - 1) < 1e-13
        Iv = np.abs(v) ** 2
        expect = math.fsum((Iv * np.exp(-cfg["betaK"] * Iv ** 7 * cfg["dz"])).ravel()) * dx2
        U, pw, _ = oracle.march(U, cfg, 1)
        assert abs(pw[1] / expect - 1) < 1e-13
        lost = max(lost, 1 - pw[1] / pw[0])
    assert lost > 1e-6  # absorption is active in this case


def test_radial_beam_keeps_mirror_and_transpose_symmetry():
    """A radially symmetric input stays symmetric under x<->y and x -> -x (cell-centred
    grid: j -> N-1-j).  Checked before the collapse, where rounding asymmetries
    are not yet amplified (they grow to 1e-10 within ten more steps)."""
    cfg = small_cfg(64, configs.ALL_TERMS, 4, power_pcr=200.0, w0=0.25, dz=20.0, noise=False)
    U0 = beams.make_field(cfg)
    U, _, pk = oracle.march(U0, cfg, 4)
    assert pk[-1] > 2 * pk[0]
    scale = np.max(np.abs(U))
    assert np.max(np.abs(U - U.T)) / scale < 1e-12
    assert np.max(np.abs(U - U[::-1, :])) / scale < 1e-12
    assert np.max(np.abs(U - U[:, ::-1])) / scale < 1e-12


def test_linear_operator_adjoint_dot_product():
    """<L a, b> = <a, L^H b> with L^H = IFFT2 conj(P) FFT2 = L(-dz)."""
    cfg = configs.physics(32, 1.0, 7.0, configs.DIFFRACTION)
    rng = np.random.default_rng(5)
    a, b = crand((32, 32), rng), crand((32, 32), rng)
    lhs = np.vdot(oracle.linear(a, cfg), b)
    rhs = np.vdot(a, oracle.linear(b, dict(cfg, dz=-cfg["dz"])))
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


# --------------------------------------------------------------- readouts

def test_power_peak_fluence_loss():
    rng = np.random.default_rng(6)
    U = crand((64, 64), rng) * 1e5
    L = 3.2
    dx2 = (L / 64) ** 2
    assert abs(oracle.power(U, L) / (math.fsum((np.abs(U) ** 2).ravel()) * dx2) - 1) < 1e-15
    assert oracle.peak(U) == pytest.approx(float(np.max(np.abs(U) ** 2)), rel=1e-15)
    F8 = oracle.fluence(U, 8)
    brute = np.zeros((8, 8))
    for R in range(8):
        for C in range(8):
            brute[R, C] = sum(abs(U[R * 8 + r, C * 8 + c]) ** 2
                              for r in range(8) for c in range(8)) / 64
    assert rel_max(F8, brute) < 1e-14
    D = np.abs(crand((64, 64), rng)) ** 2
    assert oracle.loss(np.sqrt(D), D) < 1e-28
    assert oracle.loss(np.zeros((64, 64)), D) == pytest.approx(1.0, rel=1e-14)
    Us = crand((4, 4), rng)
    Ds = np.abs(crand((4, 4), rng))
    num = sum((abs(Us[i, j]) ** 2 - Ds[i, j]) ** 2 for i in range(4) for j in range(4))
    den = sum(Ds[i, j] ** 2 for i in range(4) for j in range(4))
    assert oracle.loss(Us, Ds) == pytest.approx(num / den, rel=1e-14)


# ---------------------------------------------------------------- adjoint

def adjoint_case():
    cfg = small_cfg(32, configs.ALL_TERMS, 12, power_pcr=300.0, L=1.6, w0=0.12, dz=3.0)
    U0 = beams.make_field(cfg)
    other = small_cfg(32, configs.ALL_TERMS, 12, power_pcr=250.0, L=1.6, w0=0.14, dz=3.0)
    D = np.abs(beams.make_field(other)) ** 2
    return cfg, U0, D


def loss_of(cfg, U0, D, nsteps):
    U, _, _ = oracle.march(U0, cfg, nsteps, record=False)
    return oracle.loss(U, D)


def test_adjoint_theta_gradient_matches_central_differences():
    cfg, U0, D = adjoint_case()
    J, dth, _ = oracle.adjoint(U0, D, cfg, 12, ckpt=5)
    _, _, pk = oracle.march(U0, cfg, 12)
    assert pk.max() > 2e13  # plasma and absorption matter along this path
    assert J == pytest.approx(loss_of(cfg, U0, D, 12), rel=1e-14)
    def central(j, h):
        tp = list(cfg["theta"]); tp[j] += h
        tm = list(cfg["theta"]); tm[j] -= h
        return (loss_of(dict(cfg, theta=tuple(tp)), U0, D, 12) -
                loss_of(dict(cfg, theta=tuple(tm)), U0, D, 12)) / (2 * h)

    h = 1e-4
    for j in range(6):
        # central differences at h and h/2, Richardson-extrapolated (error O(h^4))
        fd = (4 * central(j, h / 2) - central(j, h)) / 3
        assert abs(dth[j] - fd) <= 1e-7 * max(abs(fd), 1e-3 * np.max(np.abs(dth))), (j, dth[j], fd)


def test_adjoint_field_gradient_matches_directional_difference():
    cfg, U0, D = adjoint_case()
    _, _, dU0 = oracle.adjoint(U0, D, cfg, 12, ckpt=4)
    rng = np.random.default_rng(8)
    for _ in range(2):
        d = crand(U0.shape, rng) * np.abs(U0).max()
        def central(h):
            return (loss_of(cfg, U0 + h * d, D, 12) - loss_of(cfg, U0 - h * d, D, 12)) / (2 * h)
        h = 2e-5
        fd = (4 * central(h / 2) - central(h)) / 3
        an = float(np.real(np.vdot(dU0, d)))
        assert abs(an - fd) < 1e-7 * abs(fd), (an, fd)


def test_adjoint_independent_of_checkpoint_spacing():
    cfg, U0, D = adjoint_case()
    J1, t1, g1 = oracle.adjoint(U0, D, cfg, 12, ckpt=1)
    J2, t2, g2 = oracle.adjoint(U0, D, cfg, 12, ckpt=7)
    assert J1 == J2
    assert np.array_equal(t1, t2)
    assert np.array_equal(g1, g2)


# ------------------------------------------- printed constants (golden file)

def golden():
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "printed_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


def test_critical_power_reproduces_printed_ratio():
    """380 GW = 112 Pcr (Sec. 3.2) is lambda^2/(2 pi n0 n2) at n2 = 3.0e-19."""
    g = golden()
    pcr = configs.critical_power(g["lambda0_cm"], 1.0, 3.0e-19)
    assert pcr == pytest.approx(g["P0_W"] / g["P0_over_Pcr"], rel=2e-3)
    # at the build's n2 = 3.2e-19 the value stays near the 4-7 GW range quoted in Sec. 2
    assert 0.75 * g["Pcr_low_W"] < configs.critical_power() < g["Pcr_high_W"]


def test_pulse_duration_and_thresholds_from_printed_values():
    g = golden()
    assert configs.TAU_PL == pytest.approx(g["pulse_energy_J"] / g["peak_power_W"], rel=1e-12)
    assert configs.W_PF == g["wpf_low_Wcm2"]
    assert configs.LAMBDA0 == g["lambda0_cm"]


# --------------------------------------------------------- input generator

def test_input_generator_power_and_noise_statistics():
    b = configs.cfg_plain_fp64()["beam"]
    U = beams.gaussian_beam(256, 2.56, b["w0"], b["P"])
    dx2 = (2.56 / 256) ** 2
    assert math.fsum((np.abs(U) ** 2).ravel()) * dx2 == pytest.approx(b["P"], rel=1e-12)
    eta = beams.smoothed_noise(128, 4.0, 1)
    assert abs(eta.mean()) < 1e-12 and abs(eta.std() - 1) < 1e-12
    assert np.array_equal(eta, beams.smoothed_noise(128, 4.0, 1))
    # correlation: neighbouring cells strongly correlated at l = 4 cells
    c = np.mean(eta * np.roll(eta, 1, axis=1))
    assert c > 0.8


# ------------------------------------------------ hot areas (Sec. 3.3)

def test_hot_areas_hand_made_patterns():
    """Closed regions with w >= w_p, counted by hand: none, one, a ring (one
    region around a hole), a 4-connected chain, diagonal touching (two regions
    with edge neighbours, one with corner neighbours), a checkerboard."""
    z = np.zeros((8, 8))
    assert oracle.hot_areas(z, 0.5)[0] == 0
    assert oracle.hot_areas(z + 1, 0.5)[0] == 1
    ring = np.zeros((8, 8)); ring[1:6, 1:6] = 1; ring[2:5, 2:5] = 0
    assert oracle.hot_areas(ring, 0.5, 4)[0] == 1
    diag = np.zeros((8, 8)); diag[1, 1] = diag[2, 2] = 1
    assert oracle.hot_areas(diag, 0.5, 4)[0] == 2
    assert oracle.hot_areas(diag, 0.5, 8)[0] == 1
    board = np.indices((8, 8)).sum(axis=0) % 2 == 0
    assert oracle.hot_areas(board.astype(float), 0.5, 4)[0] == 32
    assert oracle.hot_areas(board.astype(float), 0.5, 8)[0] == 1
    edge = np.zeros((8, 8)); edge[0, :] = 1; edge[7, :] = 1  # not joined across the window edge
    assert oracle.hot_areas(edge, 0.5)[0] == 2
    w = np.array([[1.0, 0.999999], [0.0, 2.0]])
    assert oracle.hot_areas(w, 1.0, 4)[0] == 2      # w >= w_p, the threshold value included
    _, lab = oracle.hot_areas(w, 1.0, 4)
    assert lab.tolist() == [[0, -1], [-1, 3]]


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("density", [0.3, 0.55, 0.6, 0.8])
def test_hot_areas_match_library_labelling(conn, density):
    """Random masks near and away from the percolation threshold: the count and
    the partition agree with scipy.ndimage.label (a library routine), and each
    label is the smallest index of its region."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(int(density * 100) + conn)
    w = rng.random((96, 96))
    mask = w >= 1 - density
    structure = np.ones((3, 3)) if conn == 8 else None
    ref, nref = ndimage.label(mask, structure=structure)
    count, lab = oracle.hot_areas(w, 1 - density, conn)
    assert count == nref
    assert np.array_equal(lab >= 0, mask)
    pairs = set(zip(lab[mask].tolist(), ref[mask].tolist()))
    assert len(pairs) == nref  # one-to-one between the two labellings
    idx = np.arange(96 * 96).reshape(96, 96)
    for l in np.unique(lab[mask]):
        assert l == idx[lab == l].min()


# ---------------------------------------- turbulent screen (Eqs. 9-10)

def test_turbulent_eps_single_spectral_line():
    """One random draw at bin (q0, p0) inside the cut-off: the screen is the
    single plane wave Re(tau xi e^{2 pi i (p0 x + q0 y)/n}) (the inverse DFT of
    a delta, evaluated here by direct cos/sin); a draw outside the cut-off
    (|k| > k_h) gives no screen at all."""
    n = 32
    cfg = configs.physics(n, 0.64, 1e-3, configs.KERR)
    kunit = 2 * math.pi / cfg["L"]
    for q0, p0 in [(0, 0), (3, 5), (n - 2, 7), (n // 2, 1)]:
        xi = np.zeros((n, n), complex)
        a = 0.7 - 1.3j
        xi[q0, p0] = a
        eps = oracle.turbulent_eps(xi, cfg, 2.5, 40.0 * kunit)
        y, x = np.indices((n, n))
        ph = 2 * math.pi * (p0 * x + q0 * y) / n
        expect = 2.5 * (a.real * np.cos(ph) - a.imag * np.sin(ph))
        assert np.max(np.abs(eps - expect)) < 1e-12
    xi = np.zeros((n, n), complex)
    xi[0, 6] = xi[n - 4, n - 5] = 1.0  # |k| = 6 and sqrt(41) bins
    assert np.max(np.abs(oracle.turbulent_eps(xi, cfg, 1.0, 5.5 * kunit))) == 0.0
    assert np.max(np.abs(oracle.turbulent_eps(xi, cfg, 1.0, 6.5 * kunit))) > 0.5


def test_turbulent_eps_cut_off_is_a_disc_in_k():
    """Step spectrum theta(k_h - |k|): the screen's own 2D spectrum (numpy's
    FFT) is tau xi on the bins with p~^2 + q~^2 <= (k_h L/2 pi)^2 (up to the
    Hermitian part, since eps_t is real) and zero outside; its mean is
    Re(tau xi[0, 0])."""
    n = 64
    cfg = configs.physics(n, 0.64, 1e-3, configs.KERR)
    rng = np.random.default_rng(8)
    xi = crand((n, n), rng)
    kunit = 2 * math.pi / cfg["L"]
    eps = oracle.turbulent_eps(xi, cfg, 3.0, 9.3 * kunit)
    spec = np.fft.fft2(eps) / n ** 2  # eps = sum of e^{+i k r} terms: the forward DFT / n^2 recovers them
    m = np.fft.fftfreq(n, 1.0 / n)
    inside = (m[None, :] ** 2 + m[:, None] ** 2) <= 9.3 ** 2
    herm = 0.5 * (3.0 * xi * inside + np.conj(np.roll(np.flip(3.0 * xi * inside), 1, axis=(0, 1))))
    assert np.max(np.abs(spec - herm)) < 1e-12
    assert abs(eps.mean() - 3.0 * xi[0, 0].real) < 1e-12


def test_turbulent_layer_acts_like_the_kerr_term():
    """Eq. 9 adds eps_t to the same permittivity bracket as the Kerr term of
    Eq. 1: a turbulent layer whose screen equals eps_k |U|^2 over a thickness dz
    must reproduce the pinned Kerr screen over dz exactly.  The draws that make
    eps_t = eps_k |U|^2 are its 2D spectrum (numpy FFT / n^2), cut-off above
    every bin.  The layer is a pure phase: |U| is unchanged."""
    n = 32
    cfg = configs.physics(n, 0.64, 0.37, configs.KERR)
    v = field_with_intensity(n, 2e12, np.random.default_rng(4))
    k0 = 2 * math.pi * cfg["n0"] / cfg["lambda0"]
    eps_k = 2 * k0 * k0 * cfg["n2"] / cfg["n0"]
    xi = np.fft.fft2(eps_k * np.abs(v) ** 2) / n ** 2
    kbig = 2 * math.pi / cfg["L"] * n
    U = oracle.turbulent_screen(v, xi, cfg, 1.0, kbig, cfg["dz"])
    assert rel_max(np.abs(U), np.abs(v)) < 1e-14
    assert rel_max(U, oracle.screen(v, cfg)) < 1e-10


# ------------------------------------- exact pointwise substep (Eqs. 1-3)

def rk4_point(u, cfg, dz, nsub=4000):
    """The pointwise nonlinear equation of Eqs. 1-3 integrated by RK4 with
    nsub substeps: dU/dz = [-(i/2k0)(c_K eps_k I + c_P eps_m I^K)
    - (c_A beta_K / 2) I^(K-1)] U (real gains)."""
    k0 = 2 * math.pi * cfg["n0"] / cfg["lambda0"]
    eps_k = 2 * k0 * k0 * cfg["n2"] / cfg["n0"]
    eps_m = -k0 * k0 * cfg["sigmaK"] * cfg["rho_nt"] * cfg["tau_pl"] / cfg["rho_c"]
    th, K, t = cfg["theta"], cfg["K"], cfg["terms"]

    def f(U):
        I = np.abs(U) ** 2
        br = (th[0] * eps_k * I if t & configs.KERR else 0) + (th[2] * eps_m * I ** K if t & configs.PLASMA else 0)
        damp = (th[4] * cfg["betaK"] / 2 * I ** (K - 1)) if t & configs.MPA else 0
        return (-1j / (2 * k0) * br - damp) * U

    h = dz / nsub
    for _ in range(nsub):
        k1 = f(u)
        k2 = f(u + h / 2 * k1)
        k3 = f(u + h / 2 * k2)
        k4 = f(u + h * k3)
        u = u + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return u


@pytest.mark.parametrize("K", [2, 3, 8])
def test_exact_substep_matches_rk4(K):
    """The exact substep against an RK4 solution of the same pointwise
    equation (all three terms, gains 0.9 / 0.05 / 1.5, intensities from weak to
    strongly absorbing)."""
    cfg = dict(configs.physics(4, 1.0, 0.8, configs.KERR | configs.PLASMA | configs.MPA,
                               theta=(0.9, 0.0, 0.05, 0.0, 1.5, 0.0)), K=K, screen="exact")
    if K != 8:  # keep absorption and plasma O(1) over the step for the other orders
        cfg["betaK"] = 0.3 / (3e13 ** (K - 1))
        cfg["sigmaK"] = cfg["sigmaK"] * 3e13 ** (8 - K)
    I = np.array([1e11, 2e13, 5e13, 7e13])
    v = (np.sqrt(I) * np.exp(1j * np.array([0.1, 1.0, 2.0, -2.5]))).astype(complex)
    out = oracle.screen(np.tile(v, (4, 1)), cfg)[0]
    ref = rk4_point(v.copy(), cfg, cfg["dz"])
    assert np.max(np.abs(out - ref) / np.abs(v)) < 1e-10
    assert np.max(np.abs(out) / np.abs(v)) <= 1.0 and np.min(np.abs(out) / np.abs(v)) < 0.95


def test_exact_substep_without_absorption_is_the_frozen_screen():
    """With no absorption the intensity is constant over the step, so the
    exact substep and the frozen screen of Eq. 2 agree exactly (up to rounding)."""
    cfg = configs.physics(16, 1.0, 0.5, configs.KERR | configs.PLASMA, theta=(0.9, 0.0, 1.1, 0.0, 1.0, 0.0))
    v = field_with_intensity(16, 4e13, np.random.default_rng(7))
    a = oracle.screen(v, cfg)
    b = oracle.screen(v, dict(cfg, screen="exact"))
    assert rel_max(b, a) < 1e-13


def test_exact_and_frozen_screens_differ_at_second_order():
    """Both are consistent with the pointwise equation: their one-step
    difference falls by 4 when dz halves."""
    base = configs.physics(8, 1.0, 0.4, configs.ALL_TERMS)
    v = field_with_intensity(8, 5e13, np.random.default_rng(8))
    d = []
    for dz in (0.4, 0.2, 0.1):
        c = dict(base, dz=dz)
        d.append(np.max(np.abs(oracle.screen(v, dict(c, screen="exact")) - oracle.screen(v, c))))
    assert 3.6 < d[0] / d[1] < 4.4 and 3.6 < d[1] / d[2] < 4.4


# ------------------------------------------------ moments (Eq. 8)

def test_moments_gaussian_closed_form():
    """Eq. 8 moments of a Gaussian beam I = I0 exp(-2 r^2/w0^2), centred on the
    window: int I^p r^{2q} = I0^p pi q! (w0^2 / (2 p))^(q+1) (the rectangle rule
    on the cell centres is exact to rounding for a resolved Gaussian); M(1, 0)
    is the power."""
    n, L, w0 = 128, 1.28, 0.12
    c = beams.cell_centres(n, L)
    X, Y = np.meshgrid(c, c)
    I0 = 3e11
    U = np.sqrt(I0) * np.exp(-(X ** 2 + Y ** 2) / w0 ** 2) * np.exp(0.7j)
    for p, q in [(1, 0), (1, 1), (2, 0), (2, 2), (3, 1), (1, 3)]:
        expect = I0 ** p * math.pi * math.factorial(q) * (w0 ** 2 / (2 * p)) ** (q + 1)
        assert abs(oracle.moment(U, L, p, q) / expect - 1) < 1e-12, (p, q)
    assert abs(oracle.moment(U, L, 1, 0) / oracle.power(U, L) - 1) < 1e-14
    # off-centre beam: the moment is taken about the window centre (parallel-axis rule)
    Us = np.sqrt(I0) * np.exp(-((X - 0.2) ** 2 + Y ** 2) / w0 ** 2)
    expect = I0 * math.pi * w0 ** 2 / 2 * (w0 ** 2 / 2 + 0.2 ** 2)
    assert abs(oracle.moment(Us, L, 1, 1) / expect - 1) < 1e-12


# ------------------------------------------- effective lens (Eqs. 4-6)

def test_lens_lowpass_gaussian_closed_form():
    """Eq. 4 on a well-resolved Gaussian: the low-pass exp(-l k^2) is the heat
    kernel, so exp(-r^2/s^2) becomes s^2/(s^2 + 4 l) exp(-r^2/(s^2 + 4 l))
    (continuous Fourier transform; aliasing below 1e-60 here).  l = 0 is the
    identity and a constant is kept."""
    n, L = 128, 1.28
    dx = L / n
    s = 8 * dx
    y, x = np.indices((n, n))
    r2 = ((x - 64) ** 2 + (y - 64) ** 2) * dx * dx
    w = np.exp(-r2 / s ** 2)
    for l in (1e-5, 4e-5, 1.5e-4):
        out = oracle.lens_lowpass(w, L, l)
        s2 = s * s + 4 * l
        assert np.max(np.abs(out - s * s / s2 * np.exp(-r2 / s2))) < 1e-12
    assert np.max(np.abs(oracle.lens_lowpass(w, L, 0.0) - w)) < 1e-14
    assert np.max(np.abs(oracle.lens_lowpass(np.full((n, n), 3.0), L, 1e-3) - 3.0)) < 1e-13
    # anisotropic input: the low-pass acts along both axes (a line along x keeps its x profile)
    line = np.zeros((n, n))
    line[64, :] = 1.0
    out = oracle.lens_lowpass(line, L, 1e-4)
    assert np.max(np.abs(out - out[:, :1])) < 1e-13
    assert out[64, 0] < 0.5


def test_lens_centres_hand_made():
    """Trimming at w_l leaves disconnected lenses; each centre is the lens's
    largest w_dif, the first in row-major order on a plateau."""
    w = np.zeros((8, 8))
    w[1, 1], w[1, 2], w[2, 1] = 5.0, 7.0, 6.0        # lens A, maximum at (1, 2)
    w[5, 5] = w[5, 6] = w[6, 5] = 4.0                # lens B, a plateau: first is (5, 5)
    w[3, 7] = 0.5                                    # below the level
    c = oracle.lens_centres(w, 1.0, 4)
    assert c.tolist() == [1 * 8 + 2, 5 * 8 + 5]
    w[3, 3] = w[4, 4] = 2.0                          # a diagonal chain to B: joined with 8 neighbours only
    assert oracle.lens_centres(w, 1.0, 4).tolist() == [1 * 8 + 2, 3 * 8 + 3, 4 * 8 + 4, 5 * 8 + 5]
    assert oracle.lens_centres(w, 1.0, 8).tolist() == [1 * 8 + 2, 5 * 8 + 5]
    assert oracle.lens_centres(np.zeros((8, 8)), 1.0, 4).size == 0


LENS1 = dict(l_dif=0.0, w_l=1.0, conn=4,
             re=[(0.02, 0.8, 60.0, 0.3), (0.05, -0.4, 25.0, 1.1)],
             im=[(0.03, 0.2, 40.0, -0.5)])


def test_lens_value_is_piecewise_eq6():
    """Eq. 6: segment j holds on r_{j-1} <= r < r_j (r_0 = 0); zero past the
    last joint; real and imaginary parts have their own joints."""
    for r, re, im in [(0.0, 0.8 * math.cos(0.3), 0.2 * math.cos(-0.5)),
                      (0.019, 0.8 * math.cos(60 * 0.019 + 0.3), 0.2 * math.cos(40 * 0.019 - 0.5)),
                      (0.02, -0.4 * math.cos(25 * 0.02 + 1.1), 0.2 * math.cos(40 * 0.02 - 0.5)),
                      (0.03, -0.4 * math.cos(25 * 0.03 + 1.1), 0.0),
                      (0.05, 0.0, 0.0), (1.0, 0.0, 0.0)]:
        got = oracle.lens_value(LENS1, r)
        assert abs(got[0] - re) < 1e-15 and abs(got[1] - im) < 1e-15, r


def test_lens_apply_closed_form_and_superposition():
    """Eqs. 2 and 5 for a plane field: one centre multiplies U by
    exp(i Re f(r)) exp(-Im f(r)) with r the distance across the window (a
    centre next to the edge does not wrap); two centres multiply the two
    single-centre screens (the sum over centres of Eq. 5)."""
    n, L = 64, 0.64
    dx = L / n
    U = np.full((n, n), 2.0 + 1.0j)
    y, x = np.indices((n, n))

    def single(c):
        r = dx * np.sqrt((x - c % n) ** 2.0 + (y - c // n) ** 2.0)
        re = np.where(r < 0.02, 0.8 * np.cos(60 * r + 0.3), np.where(r < 0.05, -0.4 * np.cos(25 * r + 1.1), 0.0))
        im = np.where(r < 0.03, 0.2 * np.cos(40 * r - 0.5), 0.0)
        return np.exp(1j * re - im)

    c1, c2 = 2 * n + 1, 40 * n + 30
    out = oracle.lens_apply(U, L, [c1], LENS1)
    assert np.max(np.abs(out - U * single(c1))) < 1e-13
    out = oracle.lens_apply(U, L, [c1, c2], LENS1)
    assert np.max(np.abs(out - U * single(c1) * single(c2))) < 1e-13


def test_effective_lens_finds_planted_spots():
    """The whole screen on a field with two hot spots on a weak background:
    after the low-pass the lenses are centred on the spots' peaks (symmetric
    spots keep their maxima), and the field changes only within the ansatz's
    reach of them."""
    cfg = configs.physics(128, 1.28, 1.0, configs.KERR)
    n, dx = 128, 0.01
    y, x = np.indices((n, n))
    spots = [(40, 30), (90, 100)]
    w = 1e11 * np.exp(-((x - 64.0) ** 2 + (y - 64.0) ** 2) * dx * dx / 0.3 ** 2)
    for (sy, sx) in spots:
        w = w + 5e12 * np.exp(-((x - sx) ** 2 + (y - sy) ** 2) * dx * dx / 0.02 ** 2)
    U = np.sqrt(w) * np.exp(0.3j)
    lens = dict(LENS1, l_dif=2e-5, w_l=1e12)
    out, cent = oracle.effective_lens(U, cfg, lens)
    assert cent.tolist() == sorted(sy * n + sx for sy, sx in spots)
    far = np.ones((n, n), bool)
    for (sy, sx) in spots:
        far &= (x - sx) ** 2 + (y - sy) ** 2 >= 25 ** 2
    assert np.array_equal(out[far], U[far])
    assert not np.allclose(out[~far], U[~far])


# ------------------------------------------------ planted mistakes (CPU)

MUTANTS = [
    # (name, original text, replacement, pin that must fail)
    ("propagator sign", "P[(size_t)r * n + c] = cexp(I * phase);",
     "P[(size_t)r * n + c] = cexp(-I * phase);", "gauss"),
    ("Nyquist / negative frequency index", "int mm = (m < n / 2) ? m : m - n;",
     "int mm = m;", "gauss"),
    ("Kerr factor 2 dropped", "c.eps_k = 2.0 * c.k0 * c.k0 * p->n2 / p->n0;",
     "c.eps_k = c.k0 * c.k0 * p->n2 / p->n0;", "kerr"),
    ("absorption exponent K instead of K-1",
     "bracket += c->cA * I * c->k0 * c->alpha_m * pow(In, (double)(p->K - 1));",
     "bracket += c->cA * I * c->k0 * c->alpha_m * pow(In, (double)(p->K));", "mpa"),
    ("transposed column pass", "for (int r = 0; r < n; ++r) col[r] = a[(size_t)r * n + c];",
     "for (int r = 0; r < n; ++r) col[r] = a[(size_t)c * n + r];", "fft"),
    ("adjoint screen conj dropped", "G[i] = conj(e) * gw + 2.0",
     "G[i] = e * gw + 2.0", "adjoint"),
    ("Strang half screen over the full step", "half.dz = 0.5 * p->dz;", "half.dz = p->dz;", "strang"),
    ("hot areas joined across the window edge", "if (rr < 0 || rr >= n || cc < 0 || cc >= n) continue;",
     "rr = (rr + n) % n; cc = (cc + n) % n;", "hot"),
    ("turbulent layer sign", "U[i] *= cexp(-I * c * eps[i]);", "U[i] *= cexp(I * c * eps[i]);", "turb_kerr"),
    ("turbulent layer without the 2 k0", "double c = thickness / (2.0 * wavenumber(p));",
     "double c = thickness / wavenumber(p);", "turb_kerr"),
    ("turbulent step read literally as theta(k - k_h)", "S[(size_t)q * n + c] = (m2 <= r2) ?",
     "S[(size_t)q * n + c] = (m2 > r2) ?", "turb_line"),
    ("turbulent screen without the n^2 of the unnormalised sum", "eps[i] = creal(S[i]) * (double)nn;",
     "eps[i] = creal(S[i]);", "turb_line"),
    ("exact substep amplitude without the square root", "amp = exp(-l / (2.0 * (K - 1)));",
     "amp = exp(-l / (double)(K - 1));", "exact"),
    ("exact substep Kerr integral with the wrong exponent", "double e = (double)(K - 2) / (double)(K - 1);",
     "double e = (double)(K - 1) / (double)(K - 2);", "exact"),
    ("moment about the window corner", "double xc = ((double)x - n / 2 + 0.5) * dx;",
     "double xc = ((double)x) * dx;", "moments"),
    ("moment radius exponent q instead of 2q", "pow(xc * xc + yc * yc, (double)q)",
     "pow(sqrt(xc * xc + yc * yc), (double)q)", "moments"),
    ("low-pass sign", "W[(size_t)r * n + c] *= exp(-l_dif * (kx * kx + ky * ky));",
     "W[(size_t)r * n + c] *= exp(l_dif * (kx * kx + ky * ky));", "lens_gauss"),
    ("low-pass along x only", "W[(size_t)r * n + c] *= exp(-l_dif * (kx * kx + ky * ky));",
     "W[(size_t)r * n + c] *= exp(-l_dif * (kx * kx));", "lens_gauss"),
    ("lens centre = last maximum on a plateau", "if (best[root] < 0 || wd[i] > wd[best[root]])",
     "if (best[root] < 0 || wd[i] >= wd[best[root]])", "lens_centres"),
    ("lens segment closed at its joint", "if (r < ls->r_re[j]) { *re", "if (r <= ls->r_re[j]) { *re", "lens_value"),
    ("lens screen sign", "U[(size_t)y * n + x] *= cexp(I * (dre + I * dim));",
     "U[(size_t)y * n + x] *= cexp(-I * (dre + I * dim));", "lens_apply"),
    ("lens distance wrapped across the window", "int xc = centres[c] % n, yc = centres[c] / n;",
     "int xc = centres[c] % n, yc = centres[c] / n; if (x - xc > n / 2) xc += n; if (xc - x > n / 2) xc -= n;",
     "lens_apply"),
    ("turbulent screen with x and y swapped", "S[(size_t)q * n + c] = (m2 <= r2) ? tau * xi[(size_t)q * n + c]",
     "S[(size_t)q * n + c] = (m2 <= r2) ? tau * xi[(size_t)c * n + q]", "turb_line"),
]


@pytest.mark.parametrize("name,orig,repl,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, orig, repl, pin, tmp_path, monkeypatch):
    src = oracle.source_text()
    assert orig in src, name
    lib = oracle.compile_variant(src.replace(orig, repl), str(tmp_path / "mutant.so"))
    monkeypatch.setattr(oracle, "_lib", lib)
    pins = {
        "gauss": test_linear_march_matches_closed_form_gaussian,
        "kerr": test_kerr_screen_exact_phase_identity,
        "mpa": test_mpa_screen_exact_attenuation,
        "fft": lambda: test_fft2_matches_brute_force_dft(8),
        "adjoint": test_adjoint_field_gradient_matches_directional_difference,
        "strang": test_strang_is_second_order_and_lie_first_order,
        "hot": test_hot_areas_hand_made_patterns,
        "turb_kerr": test_turbulent_layer_acts_like_the_kerr_term,
        "turb_line": test_turbulent_eps_single_spectral_line,
        "lens_gauss": test_lens_lowpass_gaussian_closed_form,
        "lens_centres": test_lens_centres_hand_made,
        "lens_value": test_lens_value_is_piecewise_eq6,
        "lens_apply": test_lens_apply_closed_form_and_superposition,
        "moments": test_moments_gaussian_closed_form,
        "exact": lambda: test_exact_substep_matches_rk4(8),
    }
    with pytest.raises(AssertionError):
        pins[pin]()
