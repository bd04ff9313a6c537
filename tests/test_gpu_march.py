"""GPU parity of the split-step march (arXiv 2306.15678, Eq. 2 with Eqs. 1 and 3)
against the FP64 CPU oracle, through the C ABI.

Tolerances: FP64 path rel-L2 <= 1e-10; FP32 path fluence rel-L2 <= 2e-4 up to the
first step whose peak reaches w_pf = 2 TW/cm^2 (Sec. 2, before Eq. 4), and
Kerr-only power drift <= 1e-6.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2306_15678_gb300 import beams, capi, configs, tune
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


def beam_cfg(n, terms, dz, L=2.56, w0=0.2, pcr=10.0, amp=0.05, ell=3.0, seed=5, phase=0.0):
    cfg = configs.physics(n, L, dz, terms)
    cfg["beam"] = dict(w0=w0, P=pcr * configs.critical_power(), amp=amp, ell_cells=ell,
                       seed=seed if amp else None, phase=phase, phase_seed=seed + 1 if phase else None)
    return cfg


# ---------------------------------------------------------------- FFT sizes

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("n", [8, 16, 32, 64, 128, 256, 512, 1024, 2048])
def test_linear_march_every_size(n, prec, tol):
    """Diffraction only: exercises every transform length and the propagator."""
    cfg = beam_cfg(n, configs.DIFFRACTION, dz=40.0, L=0.02 * n, w0=0.002 * n, ell=2.0)
    U0 = beams.make_field(cfg)
    ref, _, _ = oracle.march(U0, cfg, 5)
    with Grid(cfg, precision=prec) as g:
        U = g.load(U0).step(5).field()
    assert rel_l2(U, ref) < tol


@pytest.mark.parametrize("prec,n", [("fp32", 256), ("fp32", 1024), ("fp64", 512)])
def test_every_column_tile_agrees(prec, n, monkeypatch):
    cfg = beam_cfg(n, configs.ALL_TERMS, dz=10.0, L=0.01 * n, w0=0.0015 * n, pcr=50.0)
    U0 = beams.make_field(cfg)
    ref, _, _ = oracle.march(U0, cfg, 3)
    outs = []
    for c in (1, 2, 4, 8, 16):
        monkeypatch.setenv("NLSE_COL_TILE", str(c))
        with Grid(cfg, precision=prec) as g:
            outs.append(g.load(U0).step(3).field())
    for U in outs:
        assert rel_l2(U, ref) < (1e-11 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec,n", [("fp32", 4096), ("fp32", 2048), ("fp32", 512), ("fp64", 1024)])
def test_column_tiles_bit_identical(prec, n):
    """The column tile (its width, and per-thread accesses or bulk tensor
    copies) changes which threads transform which column and how the tile
    reaches shared memory, not the arithmetic: for one transform radix every
    valid tile gives the same bits, and the staged variant exists at these
    sizes.  Each radix (FP32: 16 and 8) stays within 2e-5 of the oracle."""
    cfg = configs.scaled(configs.cfg_dense_fp32(), n, nsteps=2)
    U0 = beams.make_field(cfg)
    if prec == "fp32":
        U0 = U0.astype(np.complex64)
    ref_or, _, _ = oracle.march(U0.astype(np.complex128), cfg, 3)
    outs = {}
    with Grid(cfg, precision=prec) as g:
        for c in tune.TILE_CODES:
            try:
                capi.nlse_set_column_tile(g.h, c)
            except capi.NlseError as e:
                assert e.status == capi.NLSE_EUNSUPPORTED
                continue
            outs[c] = g.load(U0).step(3).field()
        assert g.device_status() == capi.NLSE_OK
    assert any(c & capi.NLSE_COL_TMA for c in outs)
    if prec == "fp32":
        assert any(c & capi.NLSE_COL_R8 for c in outs)
    for radix_bit in (0, capi.NLSE_COL_R8):
        group = {c: U for c, U in outs.items() if c & capi.NLSE_COL_R8 == radix_bit}
        if not group:
            continue
        ref = next(iter(group.values()))
        for c, U in group.items():
            assert np.array_equal(U, ref), hex(c)
        assert rel_l2(ref, ref_or) < (1e-11 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("n", [8, 64, 512, 4096])
def test_row_radix_choices_match_oracle(n):
    """Both FP32 row-pass radices (16 and 8 elements per thread) against the
    oracle; FP64 grids take radix 8 only."""
    if n >= 512:
        cfg = configs.scaled(configs.cfg_dense_fp32(), n, nsteps=2)
    else:
        cfg = beam_cfg(n, configs.ALL_TERMS, dz=2.0, L=0.05 * n, w0=0.0125 * n, pcr=30.0)
    U0 = beams.make_field(cfg).astype(np.complex64)
    ref, _, _ = oracle.march(U0.astype(np.complex128), cfg, 3)
    with Grid(cfg, precision="fp32") as g:
        for r in (16, 8) + ((capi.NLSE_ROW_STAGED | 16,) if n >= 2048 else ()):
            capi.nlse_set_row_radix(g.h, r)
            U = g.load(U0).step(3).field()
            assert rel_l2(U, ref) < 2e-5, (n, r)
        with pytest.raises(capi.NlseError) as ei:
            capi.nlse_set_row_radix(g.h, 4)
        assert ei.value.status == capi.NLSE_EUNSUPPORTED
        if n < 2048:  # the staged row pass needs one row pair of whole warps per block
            with pytest.raises(capi.NlseError) as ei:
                capi.nlse_set_row_radix(g.h, capi.NLSE_ROW_STAGED | 16)
            assert ei.value.status == capi.NLSE_EUNSUPPORTED
    with Grid(cfg, precision="fp64") as g:
        capi.nlse_set_row_radix(g.h, 8)
        with pytest.raises(capi.NlseError):
            capi.nlse_set_row_radix(g.h, 16)
        with pytest.raises(capi.NlseError):
            capi.nlse_set_row_radix(g.h, capi.NLSE_ROW_STAGED | 16)


@pytest.mark.parametrize("n", [2048, 4096, 8192])
@pytest.mark.parametrize("scheme", ["lie", "strang"])
def test_staged_row_pass_bit_identical_to_radix16(n, scheme):
    """The persistent row pass that stages each row pair by a bulk copy gives
    the bits of the radix-16 row pass: the field and the per-step power and
    peak history (one partial per row pair in both), Lie and Strang steps
    (whose opening half screen runs the row pass alone)."""
    cfg = configs.scaled(configs.cfg_dense_fp32(), n, nsteps=5)
    if scheme == "strang":
        cfg = dict(cfg, scheme="strang")
    U0 = beams.make_field(cfg).astype(np.complex64)
    out = {}
    for r in (16, capi.NLSE_ROW_STAGED | 16):
        with Grid(cfg, precision="fp32", diag_every=1) as g:
            capi.nlse_set_row_radix(g.h, r)
            g.load(U0).step(2).step(3)
            pw, pk = g.history()
            out[r] = (g.field(), pw, pk)
            assert g.device_status() == capi.NLSE_OK
    a, b = out[16], out[capi.NLSE_ROW_STAGED | 16]
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_staged_column_pass_wait_runs_out_cleanly(monkeypatch):
    """Block 0 of the staged column pass is made to expect 16 bytes that its
    copies never bring: its bounded wait runs out after 1 s, the grid reports
    NLSE_ETIMEOUT, and the context stays usable for the next grid."""
    cfg = beam_cfg(512, configs.ALL_TERMS, dz=2.0, L=0.64, w0=0.05)
    U0 = beams.make_field(cfg).astype(np.complex64)
    monkeypatch.setenv("NLSE_DEBUG_COL_EXTRA_TX", "16")
    with Grid(cfg, precision="fp32") as g:
        capi.nlse_set_column_tile(g.h, 4 | capi.NLSE_COL_TMA)
        g.load(U0).step(1)
        torch.cuda.synchronize()
        assert g.device_status() == capi.NLSE_ETIMEOUT
        assert g.device_status() == capi.NLSE_OK  # reading clears the word
    monkeypatch.delenv("NLSE_DEBUG_COL_EXTRA_TX")
    ref, _, _ = oracle.march(U0.astype(np.complex128), cfg, 3)
    with Grid(cfg, precision="fp32") as g:
        capi.nlse_set_column_tile(g.h, 4 | capi.NLSE_COL_TMA)
        U = g.load(U0).step(3).field()
        assert g.device_status() == capi.NLSE_OK
    assert rel_l2(U, ref) < 1e-5


def test_staged_row_pass_wait_runs_out_cleanly(monkeypatch):
    """Block 0 of the staged (persistent) row pass is made to expect 16 bytes
    more than its first bulk copy brings: its bounded waits run out (1 s
    each), the grid reports NLSE_ETIMEOUT, and the context stays usable: the
    next grid's staged row pass gives the bits of the radix-16 row pass."""
    cfg = configs.scaled(configs.cfg_dense_fp32(), 2048, nsteps=3)
    U0 = beams.make_field(cfg).astype(np.complex64)
    monkeypatch.setenv("NLSE_DEBUG_ROW_EXTRA_TX", "16")
    with Grid(cfg, precision="fp32") as g:
        capi.nlse_set_row_radix(g.h, capi.NLSE_ROW_STAGED | 16)
        g.load(U0).step(1)
        torch.cuda.synchronize()
        assert g.device_status() == capi.NLSE_ETIMEOUT
        assert g.device_status() == capi.NLSE_OK  # reading clears the word
    monkeypatch.delenv("NLSE_DEBUG_ROW_EXTRA_TX")
    out = []
    for r in (capi.NLSE_ROW_STAGED | 16, 16):
        with Grid(cfg, precision="fp32") as g:
            capi.nlse_set_row_radix(g.h, r)
            out.append(g.load(U0).step(3).field())
            assert g.device_status() == capi.NLSE_OK
    assert np.array_equal(out[0], out[1])


# ------------------------------------------------------------ plain FP64

def test_plain_fp64_256_matches_oracle():
    """256^2 FP64, Kerr + diffraction, 200 steps of 1 cm: rel-L2 <= 1e-10."""
    cfg = configs.cfg_plain_fp64()
    U0 = beams.make_field(cfg)
    ref, pw, pk = oracle.march(U0, cfg, 200)
    with Grid(cfg, precision="fp64", diag_every=1) as g:
        g.load(U0).step(200)
        U = g.field()
        hpw, hpk = g.history()
        assert rel_l2(U, ref) <= 1e-10
        assert np.max(np.abs(hpw / pw[1:] - 1)) < 1e-12
        assert np.max(np.abs(hpk / pk[1:] - 1)) < 1e-10
        assert g.steps_taken == 200


def test_full_screen_fp64_strong_nonlinearity():
    """Into the plasma-clamping regime (peak > 5e13 W/cm^2).  dz = 5 mm keeps the
    march well conditioned there: a 1e-15 input perturbation stays below 1e-11
    after 40 steps (at dz >= 1 cm it grows to O(1), on the oracle too)."""
    cfg = beam_cfg(128, configs.ALL_TERMS, dz=0.5, L=1.6, w0=0.12, pcr=300.0, phase=0.1)
    U0 = beams.make_field(cfg)
    U_ref = U0
    peak = 0.0
    with Grid(cfg, precision="fp64") as g:
        g.load(U0)
        for chunk in range(4):
            U_ref, _, pk = oracle.march(U_ref, cfg, 10)
            peak = max(peak, pk.max())
            U = g.step(10).field()
            assert rel_l2(U, U_ref) <= 1e-10, chunk
    assert peak > 5e13  # plasma and absorption active


# ------------------------------------------------------------- FP32 path

def test_fp32_dense_physics_until_first_collapse():
    """cfg-2 physics (full screen, 5 mm steps, 5 % amplitude + 0.1 rad phase
    noise) on a 512^2 window: fluence rel-L2 <= 2e-4 at every compared step up to
    the first step whose peak reaches 2 TW/cm^2."""
    cfg = configs.scaled(configs.cfg_dense_fp32(), 512)
    U0 = beams.make_field(cfg).astype(np.complex64)  # same input bytes on both sides
    U_ref = U0.astype(np.complex128)
    worst = 0.0
    with Grid(cfg, precision="fp32") as g:
        g.load(U0)
        for chunk in range(40):
            U_ref, _, pk = oracle.march(U_ref, cfg, 50)
            g.step(50)
            F = g.fluence().astype(np.float64)
            Fr = np.abs(U_ref) ** 2
            err = float(np.linalg.norm(F - Fr) / np.linalg.norm(Fr))
            worst = max(worst, err)
            assert err <= 2e-4, (chunk, err)
            if pk.max() >= configs.W_PF:
                break
    assert worst > 0


def test_fp32_full_size_dense_grid_two_steps():
    """4096^2, the launch configuration of the benchmark, against the oracle."""
    cfg = configs.cfg_dense_fp32()
    U0 = beams.make_field(cfg).astype(np.complex64)
    ref, pw, pk = oracle.march(U0.astype(np.complex128), cfg, 2)
    with Grid(cfg, precision="fp32", diag_every=1) as g:
        g.load(U0.astype(np.complex64)).step(2)
        U = g.field()
        assert rel_l2(U, ref) < 2e-5
        hpw, hpk = g.history()
        assert np.max(np.abs(hpw / pw[1:] - 1)) < 1e-6
        assert np.max(np.abs(hpk / pk[1:] - 1)) < 1e-5


def test_fp32_kerr_only_power_drift_full_size():
    """Kerr + diffraction (lossless) at 4096^2: |P/P0 - 1| <= 1e-6 up to the first
    collapse (peak >= 2 TW/cm^2) or 2000 steps."""
    cfg = dict(configs.cfg_dense_fp32(), terms=configs.KERR | configs.DIFFRACTION)
    U0 = beams.make_field(cfg)
    P0 = oracle.power(U0.astype(np.complex64), cfg["L"])
    with Grid(cfg, precision="fp32", diag_every=10) as g:
        g.load(U0.astype(np.complex64)).step(2000)
        pw, pk = g.history()
    stop = int(np.argmax(pk >= configs.W_PF)) if np.any(pk >= configs.W_PF) else len(pk)
    assert stop > 5
    drift = np.max(np.abs(pw[:stop] / P0 - 1))
    assert drift <= 1e-6, drift


@pytest.mark.parametrize("terms", [configs.KERR, configs.KERR | configs.PLASMA | configs.MPA])
def test_fp32_screen_against_exact_phase_up_to_large_phases(terms):
    """Screen only (no diffraction), 20 cm step: the FP32 phase factor against the
    oracle for per-step phases from ~0 to over 100 rad; the error allowed grows
    with the phase as the FP32 rounding of the phase itself (eps * phase)."""
    n = 256
    cfg = configs.physics(n, 1.0, 70.0 if terms == configs.KERR else 20.0, terms)
    rng = np.random.default_rng(9)
    I = np.geomspace(1e9, 6e13, n * n)
    rng.shuffle(I)
    I = I.reshape(n, n)
    v = np.sqrt(I) * np.exp(1j * rng.uniform(-np.pi, np.pi, (n, n)))
    v = v.astype(np.complex64).astype(np.complex128)
    Iv = np.abs(v) ** 2
    ref = oracle.screen(v, cfg)
    k0 = 2 * math.pi / cfg["lambda0"]
    phi_k = k0 * cfg["n2"] * Iv * cfg["dz"]
    phi_p = np.zeros_like(Iv)
    mpa = np.zeros_like(Iv)
    if terms & configs.PLASMA:
        phi_p = (k0 * cfg["sigmaK"] * cfg["rho_nt"] * cfg["tau_pl"] / (2 * cfg["rho_c"])
                 * Iv ** 8 * cfg["dz"])
        mpa = cfg["betaK"] / 2 * Iv ** 7 * cfg["dz"]
    assert (phi_k + phi_p).max() > 100
    with Grid(cfg, precision="fp32") as g:
        U = g.load(v).step(1).field().astype(np.complex128)
    # FP32 error budget: |v|^2 carries ~3 roundings, so the Kerr phase has a
    # relative error of a few eps; I^8 multiplies it by 8 for the plasma phase and
    # I^7 by 7 for the absorption exponent.  The (idle) column pass also
    # round-trips the field through FP32 FFTs, with an error relative to the
    # field's rms rather than to each of its 250x-spread values (the field goes
    # through four transforms in the two passes and one more in the readout).
    eps = 2.0 ** -24
    rms = float(np.sqrt(np.mean(Iv)))
    err = np.abs(U - ref)
    allowed = (1e-6 + 24 * eps * phi_k + 48 * eps * phi_p + 32 * eps * mpa) * np.abs(v) + 32 * eps * rms
    assert np.all(err <= allowed), float(np.max(err / allowed))


# -------------------------------------------------------------- readouts

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_readouts_match_oracle(prec):
    cfg = beam_cfg(256, configs.ALL_TERMS, dz=1.0, L=2.56, w0=0.2, pcr=100.0, phase=0.1)
    U0 = beams.make_field(cfg)
    if prec == "fp32":
        U0 = U0.astype(np.complex64).astype(np.complex128)
    ref, pw, pk = oracle.march(U0, cfg, 7)
    tol = 1e-12 if prec == "fp64" else 2e-5
    with Grid(cfg, precision=prec) as g:
        g.load(U0).step(7)
        assert abs(g.power() / oracle.power(ref, cfg["L"]) - 1) < tol
        assert abs(g.peak() / oracle.peak(ref) - 1) < 10 * tol
        for ds in (1, 2, 8):
            F = g.fluence(ds).astype(np.float64)
            Fr = oracle.fluence(ref, ds)
            assert np.linalg.norm(F - Fr) / np.linalg.norm(Fr) < 10 * tol
        Fd = g.fluence(8, device=True).cpu().numpy()
        assert np.array_equal(Fd, g.fluence(8))
        Ud = g.field(device=True).cpu().numpy()
        assert np.array_equal(Ud, g.field())


def test_fp32_power_reductions_against_an_fp64_sum_of_the_same_values():
    """The FP32 stage of the power reductions (per-thread sums and the block
    tree; the sum across blocks is FP64) against an FP64 sum of the very
    |U|^2 values the readout produces, on the 4096^2 dense grid after 50 full
    steps: the readout's power and the march's recorded power (its own
    partials of the screened field) both within 2e-7 of the FP64 sum."""
    cfg = configs.cfg_dense_fp32()
    U0 = beams.make_field(cfg).astype(np.complex64)
    dx2 = (cfg["L"] / cfg["n"]) ** 2
    with Grid(cfg, precision="fp32", diag_every=1) as g:
        g.load(U0).step(50)
        F = g.fluence().astype(np.float64)
        exact = math.fsum(F.ravel()) * dx2
        p_readout = g.power()
        pw, _ = g.history()
    err_readout = abs(p_readout / exact - 1)
    err_march = abs(pw[-1] / exact - 1)  # its values come before the readout's round trip
    print(f"FP32 reduction stage: readout {err_readout:.2e}, march {err_march:.2e}")
    assert err_readout <= 2e-7, err_readout
    assert err_march <= 2e-7, err_march


def test_load_from_device_equals_load_from_host():
    cfg = beam_cfg(128, configs.ALL_TERMS, dz=5.0, L=1.28, w0=0.1, pcr=60.0)
    U0 = beams.make_field(cfg)
    with Grid(cfg, precision="fp32") as a, Grid(cfg, precision="fp32") as b:
        a.load(U0).step(4)
        b.load(torch.from_numpy(U0.astype(np.complex64)).cuda()).step(4)
        assert np.array_equal(a.field(), b.field())


def test_runs_are_bit_reproducible():
    cfg = configs.scaled(configs.cfg_dense_fp32(), 1024)
    U0 = beams.make_field(cfg)
    res = []
    for _ in range(2):
        with Grid(cfg, precision="fp32", diag_every=3) as g:
            g.load(U0).step(12)
            res.append((g.field(), g.history()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1][0], res[1][1][0])


def test_radial_input_keeps_symmetry_on_gpu():
    cfg = beam_cfg(256, configs.ALL_TERMS, dz=20.0, L=2.56, w0=0.25, pcr=200.0, amp=0.0)
    U0 = beams.make_field(cfg)
    with Grid(cfg, precision="fp64") as g:
        U = g.load(U0).step(4).field()
    s = np.max(np.abs(U))
    assert np.max(np.abs(U - U.T)) / s < 1e-12
    assert np.max(np.abs(U - U[::-1, ::-1])) / s < 1e-12


# ----------------------------------------------------------- edge cases

def test_max_size_8192_against_closed_form_gaussian():
    """n = 8192 (largest supported), diffraction only: compare sampled points
    with the closed-form Gaussian beam of the paper's sign convention.  The beam
    (w0 = 5 mm in the 16 cm window) is negligible at the periodic boundary."""
    n, L, w0, dz, steps = 8192, 16.0, 0.5, 500.0, 4
    cfg = configs.physics(n, L, dz, configs.DIFFRACTION)
    P = 500 * configs.critical_power()
    U0 = beams.gaussian_beam(n, L, w0, P)
    with Grid(cfg, precision="fp32") as g:
        U = g.load(U0.astype(np.complex64)).step(steps).field()
    k0 = 2 * math.pi / cfg["lambda0"]
    zR = k0 * w0 * w0 / 2
    q = 1 - 1j * steps * dz / zR
    A = math.sqrt(2 * P / (math.pi * w0 * w0))
    x = beams.cell_centres(n, L)
    rng = np.random.default_rng(0)
    rows = rng.integers(0, n, 64)
    cols = rng.integers(n // 4, 3 * n // 4, 64)
    exact = A / q * np.exp(-(x[rows] ** 2 + x[cols] ** 2) / (w0 * w0 * q))
    got = U[rows, cols]
    assert abs(1 - 1 / abs(q)) > 0.01  # diffraction is visible
    assert np.max(np.abs(got - exact)) / A < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smallest_size_8_full_screen(prec):
    cfg = beam_cfg(8, configs.ALL_TERMS, dz=2.0, L=0.4, w0=0.1, pcr=30.0, amp=0.1, ell=1.0)
    U0 = beams.make_field(cfg)
    ref, _, _ = oracle.march(U0, cfg, 6)
    with Grid(cfg, precision=prec) as g:
        U = g.load(U0).step(6).field()
    assert rel_l2(U, ref) < (1e-12 if prec == "fp64" else 1e-5)


def test_zero_steps_and_roundtrip():
    cfg = beam_cfg(64, configs.ALL_TERMS, dz=2.0, L=0.64, w0=0.05)
    U0 = beams.make_field(cfg)
    with Grid(cfg, precision="fp64") as g:
        U = g.load(U0).step(0).field()
    assert rel_l2(U, U0) < 1e-15


def test_error_paths():
    cfg = beam_cfg(64, configs.ALL_TERMS, dz=2.0, L=0.64, w0=0.05)
    with Grid(cfg, precision="fp32") as g:
        with pytest.raises(capi.NlseError) as ei:
            g.step(1)  # before load
        assert ei.value.status == capi.NLSE_ESTATE
        with pytest.raises(capi.NlseError) as ei:
            g.step(-1)
        assert ei.value.status == capi.NLSE_EINVAL
        bad = beams.make_field(cfg).astype(np.complex64)
        bad[3, 5] = np.nan
        g.load(bad)
        with pytest.raises(capi.NlseError) as ei:
            g.power()
        assert ei.value.status == capi.NLSE_ENONFINITE
        assert g.device_status() == capi.NLSE_ENONFINITE
        assert g.device_status() == capi.NLSE_OK  # cleared
        with pytest.raises(capi.NlseError) as ei:
            g.fluence(3)
        assert ei.value.status == capi.NLSE_EINVAL
