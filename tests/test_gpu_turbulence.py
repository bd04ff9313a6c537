"""GPU turbulent layer (Sec. 3.3, Eqs. 9-10: spectral phase screen with a step
spectrum up to the cut-off k_h, applied as exp(-i thickness eps_t / (2 k0)))
against the oracle, through the C ABI.

Tolerances: FP64 rel-L2 <= 1e-10 (as for the march).  FP32: the layer itself
is a readout, two FP32 inverse transforms of the draws and a reload; its
phase error is ~1e-7 of the screen's amplitude, so the single layer is held to
rel-L2 <= 2e-6; after marching on, the march's FP32 bar (fluence rel-L2 <=
2e-4 before the first collapse) applies.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2306_15678_gb300 import beams, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


def layer_case(n, terms=configs.KERR | configs.DIFFRACTION):
    cfg = configs.physics(n, 1.6, 0.5, terms)
    cfg["beam"] = dict(w0=0.3, P=5 * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=21,
                       phase=0.05, phase_seed=22)
    kunit = 2 * math.pi / cfg["L"]
    # cut-off at 17.3 bins (no bin on the circle); tau such that the layer's
    # phase has an rms of ~1 rad over a 50 cm layer
    kh = 17.3 * kunit
    k0 = 2 * math.pi * cfg["n0"] / cfg["lambda0"]
    nbins = math.pi * 17.3 ** 2
    tau = 2 * k0 / 50.0 / math.sqrt(nbins)
    return cfg, tau, kh, 50.0


@pytest.mark.parametrize("n", [64, 512])
def test_layer_fp64_matches_oracle(n):
    cfg, tau, kh, thick = layer_case(n)
    U0 = beams.make_field(cfg)
    xi = beams.turbulence_draws(n, 5)
    ref = oracle.turbulent_screen(U0, xi, cfg, tau, kh, thick)
    assert np.std(np.angle(ref / U0)) > 0.3  # the layer does something
    with Grid(cfg, precision="fp64") as g:
        U = g.load(U0).turbulent_screen(xi, tau, kh, thick).field()
    assert rel_l2(U, ref) <= 1e-10


def test_layer_fp32_host_and_device_draws():
    n = 1024
    cfg, tau, kh, thick = layer_case(n)
    U0 = beams.make_field(cfg).astype(np.complex64)
    xi = beams.turbulence_draws(n, 6).astype(np.complex64)
    ref = oracle.turbulent_screen(U0, xi, cfg, tau, kh, thick)
    with Grid(cfg, precision="fp32") as g:
        U = g.load(U0).turbulent_screen(xi, tau, kh, thick).field()
        assert rel_l2(U, ref) <= 2e-6
        Ud = g.load(U0).turbulent_screen(torch.from_numpy(xi).cuda(), tau, kh, thick).field()
        assert np.array_equal(U, Ud)


def test_layer_then_march_fp64():
    """The paper's use: march, pass a turbulent layer, march on; the step count
    and the recorded history continue across the layer."""
    n = 256
    cfg, tau, kh, thick = layer_case(n, configs.ALL_TERMS)
    cfg["dz"] = 0.5
    U0 = beams.make_field(cfg)
    xi = beams.turbulence_draws(n, 7)
    a, _, pk1 = oracle.march(U0, cfg, 30)
    b = oracle.turbulent_screen(a, xi, cfg, tau, kh, thick)
    ref, pw2, pk2 = oracle.march(b, cfg, 30)
    with Grid(cfg, precision="fp64", diag_every=1) as g:
        g.load(U0).step(30).turbulent_screen(xi, tau, kh, thick).step(30)
        U = g.field()
        hpw, hpk = g.history()
        assert g.steps_taken == 60
    assert rel_l2(U, ref) <= 1e-10
    assert len(hpw) == 60
    assert np.max(np.abs(hpk[:30] / pk1[1:] - 1)) < 1e-10
    assert np.max(np.abs(hpk[30:] / pk2[1:] - 1)) < 1e-10


def test_layer_then_march_fp32_fluence():
    n = 1024
    cfg, tau, kh, thick = layer_case(n)
    cfg["dz"] = 1.0
    U0 = beams.make_field(cfg).astype(np.complex64)
    xi = beams.turbulence_draws(n, 8).astype(np.complex64)
    a, _, _ = oracle.march(U0, cfg, 20, record=False)
    b = oracle.turbulent_screen(a, xi, cfg, tau, kh, thick)
    ref, _, pk = oracle.march(b, cfg, 40)
    assert pk.max() < 2e12  # before the first collapse
    with Grid(cfg, precision="fp32") as g:
        F = g.load(U0).step(20).turbulent_screen(xi, tau, kh, thick).step(40).fluence()
    Fref = np.abs(ref) ** 2
    assert np.linalg.norm(F - Fref) / np.linalg.norm(Fref) <= 2e-4


def test_degenerate_layers_leave_the_field():
    """A zero thickness, a zero amplitude, or a cut-off below the first
    non-zero bin with draws only there: the field comes back unchanged up to
    the readout/reload round trip."""
    n = 128
    cfg, tau, kh, thick = layer_case(n)
    U0 = beams.make_field(cfg)
    xi = beams.turbulence_draws(n, 9)
    xi[0, 0] = 0.0
    with Grid(cfg, precision="fp64") as g:
        for args in ((tau, kh, 0.0), (0.0, kh, thick), (tau, 0.5 * 2 * math.pi / cfg["L"], thick)):
            U = g.load(U0).turbulent_screen(xi, *args).field()
            assert rel_l2(U, U0) <= 1e-13


def test_layer_fp32_full_size_4096():
    """The dense-grid size (4096^2 FP32, 8 cm window, as the benchmark runs it):
    the layer against the oracle on the whole field."""
    cfg = configs.cfg_dense_fp32()
    n = cfg["n"]
    kunit = 2 * math.pi / cfg["L"]
    k0 = 2 * math.pi * cfg["n0"] / cfg["lambda0"]
    kh = 40.3 * kunit
    tau = 2 * k0 / 50.0 / math.sqrt(math.pi * 40.3 ** 2)
    U0 = beams.make_field(cfg).astype(np.complex64)
    xi = beams.turbulence_draws(n, 77).astype(np.complex64)
    ref = oracle.turbulent_screen(U0, xi, cfg, tau, kh, 50.0)
    with Grid(cfg, precision="fp32") as g:
        U = g.load(U0).turbulent_screen(xi, tau, kh, 50.0).field()
    assert rel_l2(U, ref) <= 2e-6
