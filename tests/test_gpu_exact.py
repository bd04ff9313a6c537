"""GPU exact pointwise substep (the nonlinear part of Eqs. 1-3 over a step in
closed form, NLSE_EXACT_SCREEN) against the oracle's march with the same
substep, through the C ABI: FP64 rel-L2 <= 1e-10; FP32 fluence rel-L2 <= 2e-4
up to the first collapse."""
import numpy as np
import pytest

import oracle
from paper_2306_15678_gb300 import beams, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


def clamping_cfg(scheme="lie", theta=(1.0, 0.0, 1.0, 0.0, 1.0, 0.0)):
    cfg = configs.physics(64, 1.6, 0.5, configs.ALL_TERMS, theta=theta)
    cfg["beam"] = dict(w0=0.12, P=300 * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=11,
                       phase=0.1, phase_seed=12)
    cfg["scheme"] = scheme
    cfg["screen"] = "exact"
    return cfg


@pytest.mark.parametrize("scheme", ["lie", "strang"])
def test_exact_fp64_clamping_regime(scheme):
    """Kerr, plasma and absorption into the intensity-clamping regime, where the
    absorption over a step is strong and the two screens differ."""
    cfg = clamping_cfg(scheme, theta=(0.9, 0.0, 1.1, 0.0, 1.3, 0.0))
    U0 = beams.make_field(cfg)
    ref, pw, pk = oracle.march(U0, cfg, 40)
    frozen, _, _ = oracle.march(U0, dict(cfg, screen="frozen"), 40)
    assert pk.max() > 3e13 and rel_l2(frozen, ref) > 1e-6
    with Grid(cfg, precision="fp64", diag_every=1) as g:
        U = g.load(U0).step(17).step(23).field()
        hpw, _ = g.history()
    assert rel_l2(U, ref) <= 1e-10
    assert np.max(np.abs(hpw / pw[1:] - 1)) < 1e-10


def test_exact_fp32_dense_physics_fluence():
    cfg = configs.physics(512, 2.0, 0.5, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=0.25, P=40 * configs.critical_power(), amp=0.1, ell_cells=4.0, seed=41,
                       phase=0.1, phase_seed=42)
    cfg["screen"] = "exact"
    U0 = beams.make_field(cfg)
    ref, _, pk = oracle.march(U0, cfg, 120)
    first = int(np.argmax(pk >= 2e12)) if np.any(pk >= 2e12) else len(pk) - 1
    assert first >= 10
    a, _, _ = oracle.march(U0, cfg, first)
    with Grid(cfg, precision="fp32") as g:
        F = g.load(U0.astype(np.complex64)).step(first).fluence()
    Fref = np.abs(a) ** 2
    assert np.linalg.norm(F - Fref) / np.linalg.norm(Fref) <= 2e-4


def test_exact_without_absorption_equals_frozen_on_gpu():
    """No absorption term: the exact substep is the frozen screen (FP64, up to
    the rounding of the different formulas)."""
    cfg = configs.physics(128, 1.0, 1.0, configs.KERR | configs.PLASMA | configs.DIFFRACTION)
    cfg["beam"] = dict(w0=0.1, P=20 * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=3,
                       phase=0.0, phase_seed=None)
    U0 = beams.make_field(cfg)
    with Grid(cfg, precision="fp64") as g:
        a = g.load(U0).step(20).field()
    with Grid(dict(cfg, screen="exact"), precision="fp64") as g:
        b = g.load(U0).step(20).field()
    assert rel_l2(b, a) <= 1e-12
