"""GPU parity of the symmetric (Strang) split step -- half screen over dz/2,
diffraction over dz, half screen over dz/2 (Eq. 2 split symmetrically) --
against the FP64 oracle's symmetric march, through the C ABI.

Tolerances as for the Lie march: FP64 rel-L2 <= 1e-10; FP32 fluence rel-L2
<= 2e-4 up to the first step whose peak reaches 2 TW/cm^2.
"""
import numpy as np
import pytest

import oracle
from paper_2306_15678_gb300 import beams, capi, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


def test_strang_fp64_256_matches_oracle():
    """256^2 FP64, Kerr + diffraction, 200 symmetric steps of 1 cm, in calls of
    uneven length (a call opens and closes its own half screens)."""
    cfg = dict(configs.cfg_plain_fp64(), scheme="strang")
    U0 = beams.make_field(cfg)
    ref, pw, pk = oracle.march(U0, cfg, 200)
    with Grid(cfg, precision="fp64", diag_every=1) as g:
        g.load(U0)
        for m in (1, 37, 62, 100):
            g.step(m)
        U = g.field()
        hpw, hpk = g.history()
        assert rel_l2(U, ref) <= 1e-10
        assert np.max(np.abs(hpw / pw[1:] - 1)) < 1e-12
        assert np.max(np.abs(hpk / pk[1:] - 1)) < 1e-10
        assert g.steps_taken == 200


def test_strang_fp64_full_screen_clamping_regime():
    """Kerr, plasma and absorption into the clamping regime (5 mm steps)."""
    cfg = configs.physics(64, 1.6, 0.5, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=0.12, P=300 * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=11,
                       phase=0.1, phase_seed=12)
    cfg["scheme"] = "strang"
    U0 = beams.make_field(cfg)
    ref, _, pk = oracle.march(U0, cfg, 40)
    assert pk.max() > 3e13
    with Grid(cfg, precision="fp64") as g:
        U = g.load(U0).step(40).field()
    assert rel_l2(U, ref) <= 1e-10


def test_strang_gpu_is_second_order():
    """On the GPU too: halving dz over 10 cm divides the error by ~4."""
    def cfg_m(M):
        c = configs.physics(64, 0.64, 10.0 / M, configs.KERR | configs.DIFFRACTION)
        c["beam"] = dict(w0=0.05, P=10.0 * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=3,
                         phase=0.0, phase_seed=None)
        c["scheme"] = "strang"
        return c
    U0 = beams.make_field(cfg_m(1))
    ref, _, _ = oracle.march(U0, cfg_m(640), 640)
    err = []
    for M in (10, 20, 40):
        with Grid(cfg_m(M), precision="fp64") as g:
            err.append(rel_l2(g.load(U0).step(M).field(), ref))
    for a, b in zip(err, err[1:]):
        assert abs(a / b / 4.0 - 1) < 0.1, err


def test_strang_fp32_dense_physics_until_first_collapse():
    """cfg-2 physics on a 512^2 window with symmetric steps, FP32: fluence rel-L2
    <= 2e-4 at every compared step up to the first collapse."""
    cfg = dict(configs.scaled(configs.cfg_dense_fp32(), 512), scheme="strang")
    U0 = beams.make_field(cfg).astype(np.complex64)
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


def test_strang_full_size_two_steps():
    """4096^2 FP32, the benchmark's grid, two symmetric steps against the oracle."""
    cfg = dict(configs.cfg_dense_fp32(), scheme="strang")
    U0 = beams.make_field(cfg).astype(np.complex64)
    ref, _, _ = oracle.march(U0.astype(np.complex128), cfg, 2)
    with Grid(cfg, precision="fp32") as g:
        U = g.load(U0).step(2).field()
    assert rel_l2(U, ref) < 2e-5
