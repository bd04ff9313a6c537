"""GPU effective-lens screen (Sec. 2, Eqs. 4-6: low-pass of the fluence,
trimming into lenses, lens centres, radial ansatz summed over the centres,
applied as exp(+i D_f)) against the oracle, through the C ABI.

Each step is checked on its own: the low-pass against the oracle's on the
same field (FP64 1e-12, FP32 1e-5 of the maximum); the lens centres, integer
decisions, bit for bit against the oracle's on the GPU's own w_dif (both
decide in the grid precision); the screen against the oracle's on the same
centres (FP64 1e-12, FP32 2e-6 rel-L2).  Then the whole screen in FP64 against
the oracle end to end (1e-10), and inside a march.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2306_15678_gb300 import beams, capi, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu

LENS = dict(l_dif=4e-4, w_l=1.0e11, conn=4,
            re=[(0.03, 0.9, 40.0, 0.2), (0.06, -0.5, 30.0, 1.0), (0.1, 0.2, 20.0, -0.4)],
            im=[(0.04, 0.3, 35.0, 0.1), (0.08, 0.1, 15.0, 0.5)])


def spotted_field(n, L, nspots, seed):
    """A weak Gaussian beam carrying hot spots of 2-8 TW/cm^2 (the
    pre-filamentation range) with radii 80-200 um at seeded positions, and a
    seeded smooth phase."""
    rng = np.random.default_rng(seed)
    dx = L / n
    c = (np.arange(n) - n / 2 + 0.5) * dx
    X, Y = np.meshgrid(c, c)
    w = 5e10 * np.exp(-(X ** 2 + Y ** 2) / (0.3 * L) ** 2)
    for _ in range(nspots):
        x0, y0 = rng.uniform(-0.35 * L, 0.35 * L, 2)
        r0 = rng.uniform(0.008, 0.02)
        w = w + rng.uniform(2e12, 8e12) * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / r0 ** 2)
    phase = 0.3 * np.sin(2 * math.pi * X / L + rng.uniform(0, 6)) * np.cos(2 * math.pi * Y / L)
    return np.sqrt(w) * np.exp(1j * phase)


def cfg_for(n, L=2.56):
    return configs.physics(n, L, 0.5, configs.KERR | configs.DIFFRACTION)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,conn", [(256, 4), (512, 8)])
def test_lens_steps_fp64(n, conn):
    cfg = cfg_for(n)
    lens = dict(LENS, conn=conn)
    U0 = spotted_field(n, cfg["L"], 12, 3 + n)
    with Grid(cfg, precision="fp64") as g:
        g.load(U0)
        before = g.field()
        k, cent, wd = g.effective_lens(lens, w_dif=True)
        after = g.field()
    wd = wd.cpu().numpy()
    wref = oracle.lens_lowpass(np.abs(before) ** 2, cfg["L"], lens["l_dif"])
    assert np.max(np.abs(wd - wref)) <= 1e-12 * np.max(wref)
    cref = oracle.lens_centres(wd, lens["w_l"], conn)
    assert k == len(cref) and np.array_equal(cent, cref)
    assert k >= 4
    assert rel_l2(after, oracle.lens_apply(before, cfg["L"], cent, lens)) <= 1e-12
    # end to end: the oracle's own low-pass makes the same decisions here
    Uref, cfull = oracle.effective_lens(before, cfg, lens)
    assert np.array_equal(cfull, cent)
    assert rel_l2(after, Uref) <= 1e-10


def test_lens_steps_fp32_and_device_outputs():
    n = 1024
    cfg = cfg_for(n, 5.12)
    U0 = spotted_field(n, cfg["L"], 30, 17).astype(np.complex64)
    with Grid(cfg, precision="fp32") as g:
        g.load(U0)
        before = g.field()
        k, cent, wd = g.effective_lens(LENS, w_dif=True)
        after = g.field()
        # same call again from the same field: bit-identical (fixed summation order)
        g.load(U0)
        k2, cent2, _ = g.effective_lens(LENS)
        after2 = g.field()
    wd = wd.cpu().numpy()
    wref = oracle.lens_lowpass(np.abs(before.astype(np.complex128)) ** 2, cfg["L"], LENS["l_dif"])
    assert np.max(np.abs(wd - wref)) <= 1e-5 * np.max(wref)
    cref = oracle.lens_centres(wd, float(np.float32(LENS["w_l"])), 4)
    assert k == len(cref) and np.array_equal(cent, cref) and k >= 10
    assert rel_l2(after, oracle.lens_apply(before, cfg["L"], cent, LENS)) <= 2e-6
    assert k2 == k and np.array_equal(cent2, cent) and np.array_equal(after2, after)


def test_degenerate_lenses():
    """A level above every value: no lens, field unchanged.  No ansatz
    segments: the lenses are found but the field is unchanged.  A lens touching
    the window edge: its screen is cut at the edge, not wrapped."""
    n = 128
    cfg = cfg_for(n, 1.28)
    U0 = spotted_field(n, cfg["L"], 4, 5)
    with Grid(cfg, precision="fp64") as g:
        k, cent, _ = g.load(U0).effective_lens(dict(LENS, w_l=1e16))
        assert k == 0 and cent.size == 0
        assert rel_l2(g.field(), U0) <= 1e-14
        k, cent, _ = g.load(U0).effective_lens(dict(LENS, re=[], im=[]))
        assert k >= 1 and rel_l2(g.field(), U0) <= 1e-14
        edge = np.full((n, n), 1e5 + 0j)
        edge[0, 3] = 3e6 + 0j  # one hot pixel on the first row
        k, cent, _ = g.load(edge).effective_lens(dict(LENS, l_dif=0.0, w_l=1e12))
        after = g.field()
    assert k == 1 and cent.tolist() == [3]
    assert rel_l2(after, oracle.lens_apply(edge, cfg["L"], cent, LENS)) <= 1e-12
    assert np.max(np.abs(after[n // 2:] - edge[n // 2:])) <= 1e-6  # rows beyond the reach: only the round trip


@pytest.mark.parametrize("scheme", ["lie", "strang"])
def test_march_lens_march_fp64(scheme):
    """The method's use: march to the pre-filamentation level, replace the
    filament region by the lens screen, march on; step count and history
    continue across the screen (Lie or symmetric steps around it)."""
    n = 256
    cfg = configs.physics(n, 1.28, 0.5, configs.ALL_TERMS)
    cfg["scheme"] = scheme
    U0 = spotted_field(n, cfg["L"], 6, 9)
    lens = dict(LENS, w_l=5e11)
    a, _, _ = oracle.march(U0, cfg, 10, record=False)
    b, cref = oracle.effective_lens(a, cfg, lens)
    ref, _, pk = oracle.march(b, cfg, 10)
    with Grid(cfg, precision="fp64", diag_every=1) as g:
        k, cent, _ = g.load(U0).step(10).effective_lens(lens)
        U = g.step(10).field()
        hpw, hpk = g.history()
        assert g.steps_taken == 20 and len(hpk) == 20
    assert np.array_equal(cent, cref) and k >= 1
    assert rel_l2(U, ref) <= 1e-10
    assert np.max(np.abs(hpk[10:] / pk[1:] - 1)) < 1e-10


def test_lens_argument_errors():
    n = 64
    cfg = cfg_for(n, 0.64)
    with Grid(cfg, precision="fp32") as g:
        g.load(spotted_field(n, cfg["L"], 2, 1).astype(np.complex64))
        bad = [dict(LENS, w_l=0.0), dict(LENS, l_dif=-1.0), dict(LENS, conn=6),
               dict(LENS, re=[(0.05, 1, 1, 0), (0.04, 1, 1, 0)]), dict(LENS, im=[(0.0, 1, 1, 0)]),
               dict(LENS, re=[(0.05, float("nan"), 1, 0)])]
        for lens in bad:
            with pytest.raises(capi.NlseError) as ei:
                g.effective_lens(lens)
            assert ei.value.status == capi.NLSE_EINVAL, lens
        need = capi.nlse_lens_scratch_size(g.params)
        small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
        with pytest.raises(capi.NlseError) as ei:
            capi.nlse_effective_lens(g.h, capi.make_lens(LENS), small.data_ptr(), need // 2, 0, 0, 0)
        assert ei.value.status == capi.NLSE_ENOMEM


def test_lens_fp32_full_size_4096():
    """The dense-grid size (4096^2 FP32, 8 cm window): low-pass, centres (bit
    for bit on the GPU's w_dif) and screen against the oracle."""
    cfg = configs.cfg_dense_fp32()
    n = cfg["n"]
    U0 = spotted_field(n, cfg["L"], 40, 99).astype(np.complex64)
    with Grid(cfg, precision="fp32") as g:
        g.load(U0)
        before = g.field()
        k, cent, wd = g.effective_lens(LENS, w_dif=True)
        after = g.field()
    wd = wd.cpu().numpy()
    wref = oracle.lens_lowpass(np.abs(before.astype(np.complex128)) ** 2, cfg["L"], LENS["l_dif"])
    assert np.max(np.abs(wd - wref)) <= 1e-5 * np.max(wref)
    cref = oracle.lens_centres(wd, float(np.float32(LENS["w_l"])), 4)
    assert k == len(cref) and np.array_equal(cent, cref) and k >= 20
    assert rel_l2(after, oracle.lens_apply(before, cfg["L"], cent, LENS)) <= 2e-6
