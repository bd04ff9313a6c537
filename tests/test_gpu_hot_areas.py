"""GPU hot-area count (Sec. 3.3: connected regions where the fluence reaches the
cut-off w_p) against the oracle's flood fill, through the C ABI.

The device thresholds the fluence it reads out itself; the oracle labels the
same fluence (read back with nlse_fluence, which runs the same readout) at the
same cut-off in the grid precision, so the two label arrays must be identical:
labels are integer work, compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2306_15678_gb300 import beams, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def noise_field(n, seed, corr=0):
    """Field whose fluence is uniform noise (optionally box-smoothed over corr
    cells, so that regions have extent), amplitude ~ 1e6 (W/cm^2)^(1/2)."""
    rng = np.random.default_rng(seed)
    w = rng.random((n, n))
    if corr:
        k = np.ones(corr) / corr
        w = np.apply_along_axis(lambda r: np.convolve(np.concatenate([r, r[:corr - 1]]), k, "valid"), 1, w)
        w = np.apply_along_axis(lambda c: np.convolve(np.concatenate([c, c[:corr - 1]]), k, "valid"), 0, w)
    return (1e6 * np.sqrt(w)).astype(np.complex128)


def grid_cfg(n):
    return configs.physics(n, 0.64, 1e-3, configs.KERR | configs.DIFFRACTION)


def check_against_oracle(g, wp, conn, precision):
    F = g.fluence()
    wp_g = float(np.float32(wp)) if precision == "fp32" else float(wp)
    count, labels = g.hot_areas(wp, conn, labels=True)
    ref_count, ref_labels = oracle.hot_areas(F, wp_g, conn)
    assert count == ref_count
    assert np.array_equal(labels, ref_labels)
    return count, labels


@pytest.mark.parametrize("n", [8, 16, 64, 256, 1024])
@pytest.mark.parametrize("conn", [4, 8])
def test_random_masks_near_percolation(n, conn):
    """Uncorrelated pixels with the fill fraction at the site-percolation
    threshold of the lattice (0.593 with 4 neighbours, 0.407 with 8): the
    hardest masks for union-find, with regions of every size."""
    fill = 0.593 if conn == 4 else 0.407
    U0 = noise_field(n, 100 + n + conn)
    with Grid(grid_cfg(n), precision="fp32") as g:
        g.load(U0.astype(np.complex64))
        F = g.fluence()
        wp = float(np.quantile(F.astype(np.float64), 1.0 - fill))
        count, labels = check_against_oracle(g, wp, conn, "fp32")
        assert count >= 1
        # count without labels agrees, and device labels agree with host labels
        assert g.hot_areas(wp, conn)[0] == count
        c2, dlab = g.hot_areas(wp, conn, labels=True, device=True)
        assert c2 == count
        assert np.array_equal(dlab.cpu().numpy(), labels)


@pytest.mark.parametrize("conn", [4, 8])
def test_smooth_regions_fp64_512(conn):
    """FP64 grid, box-smoothed noise: blobs of a few cells with holes and
    corner contacts, at three cut-offs."""
    n = 512
    U0 = noise_field(n, 7 + conn, corr=5)
    with Grid(grid_cfg(n), precision="fp64") as g:
        g.load(U0)
        F = g.fluence()
        for q in (0.5, 0.8, 0.97):
            wp = float(np.quantile(F, q))
            count, _ = check_against_oracle(g, wp, conn, "fp64")
            assert count >= 1


def test_degenerate_cut_offs():
    """Cut-off above the peak: no region, every label -1.  Cut-off at zero: the
    whole window is one region labelled 0.  Cut-off equal to the peak: the
    pixels at the peak only (>= includes them)."""
    n = 4096
    U0 = noise_field(n, 3).astype(np.complex64)
    with Grid(grid_cfg(n), precision="fp32") as g:
        g.load(U0)
        F = g.fluence()
        c, lab = g.hot_areas(2.0 * float(F.max()), 4, labels=True)
        assert c == 0 and np.all(lab == -1)
        c, lab = g.hot_areas(0.0, 8, labels=True)
        assert c == 1 and np.all(lab == 0)
        peak = float(F.max())
        c, lab = check_against_oracle(g, peak, 4, "fp32")
        on = np.flatnonzero(F.ravel() >= np.float32(peak))
        assert c >= 1 and np.array_equal(np.flatnonzero(lab.ravel() >= 0), on)


def test_full_size_random_mask_4096():
    """4096^2 FP32 (the dense-grid size), uncorrelated mask at the
    8-neighbour percolation threshold: one spanning region and ~10^5 small ones,
    labels identical to the oracle's."""
    n = 4096
    U0 = noise_field(n, 41).astype(np.complex64)
    with Grid(grid_cfg(n), precision="fp32") as g:
        g.load(U0)
        F = g.fluence()
        wp = float(np.quantile(F.astype(np.float64), 1.0 - 0.407))
        count, _ = check_against_oracle(g, wp, 8, "fp32")
        assert count > 1000


def test_filamented_beam():
    """A noisy beam at 300 P_cr marched into filamentation (Kerr, plasma and
    absorption): its hot areas at a tenth of the peak, as in the paper's count
    of hot areas along z, match the oracle on the same fluence."""
    cfg = configs.physics(256, 1.6, 0.005, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=0.3, P=300 * configs.critical_power(), amp=0.3, ell_cells=3.0, seed=5,
                       phase=0.1, phase_seed=6)
    U0 = beams.make_field(cfg)
    with Grid(cfg, precision="fp32") as g:
        g.load(U0.astype(np.complex64)).step(60)
        F = g.fluence()
        peak = float(F.max())
        for frac in (0.1, 0.3):
            count, _ = check_against_oracle(g, frac * peak, 4, "fp32")
            assert count >= 1


def test_maximum_size_8192():
    """The largest grid (8192^2 FP32): 4-neighbour labels identical to the
    oracle's on a mask at the percolation threshold (one spanning region
    of ~10^7 pixels and ~10^6 small ones)."""
    n = 8192
    U0 = noise_field(n, 77).astype(np.complex64)
    with Grid(grid_cfg(n), precision="fp32") as g:
        g.load(U0)
        F = g.fluence()
        wp = float(np.quantile(F[::4, ::4].astype(np.float64), 1.0 - 0.593))
        count, _ = check_against_oracle(g, wp, 4, "fp32")
        assert count > 10000
