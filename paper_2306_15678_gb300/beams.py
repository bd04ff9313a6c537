"""Seeded synthetic input fields (the initial beams of Eq. 7).

This module is the one input generator shared by the CUDA path, the oracle and
the tests.  It holds none of the march's arithmetic: it only draws noise and
samples the initial Gaussian beam on the cell-centred grid.

Initial field (Eq. 7 with seeded perturbations):

    U0(x, y) = A exp(-r^2 / w0^2) (1 + a eta(x, y)) exp(i b eta'(x, y)),

with r^2 = x^2 + y^2 on cell centres x_j = (j - N/2 + 1/2) dx, and
A^2 = 2 P / (pi w0^2) so that the beam carries power P (the printed
"P = pi A r^2" is read as the Gaussian power integral (pi/2) A^2 w0^2).
eta, eta' are i.i.d. N(0, 1) draws (NumPy PCG64, given seeds) circularly
convolved with exp(-d^2 / l^2) (l in cells) and rescaled to zero mean and unit
standard deviation.
"""
from __future__ import annotations

import math

import numpy as np


def cell_centres(n: int, L: float) -> np.ndarray:
    dx = L / n
    return (np.arange(n, dtype=np.float64) - n / 2 + 0.5) * dx


def smoothed_noise(n: int, ell_cells: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian noise with a Gaussian correlation of
    length ell_cells (in cells), periodic on the n x n grid."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    eta = rng.standard_normal((n, n))
    if ell_cells and ell_cells > 0:
        d = np.arange(n, dtype=np.float64)
        d = np.minimum(d, n - d)
        g1 = np.exp(-(d * d) / (ell_cells * ell_cells))
        kern = np.outer(g1, g1)  # exp(-(dx^2 + dy^2)/l^2) is separable
        eta = np.fft.irfft2(np.fft.rfft2(eta) * np.fft.rfft2(kern), s=(n, n))
    eta = eta - eta.mean()
    sd = eta.std()
    return eta / sd if sd > 0 else eta


def gaussian_beam(n: int, L: float, w0: float, P: float, amp: float = 0.0,
                  ell_cells: float = 0.0, seed: int | None = None, phase: float = 0.0,
                  phase_seed: int | None = None) -> np.ndarray:
    """complex128 [n, n] row-major (row = y, column = x) initial field in sqrt(W)/cm."""
    x = cell_centres(n, L)
    A = math.sqrt(2.0 * P / (math.pi * w0 * w0))
    gx = np.exp(-(x * x) / (w0 * w0))
    U = A * np.outer(gx, gx).astype(np.complex128)
    if amp and seed is not None:
        U *= 1.0 + amp * smoothed_noise(n, ell_cells, seed)
    if phase and phase_seed is not None:
        U *= np.exp(1j * phase * smoothed_noise(n, ell_cells, phase_seed))
    return U


def make_field(cfg: dict) -> np.ndarray:
    """Initial field of a workload dict from ``configs``."""
    b = cfg["beam"]
    return gaussian_beam(cfg["n"], cfg["L"], b["w0"], b["P"], b.get("amp", 0.0),
                         b.get("ell_cells", 0.0), b.get("seed"), b.get("phase", 0.0),
                         b.get("phase_seed"))


def box_mean(a: np.ndarray, ds: int) -> np.ndarray:
    """Mean over aligned ds x ds blocks (complex or real)."""
    n = a.shape[0]
    m = n // ds
    return a.reshape(m, ds, m, ds).mean(axis=(1, 3))


def turbulence_draws(n: int, seed: int) -> np.ndarray:
    """The random draws xi of the spectral turbulent screen (Eqs. 9-10): n x n
    i.i.d. complex unit Gaussians (real and imaginary parts N(0, 1/2); NumPy
    PCG64, given seed), in FFT bin order."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * math.sqrt(0.5)


def ga_draws(seed: int, count: int) -> np.ndarray:
    """The uniform [0, 1) draws a genetic search consumes, in order (NumPy
    PCG64, given seed): gene sampling, roulette picks, crossover and mutation
    all read this one stream, so that two implementations of the search given
    the same stream make the same choices."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return rng.random(int(count))


def fit_beam_set(n: int = 256, count: int = 2) -> list:
    """Eq. 7 test beams of the fit: Gaussian beams U_n = A_n exp(-(r/r_n)^2)
    spanning the paper's range (P from 3 to 9 P_cr, r_n from 0.5 to 2.5 mm),
    each on a window of 8 r_n: a list of (r_n in cm, P / P_cr, L in cm)."""
    out = []
    for i in range(count):
        t = i / max(count - 1, 1)
        r = 0.05 + t * (0.25 - 0.05)
        out.append((r, 3.0 + 6.0 * t, 8.0 * r))
    return out
