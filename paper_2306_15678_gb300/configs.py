"""Physical parameters and the five workloads of the split-step NLSE march.

Plain numbers only: no arithmetic of the method lives here.  The values that
the paper does not print are readings of it:

* carrier wavelength 800 nm (Sec. 2, below Eq. 1), n0 = 1, air n2 = 3.2e-19 cm^2/W;
* multiphoton order K = 8 (Eq. 3 "m-th order"; O2 at 800 nm);
* sigma_8 = 2.88e-99 s^-1 cm^16 W^-8, rho_nt = 5.4e18 cm^-3, rho_c = 1.7e21 cm^-3,
  beta_8 = 3.1e-98 cm^13 W^-7 (commonly tabulated air values);
* tau_pl = 87.5 fs, from 35 mJ at about 400 GW (Sec. 3.3);
* P_cr = lambda0^2 / (2 pi n0 n2) -- reproduces 380 GW = 112 P_cr (Sec. 3.2)
  at n2 = 3.0e-19.

Each workload dict carries every field of the parameter record consumed by both
the CUDA library and the oracle, plus the beam recipe used by ``beams.make_field``.
"""
from __future__ import annotations

import math

KERR, PLASMA, MPA, DIFFRACTION = 1, 2, 4, 8
ALL_TERMS = KERR | PLASMA | MPA | DIFFRACTION

LAMBDA0 = 8.0e-5       # cm (800 nm)
N0 = 1.0
N2_AIR = 3.2e-19       # cm^2/W
K_MPI = 8
SIGMA_K = 2.88e-99     # s^-1 cm^16 W^-8
RHO_NT = 5.4e18        # cm^-3
RHO_C = 1.7e21         # cm^-3
TAU_PL = 87.5e-15      # s
BETA_K = 3.1e-98       # cm^13 W^-7
NOMINAL_THETA = (1.0, 0.0, 1.0, 0.0, 1.0, 0.0)

# pre-filamentation intensity w_pf (Sec. 2, before Eq. 4): the lower end of 2..8 TW/cm^2
W_PF = 2.0e12          # W/cm^2


def critical_power(lambda0: float = LAMBDA0, n0: float = N0, n2: float = N2_AIR) -> float:
    """Critical self-focusing power lambda0^2/(2 pi n0 n2) in W."""
    return lambda0 * lambda0 / (2.0 * math.pi * n0 * n2)


def physics(n: int, L: float, dz: float, terms: int = ALL_TERMS, theta=NOMINAL_THETA) -> dict:
    return dict(n=int(n), L=float(L), dz=float(dz), lambda0=LAMBDA0, n0=N0, n2=N2_AIR,
                K=K_MPI, sigmaK=SIGMA_K, rho_nt=RHO_NT, rho_c=RHO_C, tau_pl=TAU_PL,
                betaK=BETA_K, terms=int(terms), theta=tuple(float(t) for t in theta))


def cfg_plain_fp64() -> dict:
    """256^2 FP64, 25.6 mm window, w0 = 2 mm, P = 10 P_cr, (1 + 0.05 eta) with a
    4-cell correlation length, Kerr + diffraction, 200 steps of 1 cm."""
    d = physics(256, 2.56, 1.0, KERR | DIFFRACTION)
    d.update(name="plain-fp64-256", precision="fp64", nsteps=200,
             beam=dict(w0=0.2, P=10.0 * critical_power(), amp=0.05, ell_cells=4.0, seed=1,
                       phase=0.0, phase_seed=None))
    return d


def cfg_dense_fp32() -> dict:
    """4096^2 FP32 (FP64 reductions), 8 cm window, w0 = 1 cm, P = 100 P_cr,
    5 % amplitude noise (0.5 mm correlation) + 0.1 rad phase noise, full screen,
    2000 steps of 5 mm."""
    n, L = 4096, 8.0
    ell = 0.05 / (L / n)
    d = physics(n, L, 0.5, ALL_TERMS)
    d.update(name="dense-fp32-4096", precision="fp32", nsteps=2000,
             beam=dict(w0=1.0, P=100.0 * critical_power(), amp=0.05, ell_cells=ell, seed=2,
                       phase=0.1, phase_seed=102))
    return d


def cfg_batch(nbeams: int = 64, seed: int = 3, sizes=(512, 1024, 2048)) -> list:
    """64 beams, N drawn from {512, 1024, 2048}, P ~ U[20, 200] P_cr,
    w0 ~ U[0.5, 1.5] cm, L = 8 w0, noise seeds 3000 + b, full screen, FP32,
    500 steps of 5 mm."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(nbeams):
        n = int(rng.choice(np.asarray(sizes)))
        Pm = float(rng.uniform(20.0, 200.0))
        w0 = float(rng.uniform(0.5, 1.5))
        L = 8.0 * w0
        d = physics(n, L, 0.5, ALL_TERMS)
        d.update(name=f"batch-{b}", precision="fp32", nsteps=500,
                 beam=dict(w0=w0, P=Pm * critical_power(), amp=0.05,
                           ell_cells=0.05 / (L / n), seed=3000 + b, phase=0.1,
                           phase_seed=4000 + b))
        out.append(d)
    return out


def cfg_adjoint_sparse() -> dict:
    """512^2 sparse grid over the 8 cm window of the dense problem, 400 steps of
    2.5 cm (10 m, like 2000 x 5 mm), checkpoint every 20, FP32 field."""
    d = physics(512, 8.0, 2.5, ALL_TERMS)
    d.update(name="adjoint-sparse-512", precision="fp32", nsteps=400, ckpt=20,
             beam=dict(w0=1.0, P=100.0 * critical_power(), amp=0.05,
                       ell_cells=0.05 / (8.0 / 512), seed=2, phase=0.1, phase_seed=102))
    return d


def cfg_large_adjoint(nbeams: int = 8) -> list:
    """8 beams of 8192^2, 16 cm window, w0 = 3 cm, P = 500 P_cr, 5 % noise,
    full screen, 3000 steps of 5 mm."""
    out = []
    n, L = 8192, 16.0
    for b in range(nbeams):
        d = physics(n, L, 0.5, ALL_TERMS)
        d.update(name=f"large-{b}", precision="fp32", nsteps=3000,
                 beam=dict(w0=3.0, P=500.0 * critical_power(), amp=0.05,
                           ell_cells=0.05 / (L / n), seed=5000 + b, phase=0.0,
                           phase_seed=None))
        out.append(d)
    return out


def sqrt_checkpoint(nsteps: int) -> int:
    """Checkpoint spacing ceil(sqrt(M)) for an M-step adjoint: about 2 sqrt(M)
    stored fields (checkpoints plus one recomputed segment) instead of M."""
    return max(1, math.ceil(math.sqrt(int(nsteps))))


def scaled(cfg: dict, n: int, nsteps: int | None = None, L: float | None = None) -> dict:
    """Same physics and beam on another grid size (for oracle-sized parity runs)."""
    d = dict(cfg)
    d["beam"] = dict(cfg["beam"])
    oldL = cfg["L"]
    d["L"] = float(L) if L is not None else oldL
    # keep the physical noise correlation length
    ell_cm = cfg["beam"]["ell_cells"] * oldL / cfg["n"]
    d["n"] = int(n)
    d["beam"]["ell_cells"] = ell_cm / (d["L"] / n)
    if nsteps is not None:
        d["nsteps"] = int(nsteps)
    return d
