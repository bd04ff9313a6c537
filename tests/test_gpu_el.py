"""Effective-lens march (Sec. 2, Eq. 2, Fig. 1): split steps until the peak
reaches the pre-filamentation level w_pf, then the lens screen of the field and
diffraction over the lens length, then split steps again -- against the same
sequence of oracle calls (FP64, rel-L2 <= 1e-10, identical events)."""
import numpy as np
import pytest

import oracle
from paper_2306_15678_gb300 import beams, configs
from paper_2306_15678_gb300.el import el_march

pytestmark = pytest.mark.gpu

LENS = dict(l_dif=4e-4, w_l=5e11, conn=4, re=[(0.05, -0.5, 30.0, 0.0), (0.1, 0.2, 20.0, 0.5)],
            im=[(0.06, 0.6, 25.0, 0.0)])


def test_el_march_matches_oracle_sequence():
    cfg = configs.physics(128, 1.28, 1.0, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=0.1, P=8 * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=5, phase=0.05,
                       phase_seed=6)
    U0 = beams.make_field(cfg)
    w_pf, l_f, nsteps = 2e12, 30.0, 40
    U, armed, events, z = U0, True, [], 0.0
    for s in range(nsteps):
        U, _, _ = oracle.march(U, cfg, 1, record=False)
        z += cfg["dz"]
        pk = oracle.peak(U)
        if armed and pk >= w_pf:
            U, cent = oracle.effective_lens(U, cfg, LENS)
            U = oracle.linear(U, dict(cfg, terms=configs.DIFFRACTION, dz=l_f))
            z += l_f
            events.append((s, z, len(cent)))
            armed = False
        elif not armed and pk < w_pf:
            armed = True
    r = el_march(cfg, U0, LENS, w_pf, l_f, nsteps, precision="fp64")
    assert len(events) == 2
    assert [(s, c) for s, _, c in r["events"]] == [(s, c) for s, _, c in events]
    assert abs(r["z"] - z) < 1e-9
    assert np.linalg.norm(r["field"] - U) / np.linalg.norm(U) <= 1e-10
