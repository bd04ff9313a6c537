"""GPU spatial moments (Eq. 8) against the oracle's on the GPU's own field,
through the C ABI: FP64 rel 1e-12 (summation order differs), FP32 1e-5 (the
fluence is formed in FP32)."""
import numpy as np
import pytest

import oracle
from paper_2306_15678_gb300 import beams, capi, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu

PQ = [(1, 0), (1, 1), (2, 0), (2, 2), (3, 1), (1, 3), (8, 0), (1, 8)]


@pytest.mark.parametrize("precision,n,tol", [("fp64", 256, 1e-12), ("fp32", 1024, 1e-5), ("fp64", 8, 1e-13)])
def test_moments_match_oracle(precision, n, tol):
    cfg = configs.physics(n, 1.6 if n > 8 else 0.05, 0.5, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=0.3 if n > 8 else 0.01, P=20 * configs.critical_power(), amp=0.2, ell_cells=3.0,
                       seed=31, phase=0.1, phase_seed=32)
    U0 = beams.make_field(cfg)
    with Grid(cfg, precision=precision, diag_every=1) as g:
        g.load(U0.astype(np.complex64) if precision == "fp32" else U0).step(3)
        U = g.field()
        M = g.moments(PQ)
        hpw, _ = g.history()  # the diagnostic records survive the moments
        assert len(hpw) == 3
        assert abs(M[0] / g.power() - 1) < (1e-12 if precision == "fp64" else 2e-6)
    for (p, q), m in zip(PQ, M):
        ref = oracle.moment(U, cfg["L"], p, q)
        assert abs(m / ref - 1) <= tol, (p, q, m, ref)


def test_moments_argument_errors():
    cfg = configs.physics(64, 0.64, 0.5, configs.KERR)
    with Grid(cfg, precision="fp32") as g:
        with pytest.raises(capi.NlseError) as ei:
            g.moments([(1, 0)])
        assert ei.value.status == capi.NLSE_ESTATE
        g.load(np.ones((64, 64), np.complex64))
        for pq in ([(0, 0)], [(17, 0)], [(1, -1)], [(1, 0)] * 9, []):
            with pytest.raises(capi.NlseError) as ei:
                g.moments(pq)
            assert ei.value.status == capi.NLSE_EINVAL
