"""The allocation-free readout (nlse_power_peak_noalloc) against the regular
readout (nlse_power / nlse_peak of a grid holding the same field).

It exists for callers that may not allocate device memory while running; its
scratch is a static device array shared by all calls, so two calls in a row
must both give the right answer.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2306_15678_gb300 import beams, capi, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}  # the readout tolerances of test_gpu_march


def field_case(n, seed):
    cfg = configs.physics(n, 2.56, 1.0, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=0.02 * n / 25.6 * 2.56, P=80 * configs.critical_power(), amp=0.05,
                       ell_cells=3.0, seed=seed, phase=0.1, phase_seed=seed + 1)
    return cfg, beams.make_field(cfg)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_readout_matches_grid_readout_twice(prec):
    stream = torch.cuda.current_stream()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    code = capi.NLSE_FP64 if prec == "fp64" else capi.NLSE_FP32
    for n, seed in ((256, 3), (1024, 4)):
        cfg, U = field_case(n, seed)
        with Grid(cfg, precision=prec) as g:
            g.load(U)
            ref_p, ref_k = g.power(), g.peak()
            dev = torch.from_numpy(U.astype(g.cdtype)).cuda()
        for _ in range(2):  # two calls in a row share the static scratch
            out.zero_()
            capi.nlse_power_peak_noalloc(dev.data_ptr(), n, code, cfg["L"], stream.cuda_stream,
                                         out.data_ptr())
            torch.cuda.synchronize()
            p, k = out.cpu().numpy()
            assert abs(p / ref_p - 1) < TOL[prec], (n, p, ref_p)
            assert abs(k / ref_k - 1) < 10 * TOL[prec], (n, k, ref_k)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dev = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_power_peak_noalloc(dev.data_ptr(), 16384, capi.NLSE_FP32, 1.0, 0, out.data_ptr())
    assert ei.value.status == capi.NLSE_EUNSUPPORTED
