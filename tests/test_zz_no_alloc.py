"""The allocation-free readout (nlse_power_peak_noalloc) against the FP64 oracle's
power and peak of the same field bytes, and against the regular readout
(nlse_power / nlse_peak of a grid holding the same field).

It exists for callers that may not allocate device memory while running; its
scratch is a static device array shared by all calls, so two calls in a row
must both give the right answer.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_15678_gb300 import beams, capi, configs
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu

# against the oracle on the same bytes: both sum |U|^2 in FP64 (FP32 values are
# widened exactly), so only the summation order differs
TOL_ORACLE = {"fp64": 1e-12, "fp32": 2e-6}
TOL_GRID = {"fp64": 1e-12, "fp32": 2e-5}  # the readout tolerances of test_gpu_march


def field_case(n, seed):
    cfg = configs.physics(n, 2.56, 1.0, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=0.02 * n / 25.6 * 2.56, P=80 * configs.critical_power(), amp=0.05,
                       ell_cells=3.0, seed=seed, phase=0.1, phase_seed=seed + 1)
    return cfg, beams.make_field(cfg)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_readout_matches_oracle_and_grid_twice(prec):
    stream = torch.cuda.current_stream()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    code = capi.NLSE_FP64 if prec == "fp64" else capi.NLSE_FP32
    for n, seed in ((256, 3), (1024, 4), (37, 5)):
        cfg, U = field_case(n, seed)
        ct = np.complex128 if prec == "fp64" else np.complex64
        Ub = U.astype(ct)
        ref_p = oracle.power(Ub.astype(np.complex128), cfg["L"])
        ref_k = oracle.peak(Ub.astype(np.complex128))
        grid_p = grid_k = None
        if n & (n - 1) == 0:
            with Grid(cfg, precision=prec) as g:
                g.load(Ub)
                grid_p, grid_k = g.power(), g.peak()
        dev = torch.from_numpy(Ub).cuda()
        for _ in range(2):  # two calls in a row share the static scratch
            out.fill_(-1.0)
            capi.nlse_power_peak_noalloc(dev.data_ptr(), n, code, cfg["L"], stream.cuda_stream,
                                         out.data_ptr())
            torch.cuda.synchronize()
            p, k = out.cpu().numpy()
            assert abs(p / ref_p - 1) < TOL_ORACLE[prec], (n, p, ref_p)
            assert abs(k / ref_k - 1) < TOL_ORACLE[prec], (n, k, ref_k)
            if grid_p is not None:
                assert abs(p / grid_p - 1) < TOL_GRID[prec], (n, p, grid_p)
                assert abs(k / grid_k - 1) < 10 * TOL_GRID[prec], (n, k, grid_k)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dev = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_power_peak_noalloc(dev.data_ptr(), 16384, capi.NLSE_FP32, 1.0, 0, out.data_ptr())
    assert ei.value.status == capi.NLSE_EUNSUPPORTED


def test_noalloc_rejects_misaligned_pointers_before_any_launch():
    """The host refuses pointers the kernels could not read or write whole
    values through; nothing is launched, so nothing is read or written."""
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    f32 = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    f64 = torch.zeros((8, 8), dtype=torch.complex128, device="cuda")
    cases = [(f32.data_ptr() + 4, capi.NLSE_FP32, out.data_ptr()),
             (f64.data_ptr() + 8, capi.NLSE_FP64, out.data_ptr()),
             (f32.data_ptr(), capi.NLSE_FP32, out.data_ptr() + 4)]
    for fp, prec, op in cases:
        with pytest.raises(capi.NlseError) as ei:
            capi.nlse_power_peak_noalloc(fp, 4, prec, 1.0, 0, op)
        assert ei.value.status == capi.NLSE_EINVAL
    torch.cuda.synchronize()
    assert torch.all(out == 0)
