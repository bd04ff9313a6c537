"""GPU adjoint of the split-step march (loss, adjoint step, checkpointing)
against the FP64 oracle's adjoint and against central finite differences.

Tolerances: FP64 GPU vs FP64 oracle to 1e-9; FP32 GPU vs FP64 (oracle or
finite differences) rel error <= 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_15678_gb300 import beams, configs
from paper_2306_15678_gb300.adjoint import AdjointMarch, NlseFluenceLoss

pytestmark = pytest.mark.gpu


def case(n=64, nsteps=20, dz=0.5, pcr=300.0, L=1.6, w0=0.12):
    """Plasma-clamping regime, well conditioned at dz = 5 mm."""
    cfg = configs.physics(n, L, dz, configs.ALL_TERMS)
    cfg["beam"] = dict(w0=w0, P=pcr * configs.critical_power(), amp=0.05, ell_cells=3.0, seed=21,
                       phase=0.1, phase_seed=22)
    U0 = beams.make_field(cfg)
    other = dict(cfg, beam=dict(cfg["beam"], w0=w0 * 1.1, seed=23, P=pcr * 0.9 * configs.critical_power()))
    D = np.abs(beams.make_field(other)) ** 2
    return cfg, U0, D


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def run_gpu(cfg, U0, D, nsteps, ckpt, prec, theta=None):
    fit = AdjointMarch(cfg, nsteps, ckpt, precision=prec)
    try:
        if theta is not None:
            fit.set_theta(theta)
        fit.set_target(D)
        J = fit.forward(U0)
        dth, dU = fit.backward()
        return J, dth, dU.cpu().numpy().astype(np.complex128)
    finally:
        fit.close()


def test_fp64_adjoint_matches_oracle_adjoint():
    cfg, U0, D = case()
    J0, t0, g0 = oracle.adjoint(U0, D, cfg, 20, ckpt=6)
    J, t, g = run_gpu(cfg, U0, D, 20, 6, "fp64")
    _, _, pk = oracle.march(U0, cfg, 20)
    assert pk.max() > 3e13  # plasma and absorption are active
    assert abs(J / J0 - 1) < 1e-10
    assert np.max(np.abs(t - t0)) <= 1e-9 * np.max(np.abs(t0))
    assert rel(g, g0) < 1e-9


def test_fp32_adjoint_matches_fp64_oracle_within_1e3():
    cfg, U0, D = case()
    U0 = U0.astype(np.complex64).astype(np.complex128)
    J0, t0, g0 = oracle.adjoint(U0, D, cfg, 20, ckpt=6)
    J, t, g = run_gpu(cfg, U0, D, 20, 6, "fp32")
    assert abs(J / J0 - 1) < 1e-4
    for j in range(6):
        assert abs(t[j] - t0[j]) <= 1e-3 * max(abs(t0[j]), 1e-3 * np.max(np.abs(t0))), (j, t[j], t0[j])
    assert rel(g, g0) < 1e-3


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_matches_central_differences_of_fp64_forward(prec):
    """dJ/dtheta against central differences (h = 1e-4, Richardson-extrapolated
    with h/2) of the FP64 GPU forward; dJ/dU0 along a random direction."""
    cfg, U0, D = case()
    U0 = U0.astype(np.complex64).astype(np.complex128)
    _, t, g = run_gpu(cfg, U0, D, 20, 5, prec)
    fit = AdjointMarch(cfg, 20, 5, precision="fp64")
    fit.set_target(D)
    try:
        def J(theta=None, U=U0):
            fit.set_theta(theta if theta is not None else cfg["theta"])
            return fit.forward(U)

        h = 1e-4
        for j in range(6):
            def cd(hh):
                tp = np.array(cfg["theta"], float); tp[j] += hh
                tm = np.array(cfg["theta"], float); tm[j] -= hh
                return (J(tp) - J(tm)) / (2 * hh)
            fd = (4 * cd(h / 2) - cd(h)) / 3
            assert abs(t[j] - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.max(np.abs(t))), (j, t[j], fd)
        rng = np.random.default_rng(4)
        d = (rng.standard_normal(U0.shape) + 1j * rng.standard_normal(U0.shape)) * np.abs(U0).max()
        hh = 2e-5
        def cdu(e):
            return (J(None, U0 + e * d) - J(None, U0 - e * d)) / (2 * e)
        fd = (4 * cdu(hh / 2) - cdu(hh)) / 3
        an = float(np.real(np.vdot(g, d)))
        assert abs(an - fd) <= 1e-3 * abs(fd), (an, fd)
    finally:
        fit.close()


def test_checkpoint_spacing_does_not_change_the_gradient():
    cfg, U0, D = case()
    res = [run_gpu(cfg, U0, D, 20, k, "fp32") for k in (1, 6, 20)]
    for J, t, g in res[1:]:
        assert J == res[0][0]
        assert np.array_equal(t, res[0][1])
        assert np.array_equal(g, res[0][2])


def test_launch_shape_keeps_the_gradient():
    """The staged row pass and any staged column tile of radix 16 give the
    bits of the default launch shape; codes the size does not offer are
    refused."""
    from paper_2306_15678_gb300 import capi
    cfg, U0, D = case(n=2048, nsteps=4, L=4.0, w0=0.5)
    out = []
    for launch in ({}, {"cols": capi.NLSE_COL_TMA | 2, "row_radix": capi.NLSE_ROW_STAGED | 16}):
        fit = AdjointMarch(cfg, 4, 2, precision="fp32")
        try:
            if launch:
                fit.set_launch(launch)
            fit.set_target(D)
            J = fit.forward(U0)
            dth, dU = fit.backward()
            out.append((J, dth, dU.cpu().numpy()))
        finally:
            fit.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    small, U0s, Ds = case()
    fit = AdjointMarch(small, 4, 2, precision="fp32")
    try:
        with pytest.raises(capi.NlseError) as ei:  # n = 64: no staged row pass
            fit.set_launch({"cols": 1, "row_radix": capi.NLSE_ROW_STAGED | 16})
        assert ei.value.status == capi.NLSE_EUNSUPPORTED
        with pytest.raises(capi.NlseError):
            fit.set_launch({"cols": 3, "row_radix": 16})
    finally:
        fit.close()


def test_autograd_function_gives_the_adjoint():
    cfg, U0, D = case()
    fit = AdjointMarch(cfg, 20, 5, precision="fp32")
    try:
        theta = torch.tensor(cfg["theta"], dtype=torch.float64, requires_grad=True)
        U = torch.from_numpy(U0.astype(np.complex64)).cuda().requires_grad_(True)
        Dt = torch.from_numpy(D).cuda()
        loss = NlseFluenceLoss.apply(theta, U, Dt, fit)
        (3.0 * loss).backward()
        J, t, g = run_gpu(cfg, U0.astype(np.complex64), D, 20, 5, "fp32")
        assert float(loss) == pytest.approx(J, rel=1e-12)
        assert np.allclose(theta.grad.numpy(), 3.0 * t, rtol=1e-12, atol=0)
        assert rel(U.grad.cpu().numpy(), 3.0 * g) < 1e-6
        # torch's convention for a real loss of a complex leaf: d/dRe + i d/dIm
        z = torch.tensor([1.0 + 2.0j], requires_grad=True)
        (z.abs() ** 2).sum().backward()
        assert complex(z.grad[0]) == pytest.approx(2.0 + 4.0j)
    finally:
        fit.close()


def sparse_fit_case():
    """The 512^2 sparse-grid fit geometry (8 cm window, 2.5 cm steps, checkpoint
    every 20, FP32 field).  The target -- the 8x8 box mean of a dense 4096^2
    fluence in the benchmark -- is replaced by the fluence of a neighbouring
    beam of the same shape, so that the check needs no dense run."""
    cfg = configs.cfg_adjoint_sparse()
    U0 = beams.make_field(cfg).astype(np.complex64).astype(np.complex128)
    other = dict(cfg, beam=dict(cfg["beam"], w0=1.05, seed=7))
    D = np.abs(beams.make_field(other)) ** 2
    return cfg, U0, D


def test_sparse_grid_fit_to_first_collapse_fp32_vs_differences():
    """150 steps (3.75 m): just past the first step whose peak reaches w_pf.  The
    FP32 adjoint against central differences of the FP64 forward (<= 1e-3) and
    against the FP64 adjoint."""
    cfg, U0, D = sparse_fit_case()
    J32, t32, g32 = run_gpu(cfg, U0, D, 150, 20, "fp32")
    J64, t64, g64 = run_gpu(cfg, U0, D, 150, 20, "fp64")
    assert abs(J32 / J64 - 1) < 1e-4
    assert rel(g32, g64) < 1e-3
    big = np.max(np.abs(t64))
    fit = AdjointMarch(cfg, 150, 20, precision="fp64")
    fit.set_target(D)
    try:
        for j in range(6):
            def cd(hh):
                tp = np.array(cfg["theta"], float); tp[j] += hh
                tm = np.array(cfg["theta"], float); tm[j] -= hh
                fit.set_theta(tp); jp = fit.forward(U0)
                fit.set_theta(tm); jm = fit.forward(U0)
                return (jp - jm) / (2 * hh)
            fd = (4 * cd(5e-6) - cd(1e-5)) / 3
            assert abs(t32[j] - fd) <= 1e-3 * max(abs(fd), 1e-3 * big), (j, t32[j], fd)
            assert abs(t64[j] - t32[j]) <= 1e-3 * max(abs(t64[j]), 1e-3 * big)
    finally:
        fit.close()


def test_sparse_grid_fit_full_run_is_deterministic_and_finite():
    """The whole 400-step run.  Past the first collapse the 2.5 cm march is
    chaotic (finite differences of J no longer converge as h -> 0 and FP32/FP64
    trajectories separate), so here the checks are the ones that hold at any
    length: finite results and bit-identical gradients for different checkpoint
    spacings."""
    cfg, U0, D = sparse_fit_case()
    a = run_gpu(cfg, U0, D, 400, 20, "fp32")
    b = run_gpu(cfg, U0, D, 400, 40, "fp32")
    assert np.isfinite(a[0]) and np.all(np.isfinite(a[1])) and np.all(np.isfinite(a[2]))
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_large_grid_adjoint_8192_against_differences():
    """The large batched adjoint's grid (8192^2, 16 cm window, w0 = 3 cm,
    P = 500 P_cr), a few steps with sqrt(M) checkpointing: the FP32 gradient
    against central differences of the FP64 GPU forward (Richardson, h = 1e-4)
    for the six gains, and dJ/dU0 along a random direction."""
    cfg = configs.cfg_large_adjoint(1)[0]
    M = 6
    k = configs.sqrt_checkpoint(M)
    U0 = beams.make_field(cfg).astype(np.complex64).astype(np.complex128)
    other = dict(cfg, beam=dict(cfg["beam"], w0=cfg["beam"]["w0"] * 1.02, seed=5099))
    D = np.abs(beams.make_field(other)) ** 2
    _, t, g = run_gpu(cfg, U0, D, M, k, "fp32")
    assert np.all(np.isfinite(t)) and np.all(np.isfinite(g))
    fit = AdjointMarch(cfg, M, k, precision="fp64")
    fit.set_target(D)
    try:
        def J(theta=None, U=U0):
            fit.set_theta(theta if theta is not None else cfg["theta"])
            return fit.forward(U)

        h = 1e-4
        for j in range(6):
            def cd(hh):
                tp = np.array(cfg["theta"], float); tp[j] += hh
                tm = np.array(cfg["theta"], float); tm[j] -= hh
                return (J(tp) - J(tm)) / (2 * hh)
            fd = (4 * cd(h / 2) - cd(h)) / 3
            assert abs(t[j] - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.max(np.abs(t))), (j, t[j], fd)
        rng = np.random.default_rng(6)
        d = (rng.standard_normal(U0.shape) + 1j * rng.standard_normal(U0.shape)) * np.abs(U0).max()
        hh = 2e-5
        def cdu(e):
            return (J(None, U0 + e * d) - J(None, U0 - e * d)) / (2 * e)
        fd = (4 * cdu(hh / 2) - cdu(hh)) / 3
        an = float(np.real(np.vdot(g, d)))
        assert abs(an - fd) <= 1e-3 * abs(fd), (an, fd)
    finally:
        fit.close()
