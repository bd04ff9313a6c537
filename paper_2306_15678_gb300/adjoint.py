"""Gradient-based fit of the screen gains: the adjoint of the split-step march
(include/nlse.h, nlse_adjoint_*) behind a torch.autograd.Function.

    loss = NlseFluenceLoss.apply(theta, U0, D, fit)

theta: float64 tensor (6,) of complex screen gains (re, im) on the Kerr, plasma
and absorption terms of Eq. 3; U0: complex tensor (n, n), the input field; D:
float64 tensor (n, n), the target fluence.  loss = sum (|U_M|^2 - D)^2 / sum D^2
after M steps.  backward() returns dJ/dtheta and dJ/dU0 (dJ/dRe + i dJ/dIm, the
PyTorch convention) scaled by the incoming gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .grid import _aligned_workspace, make_params


class AdjointMarch:
    """Owns the device workspace and the nlse_adjoint handle for one problem."""

    def __init__(self, cfg: dict, nsteps: int, ckpt: int = 20, precision: str | None = None,
                 device=None, stream: torch.cuda.Stream | None = None):
        self.params = make_params(cfg, precision, 0)
        self.n = int(cfg["n"])
        self.nsteps, self.ckpt = int(nsteps), int(ckpt)
        self.precision = "fp64" if self.params.precision == capi.NLSE_FP64 else "fp32"
        self.tcdtype = torch.complex128 if self.precision == "fp64" else torch.complex64
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.ws_bytes = capi.nlse_adjoint_workspace_size(self.params, self.nsteps, self.ckpt)
        self._ws, ptr = _aligned_workspace(self.ws_bytes, self.device)
        self.h = capi.nlse_adjoint_create(self.params, self.nsteps, self.ckpt, self.stream.cuda_stream,
                                          ptr, self.ws_bytes)
        self._theta = np.array(list(self.params.theta), dtype=np.float64)

    def set_launch(self, launch: dict) -> None:
        """Column tile and row radix of both sweeps (a tune.tune_launch result)."""
        capi.nlse_adjoint_set_launch(self.h, int(launch["cols"]), int(launch["row_radix"]))

    def set_theta(self, theta) -> None:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(6))
        capi.nlse_adjoint_set_theta(self.h, th.ctypes.data)
        self._theta = th.copy()

    def set_target(self, D) -> None:
        if isinstance(D, torch.Tensor) and D.is_cuda:
            d = D.to(torch.float64).contiguous()
            capi.nlse_adjoint_set_target(self.h, d.data_ptr(), True)
            torch.cuda.current_stream(self.device).synchronize()
        else:
            d = np.ascontiguousarray(D.detach().cpu().numpy() if isinstance(D, torch.Tensor) else D,
                                     dtype=np.float64)
            capi.nlse_adjoint_set_target(self.h, d.ctypes.data, False)

    def forward(self, U0) -> float:
        if isinstance(U0, torch.Tensor) and U0.is_cuda:
            u = U0.detach().to(self.tcdtype).contiguous()
            return capi.nlse_adjoint_forward(self.h, u.data_ptr(), True)
        a = np.ascontiguousarray(U0.detach().cpu().numpy() if isinstance(U0, torch.Tensor) else U0,
                                 dtype=np.complex128 if self.precision == "fp64" else np.complex64)
        return capi.nlse_adjoint_forward(self.h, a.ctypes.data, False)

    def backward(self):
        dth = np.zeros(6)
        dU = torch.empty((self.n, self.n), dtype=self.tcdtype, device=self.device)
        capi.nlse_adjoint_backward(self.h, dth.ctypes.data, dU.data_ptr(), True)
        return dth, dU

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            capi.nlse_adjoint_destroy(self.h)
            self.h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NlseFluenceLoss(torch.autograd.Function):
    """loss = J(theta, U0) through the CUDA march; gradients through its adjoint."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, U0: torch.Tensor, D: torch.Tensor, fit: AdjointMarch):
        fit.set_theta(theta.detach().cpu().numpy())
        fit.set_target(D)
        J = fit.forward(U0)
        ctx.fit = fit
        ctx.theta_dtype, ctx.theta_device = theta.dtype, theta.device
        ctx.u_dtype, ctx.u_device = U0.dtype, U0.device
        return torch.tensor(J, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        dth, dU = ctx.fit.backward()
        g = float(grad_out)
        d_theta = torch.tensor(dth * g, dtype=ctx.theta_dtype, device=ctx.theta_device)
        d_U = (dU * g).to(dtype=ctx.u_dtype, device=ctx.u_device)
        return d_theta, d_U, None, None
