"""Python view of one transverse grid marched by the C ABI (include/nlse.h).

PyTorch owns the device workspace and supplies the CUDA stream; libnlse.so does
all the work.  Host arrays are numpy; device arrays are torch tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi

_PREC = {"fp64": capi.NLSE_FP64, "fp32": capi.NLSE_FP32}
_SCHEME = {"lie": capi.NLSE_LIE, "strang": capi.NLSE_STRANG}


def make_params(cfg: dict, precision: str | None = None, diag_every: int = 0) -> capi.nlse_params:
    """nlse_params from a workload dict of ``configs`` (physical units)."""
    p = capi.nlse_params()
    p.n = int(cfg["n"])
    p.K = int(cfg["K"])
    p.terms = int(cfg["terms"])
    p.precision = _PREC[precision or cfg.get("precision", "fp32")]
    for f in ("L", "dz", "lambda0", "n0", "n2", "sigmaK", "rho_nt", "rho_c", "tau_pl", "betaK"):
        setattr(p, f, float(cfg[f]))
    th = cfg.get("theta", (1.0, 0.0, 1.0, 0.0, 1.0, 0.0))
    for i in range(6):
        p.theta[i] = float(th[i])
    p.diag_every = int(diag_every)
    scheme = cfg.get("scheme", "lie")
    if scheme not in _SCHEME:
        raise ValueError(f"scheme {scheme!r}: expected 'lie' or 'strang'")
    screen = cfg.get("screen", "frozen")
    if screen not in ("frozen", "exact"):
        raise ValueError(f"screen {screen!r}: expected 'frozen' or 'exact'")
    p.scheme = _SCHEME[scheme] | (capi.NLSE_EXACT_SCREEN if screen == "exact" else 0)
    return p


def _aligned_workspace(nbytes: int, device) -> tuple[torch.Tensor, int]:
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    ptr = buf.data_ptr()
    return buf, (ptr + 255) & ~255


class Grid:
    """One n x n field marched by split-step Fourier steps on the GPU."""

    def __init__(self, cfg: dict, precision: str | None = None, diag_every: int = 0,
                 device: str | torch.device | None = None, stream: torch.cuda.Stream | None = None):
        self.cfg = cfg
        self.params = make_params(cfg, precision, diag_every)
        self.n = int(cfg["n"])
        self.precision = "fp64" if self.params.precision == capi.NLSE_FP64 else "fp32"
        self.cdtype = np.complex128 if self.precision == "fp64" else np.complex64
        self.rdtype = np.float64 if self.precision == "fp64" else np.float32
        self.tcdtype = torch.complex128 if self.precision == "fp64" else torch.complex64
        self.trdtype = torch.float64 if self.precision == "fp64" else torch.float32
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.ws_bytes = capi.nlse_workspace_size(self.params)
        self._ws, ptr = _aligned_workspace(self.ws_bytes, self.device)
        self.h = capi.nlse_create(self.params, self.stream.cuda_stream, ptr, self.ws_bytes)
        self._keep = None

    # ------------------------------------------------------------------ io
    def load(self, U) -> "Grid":
        if isinstance(U, torch.Tensor) and U.is_cuda:
            t = U.to(self.tcdtype).contiguous()
            self._keep = t
            capi.nlse_load_field(self.h, t.data_ptr(), True)
        else:
            a = np.ascontiguousarray(U.cpu().numpy() if isinstance(U, torch.Tensor) else U,
                                     dtype=self.cdtype)
            assert a.shape == (self.n, self.n)
            capi.nlse_load_field(self.h, a.ctypes.data, False)
        return self

    def step(self, nsteps: int = 1) -> "Grid":
        capi.nlse_step(self.h, int(nsteps))
        return self

    def step_timed(self, nsteps: int) -> tuple[float, float]:
        """Step and return summed (column-pass, row-pass) kernel times in ms."""
        return capi.nlse_step_timed(self.h, int(nsteps))

    @property
    def steps_taken(self) -> int:
        return capi.nlse_steps_taken(self.h)

    def power(self) -> float:
        return capi.nlse_power(self.h)

    def peak(self) -> float:
        return capi.nlse_peak(self.h)

    def field(self, device: bool = False):
        if device:
            out = torch.empty((self.n, self.n), dtype=self.tcdtype, device=self.device)
            capi.nlse_read_field(self.h, out.data_ptr(), True)
            return out
        out = np.empty((self.n, self.n), dtype=self.cdtype)
        capi.nlse_read_field(self.h, out.ctypes.data, False)
        return out

    def fluence(self, downsample: int = 1, device: bool = False):
        m = self.n // downsample
        if device:
            out = torch.empty((m, m), dtype=self.trdtype, device=self.device)
            capi.nlse_fluence(self.h, out.data_ptr(), True, downsample)
            return out
        out = np.empty((m, m), dtype=self.rdtype)
        capi.nlse_fluence(self.h, out.ctypes.data, False, downsample)
        return out

    def hot_areas(self, w_p: float, connectivity: int = 4, labels: bool = False, device: bool = False):
        """Number of hot areas (regions with fluence >= w_p, Sec. 3.3) and, with
        labels=True, the n x n int32 labels (-1 outside, else the smallest
        row-major index of the region): (count, labels or None)."""
        if not labels:
            return capi.nlse_hot_areas(self.h, w_p, connectivity, 0, False), None
        if device:
            out = torch.empty((self.n, self.n), dtype=torch.int32, device=self.device)
            return capi.nlse_hot_areas(self.h, w_p, connectivity, out.data_ptr(), True), out
        out = np.empty((self.n, self.n), dtype=np.int32)
        return capi.nlse_hot_areas(self.h, w_p, connectivity, out.ctypes.data, False), out

    def turbulent_screen(self, xi, tau: float, k_h: float, thickness: float) -> "Grid":
        """Turbulent layer of Eqs. 9-10: U <- U exp(-i thickness eps_t / (2 k0)),
        eps_t the spectral screen of the draws xi (n x n complex, FFT bin order)
        with step amplitude tau up to the cut-off k_h (rad/cm)."""
        if isinstance(xi, torch.Tensor) and xi.is_cuda:
            t = xi.to(self.tcdtype).contiguous()
            capi.nlse_turbulent_screen(self.h, t.data_ptr(), True, tau, k_h, thickness)
            self._keep = t
        else:
            a = np.ascontiguousarray(xi.cpu().numpy() if isinstance(xi, torch.Tensor) else xi, dtype=self.cdtype)
            assert a.shape == (self.n, self.n)
            capi.nlse_turbulent_screen(self.h, a.ctypes.data, False, tau, k_h, thickness)
        return self

    def effective_lens(self, lens: dict, w_dif: bool = False):
        """Effective-lens screen of Eqs. 4-6 on the current field (see
        capi.make_lens for the dict).  Returns (count, centres as row-major
        int32 indices, w_dif as a device tensor or None)."""
        need = capi.nlse_lens_scratch_size(self.params)
        if getattr(self, "_lens_scratch", None) is None or self._lens_scratch.numel() < need:
            self._lens_scratch = torch.empty(need, dtype=torch.uint8, device=self.device)
        cap = self.n * self.n
        cent = np.empty(cap, dtype=np.int32)
        wd = torch.empty((self.n, self.n), dtype=self.trdtype, device=self.device) if w_dif else None
        k = capi.nlse_effective_lens(self.h, capi.make_lens(lens), self._lens_scratch.data_ptr(), need,
                                     cent.ctypes.data, cap, wd.data_ptr() if wd is not None else 0)
        return k, cent[:k].copy(), wd

    def moments(self, pq):
        """Eq. 8 moments M(p, q) = int I^p (x^2 + y^2)^q dx dy for the (p, q) pairs."""
        return np.array(capi.nlse_moments(self.h, list(pq)))

    def history(self):
        cap = 4096
        pw = np.empty(cap)
        pk = np.empty(cap)
        c = capi.nlse_history(self.h, pw.ctypes.data, pk.ctypes.data, cap)
        return pw[:c].copy(), pk[:c].copy()

    def device_status(self) -> int:
        return capi.nlse_device_status(self.h)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            capi.nlse_destroy(self.h)
            self.h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
