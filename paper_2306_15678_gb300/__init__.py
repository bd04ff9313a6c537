"""GB300-native split-step Fourier (phase-screen) z-march of the stationary
transverse NLSE (Bulygin & Geints, arXiv 2306.15678, Eqs. 1-3).

The compute path is a C-ABI shared library of hand-written CUDA kernels for
sm_103a (``include/nlse.h``); this package is its thin Python binding.  PyTorch
supplies device memory and streams only.  Nothing here falls back to the CPU:
when the library is missing every call raises.
"""
from . import beams, configs  # noqa: F401  (pure-Python input helpers)

__all__ = ["beams", "configs"]
