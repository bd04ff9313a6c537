"""FP64 CPU oracle for the split-step NLSE z-march (arXiv 2306.15678, Eqs. 1-3, 7).

TEST INFRASTRUCTURE ONLY: the parity oracle for the CUDA path.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The product package never does.

The arithmetic lives in ``nlse_oracle.c`` (plain C, double precision, its own
radix-2 FFT); this module only builds it with gcc and marshals numpy arrays.
Every function here follows the passage named in the C source:

* ``fft2`` / ``fft1`` -- the discrete Fourier transform used by the phase-screen
  step (Eq. 2), forward unnormalised, inverse 1/N per dimension.
* ``propagator`` / ``linear`` -- diffraction, Lap_perp -> -k^2 (Eq. 1-2).
* ``screen`` -- the pointwise Kerr / plasma / absorption screen (Eq. 2-3).
* ``march`` -- Lie steps, diffraction then screen (Eq. 2), or symmetric
  Strang steps (half screen, diffraction, half screen).
* ``power``, ``peak``, ``fluence``, ``loss`` -- readouts (w = UU*, Sec. 2-3).
* ``hot_areas`` -- number of closed regions with w >= w_p (Sec. 3.3).
* ``adjoint`` -- reverse-mode gradient of the fluence loss (derived from the
  same steps; the paper has no adjoint).

Pinned by tests/test_oracle_pins.py (brute-force DFT, numpy.fft, closed-form
Gaussian beam, exact screen identities, conservation, time reversal, symmetry,
finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nlse_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KERR, PLASMA, MPA, DIFFRACTION = 1, 2, 4, 8
ALL_TERMS = KERR | PLASMA | MPA | DIFFRACTION


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("terms", ctypes.c_uint32),
        ("reserved", ctypes.c_int32),
        ("L", ctypes.c_double),
        ("dz", ctypes.c_double),
        ("lambda0", ctypes.c_double),
        ("n0", ctypes.c_double),
        ("n2", ctypes.c_double),
        ("sigmaK", ctypes.c_double),
        ("rho_nt", ctypes.c_double),
        ("rho_c", ctypes.c_double),
        ("tau_pl", ctypes.c_double),
        ("betaK", ctypes.c_double),
        ("theta", ctypes.c_double * 6),
    ]


LENS_SEG = 8


class OrcLens(ctypes.Structure):
    _fields_ = [
        ("l_dif", ctypes.c_double),
        ("w_l", ctypes.c_double),
        ("conn", ctypes.c_int32),
        ("n_re", ctypes.c_int32),
        ("n_im", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ] + [(f, ctypes.c_double * LENS_SEG) for f in ("r_re", "a", "omega", "psi", "r_im", "b", "nu", "eta")]


def lens_record(lens: dict) -> OrcLens:
    """Pack an effective-lens dict -- l_dif (cm^2), w_l (W/cm^2), conn (4/8),
    re = [(r_j, a_j, omega_j, psi_j), ...], im = [(r_l, b_l, nu_l, eta_l), ...]
    (joints in cm, increasing) -- into the oracle's record."""
    q = OrcLens()
    q.l_dif = float(lens["l_dif"])
    q.w_l = float(lens["w_l"])
    q.conn = int(lens.get("conn", 4))
    for part, names, cnt in (("re", ("r_re", "a", "omega", "psi"), "n_re"),
                             ("im", ("r_im", "b", "nu", "eta"), "n_im")):
        segs = lens.get(part, ())
        assert len(segs) <= LENS_SEG
        setattr(q, cnt, len(segs))
        for j, seg in enumerate(segs):
            for f, v in zip(names, seg):
                getattr(q, f)[j] = float(v)
    return q


def build(force: bool = False) -> str:
    """Compile nlse_oracle.c into _build/liboracle.so with gcc (FP64, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    cp = ctypes.c_void_p
    P = ctypes.POINTER(OrcParams)
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    lib.orc_fft1d.argtypes = [cp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_fft2d.argtypes = [cp, ctypes.c_int, ctypes.c_int]
    lib.orc_propagator.argtypes = [P, cp]
    lib.orc_linear.argtypes = [P, cp]
    lib.orc_screen.argtypes = [P, cp]
    lib.orc_power.argtypes = [cp, ctypes.c_int, ctypes.c_double]
    lib.orc_power.restype = ctypes.c_double
    lib.orc_peak.argtypes = [cp, ctypes.c_int]
    lib.orc_moment.argtypes = [cp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.orc_moment.restype = ctypes.c_double
    lib.orc_peak.restype = ctypes.c_double
    lib.orc_fluence.argtypes = [cp, ctypes.c_int, ctypes.c_int, cp]
    lib.orc_loss.argtypes = [cp, cp, ctypes.c_int]
    lib.orc_loss.restype = ctypes.c_double
    lib.orc_march.argtypes = [P, cp, ctypes.c_int, cp, cp]
    lib.orc_march_strang.argtypes = [P, cp, ctypes.c_int, cp, cp]
    lib.orc_hot_areas.argtypes = [cp, ctypes.c_int, ctypes.c_double, ctypes.c_int, cp]
    lib.orc_turbulent_eps.argtypes = [P, cp, ctypes.c_double, ctypes.c_double, cp]
    LP = ctypes.POINTER(OrcLens)
    lib.orc_lens_lowpass.argtypes = [ctypes.c_int, ctypes.c_double, cp, ctypes.c_double, cp]
    lib.orc_lens_centres.argtypes = [cp, ctypes.c_int, ctypes.c_double, ctypes.c_int, cp]
    lib.orc_lens_value.argtypes = [LP, ctypes.c_double, cp, cp]
    lib.orc_lens_apply.argtypes = [ctypes.c_int, ctypes.c_double, cp, cp, ctypes.c_int, LP]
    lib.orc_effective_lens.argtypes = [P, cp, LP, cp]
    lib.orc_turbulent_screen.argtypes = [P, cp, cp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.orc_hot_areas.restype = ctypes.c_int
    lib.orc_adjoint.argtypes = [P, cp, cp, ctypes.c_int, ctypes.c_int, cp, cp]
    lib.orc_adjoint.restype = ctypes.c_double
    return lib


def compile_variant(src_text: str, out_path: str) -> ctypes.CDLL:
    """Compile a modified copy of the oracle source (used by the tests that
    plant a mistake in the oracle to show that a pin catches it)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                    "-o", out_path, src, "-lm"], check=True)
    return _configure(ctypes.CDLL(out_path))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
        return _lib


def params(cfg: dict) -> OrcParams:
    """Pack a physical parameter dict (see paper_2306_15678_gb300.configs) into
    the oracle's record."""
    p = OrcParams()
    p.n = int(cfg["n"])
    p.K = int(cfg["K"])
    p.terms = int(cfg["terms"])
    for f in ("L", "dz", "lambda0", "n0", "n2", "sigmaK", "rho_nt", "rho_c", "tau_pl", "betaK"):
        setattr(p, f, float(cfg[f]))
    th = cfg.get("theta", (1.0, 0.0, 1.0, 0.0, 1.0, 0.0))
    for i in range(6):
        p.theta[i] = float(th[i])
    screen = cfg.get("screen", "frozen")
    if screen not in ("frozen", "exact"):
        raise ValueError(f"screen {screen!r}")
    p.reserved = 1 if screen == "exact" else 0
    return p


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(k: int) -> None:
    """Threads the oracle's parallel loops use from now on in this thread."""
    _load().orc_set_num_threads(int(k))


def fft1(a, inverse: bool = False) -> np.ndarray:
    out = _c128(a).copy()
    _load().orc_fft1d(out.ctypes.data, out.shape[0], 1, int(inverse))
    return out


def fft2(a, inverse: bool = False) -> np.ndarray:
    out = _c128(a).copy()
    assert out.ndim == 2 and out.shape[0] == out.shape[1]
    _load().orc_fft2d(out.ctypes.data, out.shape[0], int(inverse))
    return out


def propagator(cfg: dict) -> np.ndarray:
    p = params(cfg)
    out = np.empty((p.n, p.n), dtype=np.complex128)
    _load().orc_propagator(ctypes.byref(p), out.ctypes.data)
    return out


def linear(U, cfg: dict) -> np.ndarray:
    out = _c128(U).copy()
    _load().orc_linear(ctypes.byref(params(cfg)), out.ctypes.data)
    return out


def screen(U, cfg: dict) -> np.ndarray:
    out = _c128(U).copy()
    _load().orc_screen(ctypes.byref(params(cfg)), out.ctypes.data)
    return out


def power(U, L: float) -> float:
    U = _c128(U)
    return float(_load().orc_power(U.ctypes.data, U.shape[0], float(L)))


def peak(U) -> float:
    U = _c128(U)
    return float(_load().orc_peak(U.ctypes.data, U.shape[0]))


def moment(U, L: float, p: int, q: int) -> float:
    """Eq. 8 moment M(p, q) = int I^p (x^2 + y^2)^q dx dy (cell-centred grid)."""
    U = _c128(U)
    return float(_load().orc_moment(U.ctypes.data, U.shape[0], float(L), int(p), int(q)))


def fluence(U, ds: int = 1) -> np.ndarray:
    U = _c128(U)
    n = U.shape[0]
    out = np.empty((n // ds, n // ds), dtype=np.float64)
    _load().orc_fluence(U.ctypes.data, n, int(ds), out.ctypes.data)
    return out


def loss(U, D) -> float:
    U = _c128(U)
    D = np.ascontiguousarray(D, dtype=np.float64)
    return float(_load().orc_loss(U.ctypes.data, D.ctypes.data, U.shape[0]))


def march(U0, cfg: dict, nsteps: int, record: bool = True, scheme: str | None = None):
    """March U0 by nsteps Lie steps (diffraction, then screen), or Strang steps
    (half screen, diffraction, half screen) when scheme -- or cfg["scheme"] --
    is "strang".  Returns (U, power[nsteps+1], peak[nsteps+1])."""
    U = _c128(U0).copy()
    p = params(cfg)
    pw = np.zeros(nsteps + 1) if record else None
    pk = np.zeros(nsteps + 1) if record else None
    scheme = scheme or cfg.get("scheme", "lie")
    if scheme not in ("lie", "strang"):
        raise ValueError(f"scheme {scheme!r}")
    fn = _load().orc_march_strang if scheme == "strang" else _load().orc_march
    fn(ctypes.byref(p), U.ctypes.data, int(nsteps),
       pw.ctypes.data if record else None,
       pk.ctypes.data if record else None)
    return U, pw, pk


def hot_areas(w, wp: float, conn: int = 4):
    """Number of connected regions where w >= wp (Sec. 3.3 "hot areas"), and the
    labels: -1 outside, else the smallest row-major index of the region."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = w.shape[0]
    labels = np.empty((n, n), dtype=np.int32)
    count = _load().orc_hot_areas(w.ctypes.data, n, float(wp), int(conn), labels.ctypes.data)
    if count < 0:
        raise ValueError("hot_areas: bad argument")
    return int(count), labels


def turbulent_eps(xi, cfg: dict, tau: float, kh: float) -> np.ndarray:
    """Turbulent screen eps_t(y, x) of Eqs. 9-10 from the random draws xi
    (n x n complex, FFT bin order): step spectrum tau for |k| <= kh."""
    xi = _c128(xi)
    out = np.empty(xi.shape, dtype=np.float64)
    _load().orc_turbulent_eps(ctypes.byref(params(cfg)), xi.ctypes.data, float(tau), float(kh), out.ctypes.data)
    return out


def turbulent_screen(U, xi, cfg: dict, tau: float, kh: float, thickness: float) -> np.ndarray:
    """U exp(-i thickness eps_t / (2 k0)): the turbulent layer of Eq. 9."""
    out = _c128(U).copy()
    xi = _c128(xi)
    _load().orc_turbulent_screen(ctypes.byref(params(cfg)), out.ctypes.data, xi.ctypes.data, float(tau),
                                 float(kh), float(thickness))
    return out


def lens_lowpass(w, L: float, l_dif: float) -> np.ndarray:
    """Eq. 4: F^-1 exp(-l_dif k^2) F w (real part), k in rad/cm on the window L."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty_like(w)
    _load().orc_lens_lowpass(w.shape[0], float(L), w.ctypes.data, float(l_dif), out.ctypes.data)
    return out


def lens_centres(w_dif, w_l: float, conn: int = 4) -> np.ndarray:
    """Row-major indices (increasing) of the lens centres: the maximum of each
    region with w_dif >= w_l (first in row-major order on a tie)."""
    wd = np.ascontiguousarray(w_dif, dtype=np.float64)
    out = np.empty(wd.size, dtype=np.int32)
    k = _load().orc_lens_centres(wd.ctypes.data, wd.shape[0], float(w_l), int(conn), out.ctypes.data)
    if k < 0:
        raise ValueError("lens_centres: bad argument")
    return out[:k].copy()


def lens_value(lens: dict, r: float):
    """Eq. 6 at distance r: (Re f_lens, Im f_lens)."""
    re, im = ctypes.c_double(0), ctypes.c_double(0)
    q = lens_record(lens)
    _load().orc_lens_value(ctypes.byref(q), float(r), ctypes.byref(re), ctypes.byref(im))
    return re.value, im.value


def lens_apply(U, L: float, centres, lens: dict) -> np.ndarray:
    """U exp(i D_f), D_f = sum over centres of f_lens(|r - r_c|) (Eqs. 2, 5)."""
    out = _c128(U).copy()
    c = np.ascontiguousarray(centres, dtype=np.int32)
    q = lens_record(lens)
    _load().orc_lens_apply(out.shape[0], float(L), out.ctypes.data, c.ctypes.data, len(c), ctypes.byref(q))
    return out


def effective_lens(U, cfg: dict, lens: dict):
    """The whole effective-lens screen: (U exp(i D_f[U]), centres)."""
    out = _c128(U).copy()
    cent = np.empty(out.size, dtype=np.int32)
    q = lens_record(lens)
    k = _load().orc_effective_lens(ctypes.byref(params(cfg)), out.ctypes.data, ctypes.byref(q), cent.ctypes.data)
    if k < 0:
        raise ValueError("effective_lens: bad argument")
    return out, cent[:k].copy()


def adjoint(U0, D, cfg: dict, nsteps: int, ckpt: int = 20):
    """Loss J and its gradients (dJ/dtheta[6], dJ/dU0 as dRe + i dIm)."""
    U0 = _c128(U0)
    D = np.ascontiguousarray(D, dtype=np.float64)
    dth = np.zeros(6)
    dU0 = np.empty_like(U0)
    J = _load().orc_adjoint(ctypes.byref(params(cfg)), U0.ctypes.data, D.ctypes.data,
                            int(nsteps), int(ckpt), dth.ctypes.data, dU0.ctypes.data)
    return float(J), dth, dU0
