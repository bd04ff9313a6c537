"""ctypes binding of the C ABI in include/nlse.h (same names, argument
marshalling only).  Every computation happens in libnlse.so's CUDA kernels;
when the library is missing or fails to load, every call raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnlse.so")

NLSE_OK, NLSE_EINVAL, NLSE_EUNSUPPORTED, NLSE_ENOMEM = 0, 1, 2, 3
NLSE_ECUDA, NLSE_ENONFINITE, NLSE_ETIMEOUT, NLSE_ESTATE = 4, 5, 6, 7
NLSE_COL_TMA = 0x100  # column tile staged with bulk tensor copies (or'ed with the width)
NLSE_COL_R8 = 0x200  # radix-8 column transform (FP32; or'ed with the tile code)
NLSE_ROW_STAGED = 0x100  # persistent row pass staging each row pair by a bulk copy (FP32, | 16)
NLSE_LIE, NLSE_STRANG = 0, 1  # splitting of a step
NLSE_EXACT_SCREEN = 2  # or'ed into the scheme: exact pointwise substep instead of the frozen screen
NLSE_KERR, NLSE_PLASMA, NLSE_MPA, NLSE_DIFFRACTION, NLSE_ALL_TERMS = 1, 2, 4, 8, 15
NLSE_FP64, NLSE_FP32 = 0, 1


class nlse_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("terms", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
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
        ("diag_every", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
    ]


class nlse_batch_tuning(ctypes.Structure):
    _fields_ = [
        ("threads", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("timeout_ms", ctypes.c_int32),
        ("debug_skip_item", ctypes.c_int64),
        ("radix", ctypes.c_int32),
        ("per_thread_columns", ctypes.c_int32),
    ]


LENS_SEGMENTS = 8


class nlse_lens(ctypes.Structure):
    _fields_ = [
        ("l_dif", ctypes.c_double),
        ("w_l", ctypes.c_double),
        ("connectivity", ctypes.c_int32),
        ("n_re", ctypes.c_int32),
        ("n_im", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ] + [(f, ctypes.c_double * LENS_SEGMENTS) for f in ("r_re", "a", "omega", "psi", "r_im", "b", "nu", "eta")]


def make_lens(lens: dict) -> nlse_lens:
    """Pack an effective-lens dict -- l_dif (cm^2), w_l (W/cm^2), conn (4/8),
    re = [(r_j, a_j, omega_j, psi_j), ...], im = [(r_l, b_l, nu_l, eta_l), ...]
    -- into the ABI's record."""
    q = nlse_lens()
    q.l_dif = float(lens["l_dif"])
    q.w_l = float(lens["w_l"])
    q.connectivity = int(lens.get("conn", 4))
    for part, names, cnt in (("re", ("r_re", "a", "omega", "psi"), "n_re"),
                             ("im", ("r_im", "b", "nu", "eta"), "n_im")):
        segs = lens.get(part, ())
        if len(segs) > LENS_SEGMENTS:
            raise ValueError(f"at most {LENS_SEGMENTS} segments per part")
        setattr(q, cnt, len(segs))
        for j, seg in enumerate(segs):
            for f, v in zip(names, seg):
                getattr(q, f)[j] = float(v)
    return q


class NlseError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {nlse_status_string(status)}")


_lock = threading.Lock()
_lib = None

_SIGS = {
    # name: (restype, argtypes)
    "nlse_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "nlse_version": (ctypes.c_int32, []),
    "nlse_workspace_size": (ctypes.c_int, [ctypes.POINTER(nlse_params), ctypes.POINTER(ctypes.c_size_t)]),
    "nlse_create": (ctypes.c_int, [ctypes.POINTER(nlse_params), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "nlse_load_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "nlse_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "nlse_step_timed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "nlse_alu_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "nlse_steps_taken": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "nlse_power": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "nlse_peak": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "nlse_fluence": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "nlse_read_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "nlse_hot_areas": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "nlse_turbulent_screen": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double]),
    "nlse_lens_scratch_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "nlse_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "nlse_effective_lens": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p]),
    "nlse_history": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)]),
    "nlse_device_status": (ctypes.c_int, [ctypes.c_void_p]),
    "nlse_power_peak_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "nlse_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "nlse_batch_workspace_size": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "nlse_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "nlse_batch_load_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    "nlse_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "nlse_batch_capture": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "nlse_batch_replay": (ctypes.c_int, [ctypes.c_void_p]),
    "nlse_batch_status": (ctypes.c_int, [ctypes.c_void_p]),
    "nlse_batch_steps_taken": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "nlse_batch_read_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    "nlse_batch_power": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "nlse_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "nlse_set_column_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "nlse_set_row_radix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "nlse_adjoint_workspace_size": (ctypes.c_int, [ctypes.POINTER(nlse_params), ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.POINTER(ctypes.c_size_t)]),
    "nlse_adjoint_create": (ctypes.c_int, [ctypes.POINTER(nlse_params), ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "nlse_adjoint_set_theta": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "nlse_adjoint_set_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "nlse_adjoint_set_target": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "nlse_adjoint_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double)]),
    "nlse_adjoint_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "nlse_adjoint_destroy": (ctypes.c_int, [ctypes.c_void_p]),
}


def lib() -> ctypes.CDLL:
    """The loaded libnlse.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libnlse.so not found at {LIB_PATH}: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def check(status: int, where: str) -> None:
    if status != NLSE_OK:
        raise NlseError(status, where)


def nlse_status_string(status: int) -> str:
    return lib().nlse_status_string(int(status)).decode()


def nlse_version() -> int:
    return int(lib().nlse_version())


def nlse_workspace_size(p: nlse_params) -> int:
    b = ctypes.c_size_t(0)
    check(lib().nlse_workspace_size(ctypes.byref(p), ctypes.byref(b)), "nlse_workspace_size")
    return int(b.value)


def nlse_create(p: nlse_params, stream: int, workspace: int, nbytes: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    check(lib().nlse_create(ctypes.byref(p), ctypes.c_void_p(stream), ctypes.c_void_p(workspace),
                            ctypes.c_size_t(nbytes), ctypes.byref(h)), "nlse_create")
    return h


def nlse_load_field(h, src: int, on_device: bool) -> None:
    check(lib().nlse_load_field(h, ctypes.c_void_p(src), int(bool(on_device))), "nlse_load_field")


def nlse_step(h, nsteps: int) -> None:
    check(lib().nlse_step(h, int(nsteps)), "nlse_step")


def nlse_step_timed(h, nsteps: int) -> tuple[float, float]:
    """Step and return the summed (column-pass, row-pass) durations in ms."""
    c = ctypes.c_double(0.0)
    r = ctypes.c_double(0.0)
    check(lib().nlse_step_timed(h, int(nsteps), ctypes.byref(c), ctypes.byref(r)), "nlse_step_timed")
    return float(c.value), float(r.value)


def nlse_alu_probe(kind: int, iters: int, blocks: int, stream: int, sink_dev: int) -> None:
    """Enqueue the FMA-rate probe (kind 0 FP32, 1 FP64, 2 packed FP32x2):
    blocks x 256 threads x 8 chains x iters fused multiply-adds (x 2 lanes for
    kind 2)."""
    check(lib().nlse_alu_probe(int(kind), int(iters), int(blocks), ctypes.c_void_p(stream),
                               ctypes.c_void_p(sink_dev)), "nlse_alu_probe")


def nlse_steps_taken(h) -> int:
    v = ctypes.c_int64(0)
    check(lib().nlse_steps_taken(h, ctypes.byref(v)), "nlse_steps_taken")
    return int(v.value)


def nlse_power(h) -> float:
    v = ctypes.c_double(0)
    check(lib().nlse_power(h, ctypes.byref(v)), "nlse_power")
    return float(v.value)


def nlse_peak(h) -> float:
    v = ctypes.c_double(0)
    check(lib().nlse_peak(h, ctypes.byref(v)), "nlse_peak")
    return float(v.value)


def nlse_fluence(h, dst: int, on_device: bool, downsample: int) -> None:
    check(lib().nlse_fluence(h, ctypes.c_void_p(dst), int(bool(on_device)), int(downsample)),
          "nlse_fluence")


def nlse_read_field(h, dst: int, on_device: bool) -> None:
    check(lib().nlse_read_field(h, ctypes.c_void_p(dst), int(bool(on_device))), "nlse_read_field")


def nlse_hot_areas(h, w_p: float, connectivity: int, labels_ptr: int, on_device: bool) -> int:
    c = ctypes.c_int32(0)
    check(lib().nlse_hot_areas(h, float(w_p), int(connectivity), ctypes.byref(c),
                               ctypes.c_void_p(labels_ptr or None), int(bool(on_device))), "nlse_hot_areas")
    return int(c.value)


def nlse_turbulent_screen(h, xi_ptr: int, on_device: bool, tau: float, k_h: float, thickness: float) -> None:
    check(lib().nlse_turbulent_screen(h, ctypes.c_void_p(xi_ptr), int(bool(on_device)), float(tau), float(k_h),
                                      float(thickness)), "nlse_turbulent_screen")


def nlse_moments(h, pq) -> list:
    """Eq. 8 moments M(p, q) for the (p, q) pairs in pq."""
    k = len(pq)
    P = (ctypes.c_int32 * max(k, 1))(*[int(a) for a, _ in pq])
    Q = (ctypes.c_int32 * max(k, 1))(*[int(b) for _, b in pq])
    out = (ctypes.c_double * max(k, 1))()
    check(lib().nlse_moments(h, k, P, Q, out), "nlse_moments")
    return [float(out[i]) for i in range(k)]


def nlse_lens_scratch_size(p: nlse_params) -> int:
    b = ctypes.c_size_t(0)
    check(lib().nlse_lens_scratch_size(ctypes.byref(p), ctypes.byref(b)), "nlse_lens_scratch_size")
    return int(b.value)


def nlse_effective_lens(h, lens: nlse_lens, scratch: int, scratch_bytes: int, centres_ptr: int, capacity: int,
                        w_dif_ptr: int) -> int:
    c = ctypes.c_int32(0)
    check(lib().nlse_effective_lens(h, ctypes.byref(lens), ctypes.c_void_p(scratch), int(scratch_bytes),
                                    ctypes.byref(c), ctypes.c_void_p(centres_ptr or None), int(capacity),
                                    ctypes.c_void_p(w_dif_ptr or None)), "nlse_effective_lens")
    return int(c.value)


def nlse_history(h, power_ptr: int, peak_ptr: int, capacity: int) -> int:
    c = ctypes.c_int32(0)
    check(lib().nlse_history(h, ctypes.c_void_p(power_ptr), ctypes.c_void_p(peak_ptr),
                             int(capacity), ctypes.byref(c)), "nlse_history")
    return int(c.value)


def nlse_device_status(h) -> int:
    return int(lib().nlse_device_status(h))


def nlse_power_peak_noalloc(field_dev: int, n: int, precision: int, L: float, stream: int,
                            out_dev: int) -> None:
    """Enqueue (power, peak) of a device field into out_dev (2 doubles); the
    library allocates nothing for it (its scratch is a static device array)."""
    check(lib().nlse_power_peak_noalloc(ctypes.c_void_p(field_dev), int(n), int(precision),
                                        float(L), ctypes.c_void_p(stream), ctypes.c_void_p(out_dev)),
          "nlse_power_peak_noalloc")


def nlse_destroy(h) -> None:
    check(lib().nlse_destroy(h), "nlse_destroy")


def nlse_adjoint_workspace_size(p: nlse_params, nsteps: int, ckpt: int) -> int:
    b = ctypes.c_size_t(0)
    check(lib().nlse_adjoint_workspace_size(ctypes.byref(p), int(nsteps), int(ckpt), ctypes.byref(b)),
          "nlse_adjoint_workspace_size")
    return int(b.value)


def nlse_adjoint_create(p: nlse_params, nsteps: int, ckpt: int, stream: int, workspace: int,
                        nbytes: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    check(lib().nlse_adjoint_create(ctypes.byref(p), int(nsteps), int(ckpt), ctypes.c_void_p(stream),
                                    ctypes.c_void_p(workspace), ctypes.c_size_t(nbytes), ctypes.byref(h)),
          "nlse_adjoint_create")
    return h


def nlse_adjoint_set_launch(h, cols: int, row_radix: int) -> None:
    check(lib().nlse_adjoint_set_launch(h, int(cols), int(row_radix)), "nlse_adjoint_set_launch")


def nlse_adjoint_set_theta(h, theta_ptr: int) -> None:
    check(lib().nlse_adjoint_set_theta(h, ctypes.c_void_p(theta_ptr)), "nlse_adjoint_set_theta")


def nlse_adjoint_set_target(h, target: int, on_device: bool) -> None:
    check(lib().nlse_adjoint_set_target(h, ctypes.c_void_p(target), int(bool(on_device))),
          "nlse_adjoint_set_target")


def nlse_adjoint_forward(h, src: int, on_device: bool) -> float:
    v = ctypes.c_double(0)
    check(lib().nlse_adjoint_forward(h, ctypes.c_void_p(src), int(bool(on_device)), ctypes.byref(v)),
          "nlse_adjoint_forward")
    return float(v.value)


def nlse_adjoint_backward(h, dtheta_ptr: int, dU0: int, on_device: bool) -> None:
    check(lib().nlse_adjoint_backward(h, ctypes.c_void_p(dtheta_ptr), ctypes.c_void_p(dU0),
                                      int(bool(on_device))), "nlse_adjoint_backward")


def nlse_adjoint_destroy(h) -> None:
    check(lib().nlse_adjoint_destroy(h), "nlse_adjoint_destroy")


def nlse_set_column_tile(h, cols: int) -> None:
    check(lib().nlse_set_column_tile(h, int(cols)), "nlse_set_column_tile")


def nlse_set_row_radix(h, radix: int) -> None:
    check(lib().nlse_set_row_radix(h, int(radix)), "nlse_set_row_radix")


def _params_array(params):
    arr = (nlse_params * len(params))()
    for i, p in enumerate(params):
        arr[i] = p
    return arr


def nlse_batch_workspace_size(params) -> int:
    arr = _params_array(params)
    b = ctypes.c_size_t(0)
    check(lib().nlse_batch_workspace_size(len(params), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(b)),
          "nlse_batch_workspace_size")
    return int(b.value)


def nlse_batch_create(params, tuning, stream: int, workspace: int, nbytes: int) -> ctypes.c_void_p:
    arr = _params_array(params)
    h = ctypes.c_void_p()
    tp = ctypes.byref(tuning) if tuning is not None else None
    check(lib().nlse_batch_create(len(params), ctypes.cast(arr, ctypes.c_void_p),
                                  ctypes.cast(tp, ctypes.c_void_p) if tp is not None else None,
                                  ctypes.c_void_p(stream), ctypes.c_void_p(workspace), ctypes.c_size_t(nbytes),
                                  ctypes.byref(h)), "nlse_batch_create")
    return h


def nlse_batch_load_field(h, beam: int, src: int, on_device: bool) -> None:
    check(lib().nlse_batch_load_field(h, int(beam), ctypes.c_void_p(src), int(bool(on_device))),
          "nlse_batch_load_field")


def nlse_batch_step(h, nsteps: int) -> None:
    check(lib().nlse_batch_step(h, int(nsteps)), "nlse_batch_step")


def nlse_batch_capture(h, nsteps: int) -> None:
    check(lib().nlse_batch_capture(h, int(nsteps)), "nlse_batch_capture")


def nlse_batch_replay(h) -> None:
    check(lib().nlse_batch_replay(h), "nlse_batch_replay")


def nlse_batch_status(h) -> int:
    return int(lib().nlse_batch_status(h))


def nlse_batch_steps_taken(h) -> int:
    v = ctypes.c_int64(0)
    check(lib().nlse_batch_steps_taken(h, ctypes.byref(v)), "nlse_batch_steps_taken")
    return int(v.value)


def nlse_batch_read_field(h, beam: int, dst: int, on_device: bool) -> None:
    check(lib().nlse_batch_read_field(h, int(beam), ctypes.c_void_p(dst), int(bool(on_device))),
          "nlse_batch_read_field")


def nlse_batch_power(h, beam: int) -> float:
    v = ctypes.c_double(0)
    check(lib().nlse_batch_power(h, int(beam), ctypes.byref(v)), "nlse_batch_power")
    return float(v.value)


def nlse_batch_destroy(h) -> None:
    check(lib().nlse_batch_destroy(h), "nlse_batch_destroy")
