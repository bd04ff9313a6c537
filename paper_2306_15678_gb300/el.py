"""Effective-lens march (Sec. 2, Eq. 2 and Fig. 1): the sparse-grid march of
Eqs. 1-3 in which every filamentation event is replaced by the effective
screen of the field entering it.

Eq. 2 writes the passage of a filamentation region of length l_f as
exp(-i(h l_f/(2 k0) - f_lens[U_in])) U_in: the lens screen of the entering field
and diffraction over l_f.  The march here takes ordinary split steps while the
peak intensity stays below the pre-filamentation level w_pf; when a step ends
with the peak at or above w_pf (and the previous event has been left behind,
the peak having fallen below w_pf since), it applies the effective lens to the
field (nlse_effective_lens) and then diffraction alone over l_f (a one-step
diffraction-only grid), and marches on.  Every step runs in the library's
kernels; this module only sequences the calls.
"""
from __future__ import annotations

from . import configs
from .grid import Grid


def el_march(cfg: dict, U0, lens: dict, w_pf: float, l_f: float, nsteps: int, precision: str = "fp32",
             device=None) -> dict:
    """March U0 by nsteps split steps of cfg["dz"] with lens events.

    Returns dict(field = final field (numpy), z = distance covered in cm
    (steps and lens lengths), events = [(step, z, lens count)], peaks = peak
    intensity after every step (before any lens event of that step))."""
    with Grid(cfg, precision=precision, device=device) as g, \
            Grid(dict(cfg, terms=configs.DIFFRACTION, dz=float(l_f), scheme="lie", screen="frozen"),
                 precision=precision, device=device) as gd:
        g.load(U0)
        z = 0.0
        armed = True
        events, peaks = [], []
        for s in range(int(nsteps)):
            g.step(1)
            z += cfg["dz"]
            pk = g.peak()
            peaks.append(pk)
            if armed and pk >= w_pf:
                count, _, _ = g.effective_lens(lens)
                gd.load(g.field(device=True)).step(1)
                g.load(gd.field(device=True))
                z += l_f
                events.append((s, z, count))
                armed = False
            elif not armed and pk < w_pf:
                armed = True
        return dict(field=g.field(), z=z, events=events, peaks=peaks)
