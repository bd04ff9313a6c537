"""Autotuner for the launch shapes of the march: the transform radix of the
row pass (16 or 8 elements per thread) and the column tile of the column pass
(its width, per-thread or staged by bulk tensor copies, and its transform
radix) per grid size and precision, and the block size and resident blocks per
SM of the persistent batched launch (per size mix).  Each candidate is timed on
the GPU with CUDA events; the fastest is cached in a JSON file
(NLSE_TUNE_CACHE, default ~/.cache/paper_2306_15678_gb300/tune.json).  For a
given radix the results do not depend on the tile, bit for bit; the radix
changes the rounding within the stated tolerances."""
from __future__ import annotations

import collections
import json
import os

import numpy as np
import torch

from . import beams, capi
from .batch import Batch
from .grid import Grid


def cache_path() -> str:
    return os.environ.get("NLSE_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2306_15678_gb300", "tune.json"))


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _gpu_key() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")


def _time_ms(fn, reps: int) -> float:
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


TILE_CODES = tuple(w | t | r for r in (0, capi.NLSE_COL_R8) for t in (0, capi.NLSE_COL_TMA)
                   for w in (1, 2, 4, 8, 16))
ROW_RADICES = (16, 8, capi.NLSE_ROW_STAGED | 16)
BATCH_RADICES = (16, 8)


def tune_launch(cfg: dict, precision: str = "fp32", steps: int = 20, path: str | None = None,
                force: bool = False) -> dict:
    """Fastest {"cols": column-tile code, "row_radix": 16 or 8} for this grid
    size and precision: the column tiles are timed with the default row radix,
    then the row radices with the chosen tile."""
    path = path or cache_path()
    cache = _load_cache(path)
    key = f"{_gpu_key()}|launch2|{precision}|{int(cfg['n'])}"
    if key in cache and not force:
        return {"cols": int(cache[key]["cols"]), "row_radix": int(cache[key]["row_radix"])}
    U0 = beams.make_field(cfg)
    best, timings, rtimes = None, {}, {}
    with Grid(cfg, precision=precision) as g:
        g.load(U0).step(2)
        for c in TILE_CODES:
            try:
                capi.nlse_set_column_tile(g.h, c)
            except capi.NlseError:
                continue
            g.step(2)
            timings[c] = _time_ms(lambda: g.step(steps), 1) / steps
            if best is None or timings[c] < timings[best]:
                best = c
        capi.nlse_set_column_tile(g.h, best)
        rbest = None
        for r in ROW_RADICES:
            try:
                capi.nlse_set_row_radix(g.h, r)
            except capi.NlseError:
                continue
            g.step(2)
            rtimes[r] = _time_ms(lambda: g.step(steps), 1) / steps
            if rbest is None or rtimes[r] < rtimes[rbest]:
                rbest = r
    cache[key] = {"cols": best, "row_radix": rbest, "ms_per_step": timings, "row_ms_per_step": rtimes}
    _save_cache(path, cache)
    return {"cols": best, "row_radix": rbest}


def apply_launch(g: Grid, launch: dict) -> None:
    """Set a grid's column tile and row radix to a tune_launch result."""
    capi.nlse_set_column_tile(g.h, int(launch["cols"]))
    capi.nlse_set_row_radix(g.h, int(launch["row_radix"]))


def tune_grid(cfg: dict, precision: str = "fp32", steps: int = 20, path: str | None = None,
              force: bool = False) -> int:
    """Fastest column-tile code for this grid size and precision (the column
    part of tune_launch)."""
    return tune_launch(cfg, precision, steps, path, force)["cols"]


def tune_batch(cfgs: list, steps: int = 10, path: str | None = None, force: bool = False,
               fields: list | None = None) -> dict:
    """Fastest (threads, radix, ctas_per_sm) for this mix of grid sizes; the
    column tiles of the beams with n >= 512 are staged (the default)."""
    path = path or cache_path()
    cache = _load_cache(path)
    mix = collections.Counter(int(c["n"]) for c in cfgs)
    key = f"{_gpu_key()}|batch3|" + ",".join(f"{n}x{mix[n]}" for n in sorted(mix))
    if key in cache and not force:
        return dict(cache[key]["tuning"])
    fields = fields or [beams.make_field(c).astype(np.complex64) for c in cfgs]
    best, timings = None, {}
    for radix in BATCH_RADICES:
        for threads in (128, 256, 512):
            for per_sm in (0, 2):
                tuning = {"threads": threads, "radix": radix, "ctas_per_sm": per_sm}
                try:
                    b = Batch(cfgs, tuning)
                except capi.NlseError:
                    continue
                with b:
                    for i, U in enumerate(fields):
                        b.load(i, U)
                    b.step(2)
                    t = _time_ms(lambda: b.step(steps), 1) / steps
                timings[f"{threads}/r{radix}/{per_sm}"] = t
                if best is None or t < best[0]:
                    best = (t, tuning)
    cache[key] = {"tuning": best[1], "ms_per_step": timings}
    _save_cache(path, cache)
    return dict(best[1])
