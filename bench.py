#!/usr/bin/env python3
"""Benchmark of the split-step Fourier NLSE march (arXiv 2306.15678, Eq. 2).

Workload: the dense-grid test problem -- one 4096 x 4096 FP32 field (complex64,
FP64 reductions), 8 cm window, w0 = 1 cm, P = 100 P_cr, 5 % correlated
amplitude noise + 0.1 rad phase noise, Kerr + plasma + multiphoton absorption,
dz = 5 mm.  One bench step = one z step of the whole hot path: column pass
(FFT_y, propagator, inverse FFT_y), row pass (inverse FFT_x, screen, FFT_x) and
the FP64 power/peak readout.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the same workload instead (bounded sample).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point·z-steps/s"
UNIT = "pt·steps/s"
BYTES_PER_PT_PASS = 16  # one read + one write of a complex64 point per pass
DIAG_BATCH = 64  # diagnostic steps the library finalises per launch


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-budget", type=float, default=150.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-strang", action="store_true")
    ap.add_argument("--no-hot", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--large-adjoint-steps", type=int, default=100)
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def workload(n: int):
    from paper_2306_15678_gb300 import configs
    cfg = configs.cfg_dense_fp32()
    if n != cfg["n"]:
        cfg = configs.scaled(cfg, n)
    return cfg


def workload_desc(cfg) -> dict:
    b = cfg["beam"]
    return {
        "workload": f"dense-grid test problem {cfg['n']}x{cfg['n']} complex64 (FP64 reductions), "
                    f"L={cfg['L']} cm, w0={b['w0']} cm, P=100 P_cr, 5% amp + 0.1 rad phase noise, "
                    f"Kerr+plasma+MPA, dz={cfg['dz']} cm",
        "n": cfg["n"], "dz_cm": cfg["dz"], "terms": "kerr+plasma+mpa+diffraction",
        "bench_step": "one z step: column pass + row pass + FP64 power/peak readout",
        "l2": f"inputs larger than L2: field {cfg['n'] ** 2 * 8 / 2 ** 20:.0f} MiB swept twice per step",
    }


def csrc_digest() -> str:
    """Digest of the sources the two march kernels are compiled and launched
    from (the FFT engine, the pass kernels, the staged column pass and their
    launch configuration): the DRAM traffic recorded for a kernel is valid
    while this digest is unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2306_15678_gb300", "csrc")
    for fn in ("dispatch.cuh", "fft.cuh", "kernels.cuh", "tma.cuh"):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_baseline(cfg, U0, seconds: float) -> dict:
    """The FP64 oracle as it stands on this host's cores, on a bounded sample of
    the same workload: whole oracle z steps of the full grid until ~seconds."""
    import oracle
    n = cfg["n"]
    U = U0
    steps = 0
    t0 = time.perf_counter()
    while True:
        U, _, _ = oracle.march(U, cfg, 1, record=False)
        steps += 1
        if time.perf_counter() - t0 >= seconds or steps >= 50:
            break
    dt = time.perf_counter() - t0
    return {"value": n * n * steps / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} full z steps of the {n}x{n} workload in FP64 ({dt:.1f} s)"}


def traffic_for(kernel_key: str) -> float | None:
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    ent = d.get(kernel_key)
    if not ent or ent.get("csrc_digest") != csrc_digest():
        return None
    return float(ent["dram_bytes_per_launch"])


def bench_batch(args, dev, peak_gbs) -> dict:
    """64 beams on grids drawn from {512, 1024, 2048}, P ~ U[20, 200] P_cr,
    w0 ~ U[0.5, 1.5] cm, full screen, one persistent launch per replay of a
    captured CUDA graph, launch shape from the autotuner."""
    import numpy as np
    import torch

    from paper_2306_15678_gb300 import beams, configs, tune
    from paper_2306_15678_gb300.batch import Batch
    cfgs = configs.cfg_batch()
    fields = [beams.make_field(c).astype(np.complex64) for c in cfgs]
    tuning = tune.tune_batch(cfgs, steps=10, fields=fields)
    pts = sum(int(c["n"]) ** 2 for c in cfgs)
    chunk = 50
    with Batch(cfgs, tuning, device=dev) as b:
        for i, U in enumerate(fields):
            b.load(i, U)
        b.capture(chunk)
        b.replay()
        torch.cuda.synchronize(dev)
        reps = max(1, args.batch_steps // chunk)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        for _ in range(reps):
            b.replay()
        e1.record(b.stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        st = b.status()
    steps = reps * chunk
    mix = {}
    for c in cfgs:
        mix[str(c["n"])] = mix.get(str(c["n"]), 0) + 1
    gbs = 2 * BYTES_PER_PT_PASS * pts * steps / (ms / 1e3) / 1e9
    return {"workload": f"{len(cfgs)} beams, grid mix {mix}, full screen, FP32, persistent launch "
                        f"under a CUDA graph ({chunk} steps per replay)",
            "value": pts * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
            "hbm_gbs": gbs, "hbm_frac": gbs / peak_gbs, "tuning": tuning,
            "status": "ok" if st == 0 else f"status {st}"}


def bench_adjoint(dev) -> dict:
    """Gradient of the fluence loss on the 512^2 sparse grid: 400 steps of
    2.5 cm, checkpoint every 20, FP32 field; the target is a box mean of a
    dense-grid fluence shape (a neighbouring beam's fluence stands in)."""
    import time

    import numpy as np
    import torch

    from paper_2306_15678_gb300 import beams, configs
    from paper_2306_15678_gb300.adjoint import AdjointMarch
    from paper_2306_15678_gb300.grid import Grid
    cfg = configs.cfg_adjoint_sparse()
    U0 = beams.make_field(cfg).astype(np.complex64)
    D = np.abs(beams.make_field(dict(cfg, beam=dict(cfg["beam"], w0=1.05, seed=7)))) ** 2
    n, M = cfg["n"], cfg["nsteps"]
    with Grid(cfg, precision="fp32", device=dev) as g:
        g.load(U0).step(20)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g.step(M)
        g.power()
        fwd = time.perf_counter() - t0
    fit = AdjointMarch(cfg, M, cfg["ckpt"], precision="fp32", device=dev)
    try:
        fit.set_target(D)
        fit.forward(U0)
        fit.backward()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        J = fit.forward(U0)
        t1 = time.perf_counter()
        dth, _ = fit.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
    finally:
        fit.close()
    return {"workload": f"{n}x{n} sparse grid, {M} steps, checkpoint every {cfg['ckpt']}, FP32, 6 gains",
            "forward_march_ms": fwd * 1e3, "adjoint_forward_ms": (t1 - t0) * 1e3,
            "adjoint_backward_ms": (t2 - t1) * 1e3,
            "adjoint_over_forward": (t2 - t0) / fwd, "loss": J,
            "grad_finite": bool(np.all(np.isfinite(dth)))}


def bench_large_adjoint(dev, nsteps: int) -> dict:
    """A sample of the large batched adjoint: one of its 8192^2 beams (16 cm
    window, w0 = 3 cm, P = 500 P_cr, full screen), nsteps steps with
    ceil(sqrt(nsteps)) checkpointing, FP32 field, FP64 loss and gradients;
    against the plain forward march of the same steps."""
    import time

    import numpy as np
    import torch

    from paper_2306_15678_gb300 import beams, configs
    from paper_2306_15678_gb300.adjoint import AdjointMarch
    from paper_2306_15678_gb300.grid import Grid
    cfg = configs.cfg_large_adjoint(1)[0]
    n = cfg["n"]
    k = configs.sqrt_checkpoint(nsteps)
    U0 = beams.make_field(cfg).astype(np.complex64)
    D = np.abs(beams.make_field(dict(cfg, beam=dict(cfg["beam"], w0=3.06, seed=5099)))) ** 2
    with Grid(cfg, precision="fp32", device=dev) as g:
        g.load(U0).step(3)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g.step(nsteps)
        g.power()
        fwd = time.perf_counter() - t0
    fit = AdjointMarch(cfg, nsteps, k, precision="fp32", device=dev)
    try:
        fit.set_target(D)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        J = fit.forward(U0)
        t1 = time.perf_counter()
        dth, _ = fit.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        ws = fit.ws_bytes
    finally:
        fit.close()
    return {"workload": f"1 of 8 beams {n}x{n}, {nsteps} of 3000 steps, checkpoint every {k} (sqrt), FP32, "
                        "6 gains + input field",
            "forward_march_ms": fwd * 1e3, "adjoint_forward_ms": (t1 - t0) * 1e3,
            "adjoint_backward_ms": (t2 - t1) * 1e3, "adjoint_over_forward": (t2 - t0) / fwd,
            "gradient_pt_steps_per_s": n * n * nsteps / (t2 - t0), "workspace_gib": ws / 2 ** 30,
            "loss": J, "grad_finite": bool(np.all(np.isfinite(dth)))}


def run_reference(args, world, rank, cfg):
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2306_15678_gb300 import beams
    U0 = beams.make_field(cfg)
    n = cfg["n"]
    U = U0
    # the requested warm-up steps, while they stay within a quarter of the time budget
    t_w0 = time.perf_counter()
    warm = 0
    while warm < max(args.warmup, 1) and (warm == 0 or time.perf_counter() - t_w0 < args.ref_budget / 4):
        U, _, _ = oracle.march(U, cfg, 1, record=False)
        warm += 1
    per = (time.perf_counter() - t_w0) / warm
    budget_steps = max(1, int(args.ref_budget / max(per, 1e-3)))
    k = min(args.steps, budget_steps)
    t0 = time.perf_counter()
    U, _, _ = oracle.march(U, cfg, k, record=False)
    dt = time.perf_counter() - t0
    val = n * n * k / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
        "steps": k, "warmup": warm, "ms_per_step": dt * 1e3 / k,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_desc(cfg),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{k} of {args.steps} requested z steps of the {n}x{n} workload "
                                   f"(time budget {args.ref_budget:.0f} s)"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    del np


def main():
    args = parse()
    world, rank, local, dist = dist_setup(args)
    cfg = workload(args.n)
    if args.impl == "reference":
        run_reference(args, world, rank, cfg)
        if dist is not None:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    from paper_2306_15678_gb300 import beams
    from paper_2306_15678_gb300.grid import Grid

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = cfg["n"]
    U0 = beams.make_field(cfg).astype(np.complex64)
    stream = torch.cuda.Stream(device=dev)
    from paper_2306_15678_gb300 import capi, shard, tune
    with torch.cuda.stream(stream):
        cols = tune.tune_grid(cfg, "fp32", steps=10)
        g = Grid(cfg, precision="fp32", diag_every=1, device=dev, stream=stream)
        capi.nlse_set_column_tile(g.h, cols)
        g.load(U0)
        g.step(max(args.warmup, 3))
        torch.cuda.synchronize(dev)
        # kernels launched in the timed region: a column and a row pass per step,
        # plus one finalisation of the recorded power/peak every DIAG_BATCH steps
        launches = 2 * args.steps + (max(args.warmup, 3) % DIAG_BATCH + args.steps) // DIAG_BATCH

        def barrier():
            if dist is not None:
                dist.barrier()

        # ---- timed region: K z steps, CUDA events on the grid's stream
        clocks = ClockSampler(local)
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop()
        # replicas: sum of every rank's point-steps over the slowest rank's time
        value, ms = shard.aggregate(float(n * n * args.steps), ms, dist, dev)

        # ---- per-kernel times for the roofline (events around every launch)
        kroof = min(args.steps, 500)
        col_ms, row_ms = g.step_timed(kroof)
        g.power()  # readout works after the run (raises on non-finite)
        col_avg, row_avg = col_ms / kroof, row_ms / kroof
        dom = "column pass" if col_avg >= row_avg else "row pass"
        dom_ms = max(col_avg, row_avg)
        bytes_launch = BYTES_PER_PT_PASS * n * n
        peaks = measured_peaks()
        peak_gbs = peaks.get("hbm_gbs")
        peak_note = "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_gbs else "fallback 6800 GB/s"
        peak_gbs = peak_gbs or 6800.0
        achieved = bytes_launch / (dom_ms / 1e3) / 1e9
        if dom == "column pass":
            kkey = f"{'k_col_pass_tma' if cols & capi.NLSE_COL_TMA else 'k_col_pass'}<float,{n},{cols & 0xff}>"
        else:
            kkey = f"k_row_pass<float,{n},diag>"
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                    "frac": achieved / peak_gbs, "traffic": traffic_for(kkey),
                    "kernel": dom, "kernel_ms": dom_ms,
                    "other_kernel_ms": min(col_avg, row_avg),
                    "step_hbm_frac": (2 * bytes_launch) / (ms / args.steps / 1e3) / 1e9 / peak_gbs,
                    "algorithmic_bytes_per_launch": bytes_launch, "peak_source": peak_note}

        # ---- hot areas (closed regions with fluence >= 0.01 TW/cm^2) of the marched field
        hot = None
        if not args.no_hot:
            wp = 1.0e10
            g.hot_areas(wp, 4)
            ts = []
            for _ in range(5):
                h0 = torch.cuda.Event(enable_timing=True)
                h1 = torch.cuda.Event(enable_timing=True)
                h0.record(stream)
                count, _ = g.hot_areas(wp, 4)
                h1.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(h0.elapsed_time(h1))
            # HBM sweeps of the implementation, bytes per point (FP32 grid): readout 12,
            # runs 8, merge 4, roots 4, spread 8
            hot_gbs = 36.0 * n * n / (min(ts) / 1e3) / 1e9
            hot = {"w_p_w_per_cm2": wp, "connectivity": 4, "count": count, "ms": min(ts),
                   "steps_marched": g.steps_taken, "sweep_bytes_per_point": 36, "sweep_gbs": hot_gbs,
                   "hbm_frac": hot_gbs / (measured_peaks().get("hbm_gbs") or 6800.0),
                   "includes": "fluence readout, run labelling, union-find merge, roots, spread; count to host"}

        # ---- effective lens (Eqs. 4-6) and a turbulent layer (Eqs. 9-10) on the marched field
        lens_t = None
        if not args.no_hot:
            lens = dict(l_dif=4e-4, w_l=1e11, conn=4,
                        re=[(0.03, 0.9, 40.0, 0.2), (0.06, -0.5, 30.0, 1.0), (0.1, 0.2, 20.0, -0.4)],
                        im=[(0.04, 0.3, 35.0, 0.1), (0.08, 0.1, 15.0, 0.5)])
            xi = torch.from_numpy(beams.turbulence_draws(n, 77).astype(np.complex64)).to(dev)
            tl, tt = [], []
            for _ in range(3):
                h0 = torch.cuda.Event(enable_timing=True)
                h1 = torch.cuda.Event(enable_timing=True)
                h0.record(stream)
                nlens, _, _ = g.effective_lens(lens)
                h1.record(stream)
                torch.cuda.synchronize(dev)
                tl.append(h0.elapsed_time(h1))
                h0.record(stream)
                g.turbulent_screen(xi, 1e-3, 2 * math.pi / cfg["L"] * 40.0, 50.0)
                h1.record(stream)
                torch.cuda.synchronize(dev)
                tt.append(h0.elapsed_time(h1))
            # HBM sweeps of the implementation, bytes per point (FP32 grid): lens 196
            # (readout 16, fluence 16, DFT pair and filter 80, labelling 28, centres 36,
            # reload 16, plus the screen near the lenses), layer 104 (readout 16,
            # spectrum 16, inverse DFT 32, phase 24, reload 16)
            pk_gbs = measured_peaks().get("hbm_gbs") or 6800.0
            lens_gbs = 196.0 * n * n / (min(tl) / 1e3) / 1e9
            turb_gbs = 104.0 * n * n / (min(tt) / 1e3) / 1e9
            lens_t = {"effective_lens_ms": min(tl), "lenses": nlens, "w_l_w_per_cm2": lens["w_l"],
                      "l_dif_cm2": lens["l_dif"], "turbulent_layer_ms": min(tt),
                      "lens_sweep_gbs": lens_gbs, "lens_hbm_frac": lens_gbs / pk_gbs,
                      "layer_sweep_gbs": turb_gbs, "layer_hbm_frac": turb_gbs / pk_gbs,
                      "includes": "lens: readout, low-pass DFT pair, labelling, centres, ansatz sum, reload; "
                                  "layer: readout, spectrum, inverse DFT pair, phase, reload"}

        # ---- symmetric (Strang) steps on the same field: one more screen per row pass
        strang = None
        if not args.no_strang:
            gs = Grid(dict(cfg, scheme="strang"), precision="fp32", diag_every=1, device=dev, stream=stream)
            capi.nlse_set_column_tile(gs.h, cols)
            gs.load(U0)
            gs.step(3)
            ks = max(50, min(args.steps // 4, 500))
            torch.cuda.synchronize(dev)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            gs.step(ks)
            a1.record(stream)
            torch.cuda.synchronize(dev)
            mss = a0.elapsed_time(a1)
            strang = {"value": n * n * ks / (mss / 1e3), "unit": UNIT, "steps": ks,
                      "ms_per_step": mss / ks, "over_lie_time": (mss / ks) / (ms / args.steps),
                      "note": "global error O(dz^2) instead of O(dz): one call opens and closes its half screens"}
            gs.close()

        # ---- FP64 march on the same field (precision comparison)
        fp64 = None
        if not args.no_fp64:
            g64 = Grid(cfg, precision="fp64", diag_every=1, device=dev, stream=stream)
            g64.load(U0.astype(np.complex128))
            g64.step(3)
            k64 = max(5, min(args.steps // 20, 50))
            torch.cuda.synchronize(dev)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            g64.step(k64)
            a1.record(stream)
            torch.cuda.synchronize(dev)
            ms64 = a0.elapsed_time(a1)
            v64 = n * n * k64 / (ms64 / 1e3)
            fp64 = {"value": v64, "unit": UNIT, "steps": k64, "fp32_over_fp64": value / world / v64}
            g64.close()

        # ---- end to end through the public API with host buffers
        e2e = None
        if not args.no_e2e:
            host_in = torch.from_numpy(U0).pin_memory()
            host_out = torch.empty((n, n), dtype=torch.float32).pin_memory()
            ke = args.steps
            times = []
            for it in range(2):
                barrier()
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                capi.nlse_load_field(g.h, host_in.data_ptr(), False)
                g.step(ke)
                capi.nlse_fluence(g.h, host_out.data_ptr(), False, 1)
                times.append(time.perf_counter() - t0)
            te = min(times)
            e2e = {"value": world * n * n * ke / te, "unit": UNIT,
                   "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 4,
                   "e2e_step": f"load field from pinned host + {ke} z steps + fluence to pinned host"}

        g.close()

    batch = None if args.no_batch else bench_batch(args, dev, peak_gbs)
    adjoint = None if args.no_adjoint else bench_adjoint(dev)
    large_adjoint = None if args.no_adjoint else bench_large_adjoint(dev, args.large_adjoint_steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(cfg, beams.make_field(cfg), args.cpu_seconds)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_desc(cfg), parallelism=f"replicas x{world}", column_tile=cols),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "fp64_march": fp64,
            "strang": strang, "hot_areas": hot, "lens_and_turbulence": lens_t, "batch": batch, "adjoint": adjoint, "large_adjoint": large_adjoint,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
