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
    ap.add_argument("--large-adjoint-steps", type=int, default=3000)
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


FP32_MARCH_SOURCES = ("dispatch.cuh", "dispatch32.cuh", "fft.cuh", "kernels.cuh", "pair.cuh", "pass32.cuh",
                      "tma.cuh")
FP64_MARCH_SOURCES = ("adjoint.cuh", "dispatch.cuh", "fft.cuh", "kernels.cuh", "nlse_f64.cu", "tma.cuh")


def csrc_digest(files=FP32_MARCH_SOURCES) -> str:
    """Digest of the sources the march kernels are compiled and launched from
    (by default the FP32 march: the FFT engines, the pass kernels, the staged
    column pass and their launch configuration): counters recorded for a
    kernel are valid while this digest is unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2306_15678_gb300", "csrc")
    for fn in files:
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
    """nvidia-smi samples (every 200 ms) of the SM clock, power and throttle
    reasons, each stamped with its arrival time, so that the samples taken
    while a given window of work ran can be picked out afterwards."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        import threading
        self.proc = None
        self.rows = []  # (arrival time, fields)
        self.error = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                text=True)
        except Exception as e:  # no nvidia-smi on this host
            self.error = f"nvidia-smi not started: {e}"
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.perf_counter(), parts))
            elif line.strip():
                self.error = f"unexpected nvidia-smi line: {line.strip()[:120]}"

    def wait_for_samples(self, k: int, timeout: float = 3.0, busy=None):
        """Run busy() (work on the GPU) until k more samples have arrived."""
        target = len(self.rows) + k
        t0 = time.perf_counter()
        while len(self.rows) < target and time.perf_counter() - t0 < timeout and self.proc is not None:
            if busy is not None:
                busy()
            else:
                time.sleep(0.02)

    def stop(self, t_lo: float, t_hi: float) -> dict | None:
        """Summary of the samples that arrived between t_lo and t_hi (perf_counter)."""
        if self.proc is None:
            return {"error": self.error} if self.error else None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.rows:
            err = self.error or (self.proc.stderr.read()[:200] if self.proc.stderr else "")
            return {"error": f"no samples: {err}".strip()}
        rows = [r for t, r in self.rows if t_lo <= t <= t_hi]
        num = lambda v: v.replace(".", "", 1).isdigit()
        sm = [float(r[1]) for r in rows if num(r[1])]
        mx = [float(r[2]) for _, r in self.rows if num(r[2])]
        pw = [float(r[3]) for r in rows if num(r[3])]
        reasons = set()
        for r in rows:
            for nm, v in zip(self.NAMES, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(cfg, U0, seconds: float) -> dict:
    """The FP64 oracle as it stands on this host's cores, on a bounded sample of
    the same workload: whole oracle z steps of the full grid, about 60 % of
    `seconds` on every core and the rest on one core."""
    import oracle

    def timed(budget: float, max_steps: int):
        U = U0
        steps = 0
        t0 = time.perf_counter()
        while True:
            U, _, _ = oracle.march(U, cfg, 1, record=False)
            steps += 1
            if time.perf_counter() - t0 >= budget or steps >= max_steps:
                break
        return steps, time.perf_counter() - t0

    n = cfg["n"]
    cores = oracle.num_threads()
    steps, dt = timed(0.6 * seconds, 50)
    oracle.set_num_threads(1)
    try:
        steps1, dt1 = timed(0.4 * seconds, 20)
    finally:
        oracle.set_num_threads(cores)
    return {"value": n * n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{steps} full z steps of the {n}x{n} workload in FP64 on {cores} threads ({dt:.1f} s)",
            "one_core": {"value": n * n * steps1 / dt1, "unit": UNIT, "cores": 1,
                         "sample": f"{steps1} full z steps on 1 thread ({dt1:.1f} s)"}}


def alu_peak(kind: int, dev, stream) -> float:
    """Peak fused multiply-add rate (FMAs/s, lanes counted) of the GPU for kind
    0 FP32, 1 FP64, 2 packed FP32x2, from the library's probe kernel timed with
    CUDA events on its stream; the launch is scaled to run >= 30 ms."""
    import torch

    from paper_2306_15678_gb300 import capi
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    sink = torch.zeros(blocks, dtype=torch.float64, device=dev)
    lanes = 2 if kind == 2 else 1

    def run(iters: int) -> float:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        capi.nlse_alu_probe(kind, iters, blocks, stream.cuda_stream, sink.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    iters = 256
    for _ in range(24):
        ms = run(iters)
        if ms >= 30.0 or iters >= (1 << 28):
            break
        iters = int(iters * (40.0 / ms if ms > 1.0 else 8.0))
    iters = (iters + 15) // 16 * 16  # the kernel runs whole trips of 16 rounds
    fmas = blocks * 256 * 8 * lanes * iters
    return max(fmas / (run(iters) / 1e3) for _ in range(3))


def fp64_ops_per_point_step() -> dict | None:
    """FP64 arithmetic instructions (per lane) per grid point and z step of the
    FP64 march at 4096^2, from the ncu capture summarised in profiles/ (valid
    while the march sources are unchanged)."""
    path = os.path.join(ROOT, "profiles", "fp64_march_ops.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    return d if d.get("csrc_digest") == csrc_digest(FP64_MARCH_SOURCES) else None


def fp32_fma_record() -> dict | None:
    """FMA-pipe time of the FP32 march kernels at 4096^2 from the ncu capture
    summarised in profiles/ (valid while the march sources are unchanged)."""
    try:
        with open(os.path.join(ROOT, "profiles", "fp32_march_fma.json")) as f:
            d = json.load(f)
    except Exception:
        return None
    return d if d.get("csrc_digest") == csrc_digest() else None


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
    # the same beams marched one after another on single grids (autotuned
    # launch per size; one beam of each size timed, times its count)
    from paper_2306_15678_gb300.grid import Grid
    seq_ms = 0.0
    for n_s, count in mix.items():
        c0 = next(c for c in cfgs if str(c["n"]) == n_s)
        launch = tune.tune_launch(c0, "fp32", steps=10)
        with Grid(c0, precision="fp32", device=dev) as g:
            tune.apply_launch(g, launch)
            g.load(fields[cfgs.index(c0)]).step(5)
            torch.cuda.synchronize(dev)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(g.stream)
            g.step(100)
            a1.record(g.stream)
            torch.cuda.synchronize(dev)
            seq_ms += count * a0.elapsed_time(a1) / 100
    return {"workload": f"{len(cfgs)} beams, grid mix {mix}, full screen, FP32, persistent launch "
                        f"under a CUDA graph ({chunk} steps per replay)",
            "value": pts * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
            "hbm_gbs": gbs, "hbm_frac": gbs / peak_gbs, "tuning": tuning,
            "single_grids_ms_per_step": seq_ms, "single_grids_value": pts / (seq_ms / 1e3),
            "over_single_grids": seq_ms / (ms / steps),
            "status": "ok" if st == 0 else f"status {st}"}


def bench_adjoint(dev) -> dict:
    """The sparse-grid fit end to end: the dense 4096^2 march of the headline
    workload over 10 m (2000 steps of 5 mm), its fluence averaged over 8 x 8
    blocks onto the 512^2 sparse grid of the same window (nlse_fluence with
    downsample 8) as the target, then the gradient of the fluence loss on the
    sparse grid: 400 steps of 2.5 cm, checkpoint every 20, FP32 field, six
    gains.  Times from CUDA events on the march's stream, against the plain
    forward march of the sparse grid."""
    import numpy as np
    import torch

    from paper_2306_15678_gb300 import beams, configs
    from paper_2306_15678_gb300.adjoint import AdjointMarch
    from paper_2306_15678_gb300.grid import Grid
    stream = torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    dense = configs.cfg_dense_fp32()
    cfg = configs.cfg_adjoint_sparse()
    n, M = cfg["n"], cfg["nsteps"]
    ds = dense["n"] // n
    with torch.cuda.stream(stream):
        with Grid(dense, precision="fp32", device=dev, stream=stream) as g:
            g.load(beams.make_field(dense).astype(np.complex64))
            d0, d1, d2 = ev(), ev(), ev()
            d0.record(stream)
            g.step(dense["nsteps"])
            d1.record(stream)
            D = g.fluence(ds, device=True)
            d2.record(stream)
            torch.cuda.synchronize(dev)
            dense_ms, target_ms = d0.elapsed_time(d1), d1.elapsed_time(d2)
            D = D.to(torch.float64)  # (outside the timed interval: torch loads its cast kernel on first use)
        U0 = torch.from_numpy(beams.make_field(cfg).astype(np.complex64)).to(dev)
        with Grid(cfg, precision="fp32", device=dev, stream=stream) as g:
            g.load(U0).step(20)
            g.load(U0)
            torch.cuda.synchronize(dev)
            f0, f1 = ev(), ev()
            f0.record(stream)
            g.step(M)
            f1.record(stream)
            g.power()
            fwd = f0.elapsed_time(f1)
        fit = AdjointMarch(cfg, M, cfg["ckpt"], precision="fp32", device=dev, stream=stream)
        try:
            fit.set_target(D)
            fit.forward(U0)
            fit.backward()
            torch.cuda.synchronize(dev)
            a0, a1, a2 = ev(), ev(), ev()
            a0.record(stream)
            J = fit.forward(U0)
            a1.record(stream)
            dth, dU = fit.backward()
            a2.record(stream)
            torch.cuda.synchronize(dev)
            afwd, abwd = a0.elapsed_time(a1), a1.elapsed_time(a2)
        finally:
            fit.close()
    return {"workload": f"dense {dense['n']}x{dense['n']} march over {dense['nsteps']} steps -> fluence averaged "
                        f"{ds}x{ds} -> target of the {n}x{n} sparse fit, {M} steps, checkpoint every {cfg['ckpt']}, "
                        "FP32, 6 gains",
            "dense_march_ms": dense_ms, "target_downsample_ms": target_ms,
            "forward_march_ms": fwd, "adjoint_forward_ms": afwd, "adjoint_backward_ms": abwd,
            "adjoint_over_forward": (afwd + abwd) / fwd, "loss": J,
            "grad_finite": bool(np.all(np.isfinite(dth))) and bool(torch.isfinite(torch.view_as_real(dU)).all())}


def bench_large_adjoint(dev, nsteps: int) -> dict:
    """One beam of the large batched adjoint: an 8192^2 grid (16 cm window,
    w0 = 3 cm, P = 500 P_cr, full screen), nsteps steps (3000: the whole
    march) with ceil(sqrt(nsteps)) checkpointing, FP32 field, FP64 loss and
    gradients; against the plain forward march of the same steps.  The input
    field is resident on the device for both, and both are timed with CUDA
    events on the march's stream (the adjoint forward ends with the loss
    readout, which synchronises)."""
    import time

    import numpy as np
    import torch

    from paper_2306_15678_gb300 import beams, configs, tune
    from paper_2306_15678_gb300.adjoint import AdjointMarch
    from paper_2306_15678_gb300.grid import Grid
    cfg = configs.cfg_large_adjoint(1)[0]
    n = cfg["n"]
    k = configs.sqrt_checkpoint(nsteps)
    stream = torch.cuda.Stream(device=dev)
    U0 = torch.from_numpy(beams.make_field(cfg).astype(np.complex64)).to(dev)
    D = torch.from_numpy(np.abs(beams.make_field(dict(cfg, beam=dict(cfg["beam"], w0=3.06, seed=5099)))) ** 2).to(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        launch = tune.tune_launch(cfg, "fp32", steps=5)  # the same launch shape for both arms
        with Grid(cfg, precision="fp32", device=dev, stream=stream) as g:
            tune.apply_launch(g, launch)
            g.load(U0).step(3)
            g.load(U0)
            torch.cuda.synchronize(dev)
            f0, f1 = ev(), ev()
            f0.record(stream)
            g.step(nsteps)
            f1.record(stream)
            p_end = g.power()
            fwd_ms = f0.elapsed_time(f1)
        fit = AdjointMarch(cfg, nsteps, k, precision="fp32", device=dev, stream=stream)
        try:
            fit.set_launch(launch)
            fit.set_target(D)
            torch.cuda.synchronize(dev)
            a0, a1, a2 = ev(), ev(), ev()
            t0 = time.perf_counter()
            a0.record(stream)
            J = fit.forward(U0)
            a1.record(stream)
            dth, dU = fit.backward()
            a2.record(stream)
            torch.cuda.synchronize(dev)
            wall = time.perf_counter() - t0
            afwd_ms, abwd_ms = a0.elapsed_time(a1), a1.elapsed_time(a2)
            ws = fit.ws_bytes
            dU_finite = bool(torch.isfinite(torch.view_as_real(dU)).all())
        finally:
            fit.close()
    return {"workload": f"1 of 8 beams {n}x{n}, {nsteps} of 3000 steps, checkpoint every {k} (sqrt), FP32, "
                        "6 gains + input field; input field resident on the device",
            "steps": nsteps, "checkpoint_every": k, "launch": launch,
            "forward_march_ms": fwd_ms, "adjoint_forward_ms": afwd_ms, "adjoint_backward_ms": abwd_ms,
            "adjoint_over_forward": (afwd_ms + abwd_ms) / fwd_ms,
            "backward_over_forward": abwd_ms / fwd_ms,
            "forward_pt_steps_per_s": n * n * nsteps / (fwd_ms / 1e3),
            "gradient_pt_steps_per_s": n * n * nsteps / ((afwd_ms + abwd_ms) / 1e3),
            "adjoint_wall_s": wall, "workspace_gib": ws / 2 ** 30, "final_power_w": p_end,
            "loss": J, "grad_finite": bool(np.all(np.isfinite(dth))) and dU_finite}


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
        "data": "synthetic", "config": dict(workload_desc(cfg), parallelism=f"replicas x{world}"),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "cpu": cpu_model(),
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
        launch = tune.tune_launch(cfg, "fp32", steps=10)
        cols = launch["cols"]
        g = Grid(cfg, precision="fp32", diag_every=1, device=dev, stream=stream)
        tune.apply_launch(g, launch)
        g.load(U0)
        g.step(max(args.warmup, 3))
        torch.cuda.synchronize(dev)
        # kernels launched in the timed region: a column and a row pass per step,
        # plus one finalisation of the recorded power/peak every DIAG_BATCH steps
        launches = 2 * args.steps + (max(args.warmup, 3) % DIAG_BATCH + args.steps) // DIAG_BATCH

        def barrier():
            if dist is not None:
                dist.barrier()

        # ---- clocks: nvidia-smi samples every 200 ms, so a timed region of a few
        # milliseconds falls between two samples; the same march runs on a second
        # grid for >= 3 samples right before and right after the timed region,
        # and the samples of that whole window are reported
        clocks = ClockSampler(local)
        g_clk = Grid(cfg, precision="fp32", diag_every=1, device=dev, stream=stream)
        tune.apply_launch(g_clk, launch)
        g_clk.load(U0)

        def busy():
            g_clk.step(100)
            torch.cuda.synchronize(dev)

        busy()
        clocks.wait_for_samples(1, timeout=5.0, busy=busy)
        t_lo = time.perf_counter()
        clocks.wait_for_samples(3, timeout=3.0, busy=busy)

        # ---- timed region: K z steps, CUDA events on the grid's stream
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
        clocks.wait_for_samples(3, timeout=3.0, busy=busy)
        t_hi = time.perf_counter()
        clk = clocks.stop(t_lo, t_hi)
        if clk is not None:
            clk["window"] = (f"the timed region plus the same march on a second grid for {t_hi - t_lo:.2f} s "
                             "around it (samples every 200 ms)")
        g_clk.close()
        # replicas: sum of every rank's point-steps over the slowest rank's time
        value, ms = shard.aggregate(float(n * n * args.steps), ms, dist, dev)
        if clk is not None and clk.get("sm_mhz"):
            # clock-normalised step: SM cycles per step at the median clock under load
            clk["sm_cycles_per_step"] = ms / args.steps * 1e3 * clk["sm_mhz"]

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
            radix = 8 if cols & capi.NLSE_COL_R8 else 16
            kkey = f"{'k_col_pass32_tma' if cols & capi.NLSE_COL_TMA else 'k_col_pass32'}<{n},{radix},{cols & 0xff}>"
        elif launch["row_radix"] & capi.NLSE_ROW_STAGED:
            kkey = f"k_row_pass32_pf<{n},diag>"
        else:
            kkey = f"k_row_pass32<{n},{launch['row_radix']},diag>"
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                    "frac": achieved / peak_gbs, "traffic": traffic_for(kkey),
                    "kernel": dom, "kernel_ms": dom_ms,
                    "other_kernel_ms": min(col_avg, row_avg),
                    "step_hbm_frac": (2 * bytes_launch) / (ms / args.steps / 1e3) / 1e9 / peak_gbs,
                    "algorithmic_bytes_per_launch": bytes_launch, "peak_source": peak_note}
        # the FP32 side of the same step: FMA-pipe time at full rate (ncu) over the measured step
        fma = fp32_fma_record() if n == 4096 else None
        if fma is not None:
            fma_us = float(fma["fma_us_per_step_at_full_rate"])
            roofline["fp32_alu"] = {
                "bound": "alu", "fma_pipe_us_per_step": fma_us, "step_us": ms / args.steps * 1e3,
                "frac": fma_us / (ms / args.steps * 1e3),
                "issue_active": {k: v["issue_active"] for k, v in fma["kernels"].items()},
                "note": "FMA-pipe busy fraction x duration of one launch of each pass (ncu); the pipe's "
                        "rate is the same for FP32 and packed FP32x2 (fp64_march.fp32*_fma_peak_per_s)"}

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
            tune.apply_launch(gs, launch)
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
            # the FP32 march over the same 3 + k64 steps against this FP64 march (on the GPU)
            with Grid(cfg, precision="fp32", diag_every=1, device=dev, stream=stream) as g32:
                tune.apply_launch(g32, launch)
                g32.load(U0).step(3 + k64)
                f32 = g32.fluence(device=True).to(torch.float64)
                p32 = g32.power()
            f64 = g64.fluence(device=True)
            err32 = {"steps": 3 + k64, "fluence_rel_l2": float(torch.linalg.norm(f32 - f64) / torch.linalg.norm(f64)),
                     "power_rel": abs(p32 / g64.power() - 1),
                     "tolerance": "fluence rel-L2 <= 2e-4 before the first collapse"}
            del f32, f64
            g64.close()
            fma64 = alu_peak(1, dev, stream)
            fma32 = alu_peak(0, dev, stream)
            fma32x2 = alu_peak(2, dev, stream)
            ops = fp64_ops_per_point_step()
            fp64 = {"value": v64, "unit": UNIT, "steps": k64, "fp32_over_fp64": value / world / v64,
                    "hbm_frac": 64.0 * v64 / (peak_gbs * 1e9),
                    "fp64_fma_peak_per_s": fma64, "fp32_fma_peak_per_s": fma32,
                    "fp32x2_fma_peak_per_s": fma32x2,
                    "fp64_over_fp32_fma_rate": fma64 / fma32 if fma32 else None,
                    "fp32_error_vs_fp64": err32}
            if ops and fma64:
                # FP64 pipe: every DFMA, DMUL and DADD takes one issue slot of the FP64
                # pipe, which the probe fills with DFMA alone
                per = float(ops["fp64_inst_per_point_step"])
                fp64["alu"] = {"bound": "alu", "fp64_inst_per_point_step": per,
                               "achieved": per * v64, "peak": fma64, "unit": "FP64 inst/s",
                               "frac": per * v64 / fma64, "source": ops.get("source")}

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
            "config": dict(workload_desc(cfg), parallelism=f"replicas x{world}"),
            "launch": {"column_tile": cols, "row_radix": launch["row_radix"],
                       "source": "autotuner (tune.tune_launch: column tile incl. its radix, then the row radix)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "fp64_march": fp64,
            "strang": strang, "hot_areas": hot, "lens_and_turbulence": lens_t, "batch": batch, "adjoint": adjoint, "large_adjoint": large_adjoint,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
