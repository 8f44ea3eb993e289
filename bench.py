"""Benchmark of the lattice Boltzmann time step on GB300.

Headline workload (config 4, the largest single-GPU configuration): the ST
step on an 8192 x 8192 periodic D2Q9 grid (Taylor-Green mode 1 plus a mode-2
shear wave), FP32 storage and arithmetic.  One bench step = one ST time step
(one kernel launch), timed alone with CUDA events on the launching stream;
the state (two 2.4 GB buffers) is far larger than the 129 MB L2, so no flush is needed.
The line carries the HBM roofline of that kernel, the FP64 oracle timed on
this host's cores over a fixed 10-step window (and its error against the
GPU after the same window), and the end-to-end figure through the C ABI
(host fields in, the config's 500 steps, u_x out).

Extra lines in the same JSON object: the serving stream; ST 8192^2 with BF16
and FP16 deviation storage; FV 4096^2; FV RB 1024^2 FP32; the 3-D Table rb
grids; and, as full lines with their own roofline, oracle baseline, oracle
error and end-to-end figure, config 2 (the FV channel 256 x 512) and config
3 (FV thermal RB 1024^2 at Ra = 1e8 with FP16 deviation storage).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--case NAME]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline (FV and ST) vs FP64 oracle error; serving p50/p99 latency"
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 10):
        self.gpu, self.period = gpu_index, period_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts only once sampling has begun
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- GPU --

FV_SCHEDULE = "tune"
FV3_SCHEDULE = "auto"


def make_grid(lb, w, stream, tune=True):
    """Grid of a workload; FV grids run the library's autotuner (it restores
    the state it times on), so the timed steps use the schedule it picked,
    unless --fv-schedule fixes one."""
    grid = dict(w.grid)
    store = grid.pop("store")
    if "nz" in grid:  # D3Q19 grid (include/lb3.h): plain or staged flux passes
        g3 = lb.Grid3(store=store, stream=stream, **grid).init(**w.params, **w.init)
        if w.scheme == "fv" and FV3_SCHEDULE != "auto":
            g3.set_fv_schedule(lb.LB3_FV_PLAIN if FV3_SCHEDULE == "plain" else lb.LB3_FV_STAGED)
        return g3
    g = lb.Grid(store=store, stream=stream, **grid)
    g.init(**w.params, **w.init)
    if w.scheme == "fv":
        if FV_SCHEDULE.startswith("split"):
            g.set_fv_schedule(lb.LB_FV_SPLIT, int(FV_SCHEDULE.split(":")[1]) if ":" in FV_SCHEDULE else 0)
        elif FV_SCHEDULE.startswith("ptile"):
            g.set_fv_schedule(lb.LB_FV_PTILE, int(FV_SCHEDULE.split(":")[1]) if ":" in FV_SCHEDULE else 0)
        elif FV_SCHEDULE.startswith("tile"):
            g.set_fv_schedule(lb.LB_FV_TILE, int(FV_SCHEDULE.split(":")[1]) if ":" in FV_SCHEDULE else 0)
        elif FV_SCHEDULE.startswith("march") or FV_SCHEDULE.startswith("pair"):
            kern = lb.LB_FV_MARCH if FV_SCHEDULE.startswith("march") else lb.LB_FV_PAIR
            g.set_fv_schedule(kern, int(FV_SCHEDULE.split(":")[1]) if ":" in FV_SCHEDULE else 0)
        elif tune:
            g.autotune_fv(5)
    return g


def schedule_name(lb, g, scheme):
    if isinstance(g, lb.Grid3):
        if scheme != "fv":
            if g.store == lb.LB_STORE_F32 and g.desc.nx % 2 == 0:
                return "3-D st pair (f32x2), two cells per thread, push"
            return "3-D st push"
        if g.fv_schedule == lb.LB3_FV_STAGED:
            return "3-D fv four passes (collision; staged predictor; star; staged corrector)"
        return "3-D fv four passes (collision; predictor; star; corrector)"
    if scheme != "fv":
        if g.store == lb.LB_STORE_F64:
            return "st push, one thread per cell"
        if g.store in (lb.LB_STORE_F16DEV, lb.LB_STORE_BF16DEV) and not g.thermal:
            if g.nx % 4 == 0 and g.desc.bcx == lb.LB_BC_PERIODIC:
                return "st quad (64-bit words, f32x2), four cells of two rows per thread"
            return "st pair (f32x2), two cells of two rows per thread"
        if g.store == lb.LB_STORE_F32 and not g.thermal and g.nx % 4 == 0 and g.desc.bcx == lb.LB_BC_PERIODIC:
            return "st quad (128-bit words, f32x2), four cells per thread"
        return "st pair (f32x2), two cells per thread"
    k, c = g.fv_schedule()
    if k == lb.LB_FV_TILE:
        return "fv tile %s (halo 4)" % {0: "32x16", 16: "16x16", 8: "16x8"}[c]
    if k == lb.LB_FV_SPLIT:
        return "fv split (f32x2) %s: collision+predictor, corrector" % {0: "32x16", 16: "16x16"}[c]
    if k == lb.LB_FV_PTILE:
        return "fv pair-tile (f32x2) %s (halo 4)" % {0: "32x16", 14: "32x14", 16: "16x16", 512: "32x16, 512 threads",
                                                      526: "32x14, 512 threads"}[c]
    return ("fv pair-march (f32x2)" if k == lb.LB_FV_PAIR else "fv march") + ", %d rows per CTA" % c


def time_steps(lb, torch, g, scheme, steps, warmup, flush=None):
    """Per-step CUDA-event durations (ms) of `steps` single-step launches."""
    if isinstance(g, lb.Grid3):
        step = (lambda h, n: g.step_fv(n)) if scheme == "fv" else (lambda h, n: g.step_st(n))
    else:
        step = lb.lb_step_fv if scheme == "fv" else lb.lb_step_st
    for _ in range(warmup):
        step(g.handle, 1)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    n0 = lb.lb_kernel_launches()
    for a, b in evs:
        if flush is not None:
            flush.zero_()
        a.record()
        step(g.handle, 1)
        b.record()
    torch.cuda.synchronize()
    launches = lb.lb_kernel_launches() - n0
    return [a.elapsed_time(b) for a, b in evs], launches


def source_hash(files):
    """Hash of the code of the given csrc files with comments and whitespace
    removed, so that a comment edit does not count as a kernel change."""
    import hashlib
    import re
    m = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1505_03271_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        m.update(" ".join(text.split()).encode())
    return m.hexdigest()[:16]


def measured_traffic(schedule, case):
    """DRAM bytes per launch from the committed ncu summary of this kernel
    and workload, or None if there is none or the kernel's code has changed
    since it was captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            table = json.load(fh)
        e = table["%s|%s" % (schedule, case)]
        return e["bytes"] if source_hash(e["files"]) == e["sources"] else None
    except (OSError, KeyError, ValueError):
        return None


def aggregate(local_s, cells, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas (one per rank): the
    slowest rank's time bounds the job, every rank did cells x steps."""
    import torch
    total_s = local_s
    if dist is not None and world > 1:
        t = torch.tensor([local_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return total_s, cells * steps * world / total_s / 1e6


def roofline(bytes_per_step, mean_ms, peak, peak_kind, traffic=None):
    achieved = bytes_per_step / (mean_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": f"{peak_kind} hbm_gbs"}


def alu_roofline(cfg, w, mean_ms, clocks):
    """The second roof of the step: algorithmic FP32 flops per second
    against the non-tensor FP32 peak at the GPU's maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    fpc = cfg.flops_per_cell(w.scheme, w.grid.get("thermal", False))
    achieved = fpc * w.cells / (mean_ms * 1e-3) / 1e12
    peak = cfg.fp32_peak_tflops(sms, mhz)
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "flops_per_cell": fpc,
            "peak_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (derived)" % (sms, mhz)}


STORE_LABEL = {0: "FP64", 1: "FP32", 2: "FP16 (f - w) deviations", 3: "BF16 (f - w) deviations"}


def state_bytes(cfg, w):
    """Device bytes of a grid's two population buffers."""
    return cfg.bytes_per_cell(w.grid["store"], w.grid.get("thermal", False),
                              19 if "nz" in w.grid else 9) * w.cells


def needs_flush(cfg, w):
    """L2 is flushed between timed steps unless the state is larger than
    four times the 129 MB L2."""
    return state_bytes(cfg, w) < 4 * 129e6


def measure(lb, torch, cfg, w, stream, peak, peak_kind, flush, steps, warmup, case):
    """Time `steps` single-step launches of a workload (after warm-up, L2
    flushed before each when the state is small).  Returns the grid (its
    schedule is the autotuner's) and the figures of its line."""
    g = make_grid(lb, w, stream)
    fl = flush if needs_flush(cfg, w) else None
    ms, launches = time_steps(lb, torch, g, w.scheme, steps, warmup, fl)
    mean = sum(ms) / len(ms)
    bpc = cfg.bytes_per_cell(w.grid["store"], w.grid.get("thermal", False), 19 if "nz" in w.grid else 9)
    sched = schedule_name(lb, g, w.scheme)
    tcase, scale = case if isinstance(case, tuple) else (case, 1)
    traffic = measured_traffic(sched, tcase) if tcase else None
    rl = roofline(bpc * w.cells, mean, peak, peak_kind, traffic * scale if traffic else None)
    if traffic and scale != 1:
        rl["traffic_source"] = "ncu on the %s case, scaled x%d by cells" % (tcase, scale)
    return g, {"mlups": round(w.cells / (mean * 1e-3) / 1e6, 1), "ms_per_step": round(mean, 5),
               "bytes_per_cell": bpc, "schedule": sched, "launches": launches, "roofline": rl,
               "roofline_alu": None if "nz" in w.grid else alu_roofline(cfg, w, mean, None),
               "l2": "flushed" if fl is not None else "state > L2"}


def compact(m):
    """One extra line in few characters: throughput, both roof fractions,
    the schedule and the ncu traffic when it is current."""
    out = {"mlups": m["mlups"], "ms_per_step": m["ms_per_step"], "frac_hbm": m["roofline"]["frac"],
           "bytes_per_cell": m["bytes_per_cell"], "schedule": m["schedule"]}
    if m["roofline"]["traffic"]:
        out["traffic"] = m["roofline"]["traffic"]
    if m.get("roofline_alu"):
        out["frac_alu"] = m["roofline_alu"]["frac"]
    return out


def extra_lines(lb, torch, cfg, stream, peak, peak_kind, flush, serving=None, cpu=True):
    """The other workloads.  The compact lines first; then config 2 (the FV
    channel) and config 3 (the FV thermal RB cell, the paper's Sec. IV
    workload) as full lines with their own roofline, oracle baseline,
    oracle error and end-to-end figure, config 3 last."""
    out = {}
    if serving is not None:
        out["serving"] = serving
    specs = [("st8192_bf16dev", cfg.st_sweep(8192, lb.LB_STORE_BF16DEV), 20, ("st4096_bf16dev", 4)),
             ("st8192_f16dev", cfg.st_sweep(8192, lb.LB_STORE_F16DEV), 20, ("st4096_f16dev", 4)),
             ("fv4096_f32", _fv_big(cfg, 4096), 10, "fv4096"),
             ("fv_rb1024_f32", cfg.rayleigh_benard(1024, 1e8, store=lb.LB_STORE_F32), 20, "rb1024_f32"),
             ("rb3d_fv_f32", cfg.rb3d_table("fv"), 10, "rb3d_fv"),
             ("rb3d_st_f32", cfg.rb3d_table("st"), 20, "rb3d_st")]
    for name, w, k, case in specs:
        g, m = measure(lb, torch, cfg, w, stream, peak, peak_kind, flush, k, 3, case)
        out[name] = compact(m)
        g.close()
        torch.cuda.empty_cache()
    for name, w, k, case, window, single, inner in (
            ("channel_f32", cfg.channel(), 200, "channel", 500, 50, 1000),
            ("fv_rb1024_f16dev", cfg.rayleigh_benard(1024, 1e8), 20, "rb1024", 20, 2, 2000)):
        g, m = measure(lb, torch, cfg, w, stream, peak, peak_kind, flush, k, 3, case)
        line = {"workload": describe(w), "mlups": m["mlups"], "ms_per_step": m["ms_per_step"],
                "schedule": m["schedule"], "l2": m["l2"], "roofline": m["roofline"],
                "roofline_alu": m["roofline_alu"]}
        line["e2e"] = e2e_measure(lb, torch, w, stream, g.fv_schedule(), inner)
        if cpu:
            line["cpu_baseline"], line["oracle_error"] = cpu_leg(lb, w, stream, g, window, single)
        out[name] = line
        g.close()
        torch.cuda.empty_cache()
    return out


def roofline_sweep(lb, torch, cfg, stream, peak, flush, sizes):
    """HBM roofline curve over grid sizes: the ST step with FP32, BF16 and
    FP16 deviation storage and the FV step (FP32, periodic flow) on n x n
    grids, each step timed alone after an L2 flush.  One dict per point."""
    rows = []
    for n in sizes:
        for label, w in (("st_f32", cfg.st_sweep(n, lb.LB_STORE_F32)),
                         ("st_bf16dev", cfg.st_sweep(n, lb.LB_STORE_BF16DEV)),
                         ("st_f16dev", cfg.st_sweep(n, lb.LB_STORE_F16DEV)),
                         ("fv_f32", _fv_big(cfg, n))):
            g = make_grid(lb, w, stream)
            ms, _ = time_steps(lb, torch, g, w.scheme, 20 if w.scheme == "st" else 10, 3, flush)
            mean = sum(ms) / len(ms)
            bpc = cfg.bytes_per_cell(w.grid["store"], False, 9)
            rows.append({"sweep": label, "n": n, "cells": w.cells, "mlups": round(w.cells / (mean * 1e-3) / 1e6, 1),
                         "ms_per_step": round(mean, 5), "bytes_per_cell": bpc,
                         "frac_hbm": round(bpc * w.cells / (mean * 1e-3) / 1e9 / peak, 4),
                         "schedule": schedule_name(lb, g, w.scheme)})
            g.close()
            torch.cuda.empty_cache()
    return rows


def _fv_big(cfg, n):
    """Periodic n x n FV TGV, FP32 (flow only), dt = 0.5: FV kernel at scale."""
    from paper_1505_03271_gb300 import LB_INIT_TGV, LB_STORE_F32
    return cfg.Workload("fv%d" % n, dict(nx=n, ny=n, store=LB_STORE_F32),
                        dict(tau=0.3, dt=0.5), dict(kind=LB_INIT_TGV, u0=0.01), 10, "fv")


def serving_measure(lb, torch, count=120, rate=25.0):
    """Scaled config-5 stream through the batching server and one at a time."""
    from paper_1505_03271_gb300 import serving
    reqs = serving.make_requests(count, rate)
    srv = serving.run_server(lb, reqs, policy=lb.LB_SERVE_ARRIVAL)
    shortest = serving.run_server(lb, reqs, policy=lb.LB_SERVE_SHORTEST)
    share = serving.run_server(lb, reqs, policy=lb.LB_SERVE_SHARE)
    seq = serving.run_sequential(lb, torch, reqs)
    # the same request must give the same Nusselt numbers both ways
    diffs = [abs(srv["results"][r.rid]["nu_vol"] - seq["results"][r.rid]["nu_vol"])
             for r in reqs if srv["results"][r.rid]["status"] == 0 and seq["results"][r.rid]["status"] == 0]
    keep = ("requests", "ok", "unstable", "cell_updates", "wall_s", "mlups", "tts_p50_s", "tts_p99_s")
    return {"workload": "RB FV requests, N in {64..1024}^2 tanh plates, Ra log-uniform 1e4-1e8, Pr=1, "
                        "steps uniform 50-1000 (the 1000-20000 of the full stream divided by 20), FP16 deviation storage, "
                        "Poisson arrivals %.0f/s, %d requests" % (rate, count),
            "policy": "server: arrival order (LB_SERVE_ARRIVAL); also shortest first and equal share",
            "server": {k: srv[k] for k in keep}, "server_shortest_first": {k: shortest[k] for k in keep},
            "server_equal_share": {k: share[k] for k in keep},
            "sequential": {k: seq[k] for k in keep},
            "max_abs_nu_vol_diff_server_vs_sequential": max(diffs) if diffs else None}


def e2e_measure(lb, torch, w, stream, fv_schedule=None, inner=None, reps=2):
    """The same metric end to end through the public API, host buffers in and
    out.  Per iteration: lb_init from pinned host fields (rho, u_x, u_y, and
    T for a thermal grid), `inner` steps in one lb_step call (long runs
    replay a captured CUDA graph), then u_x (and the Nusselt numbers of a
    thermal grid) read back to host.  The fields are the workload's own
    initial state, read once from the GPU before timing."""
    inner = inner or w.steps
    nx, ny = w.grid["nx"], w.grid["ny"]
    thermal = bool(w.grid.get("thermal", False))
    grid = dict(w.grid)
    store = grid.pop("store")
    g = lb.Grid(store=store, stream=stream, **grid)
    g.init(**w.params, **w.init)
    if fv_schedule is not None and w.scheme == "fv":
        g.set_fv_schedule(*fv_schedule)
    pin = lambda: torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    rho, ux, uy, T, out = pin(), pin(), pin(), pin(), pin()
    lb.lb_moments(g.handle, rho, ux, uy, T if thermal else None)
    step = lb.lb_step_fv if w.scheme == "fv" else lb.lb_step_st
    times = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.init(**w.params, kind=lb.LB_INIT_FIELDS, rho=rho, ux=ux, uy=uy, T=T if thermal else None)
        step(g.handle, inner)
        lb.lb_moments(g.handle, None, out, None, None)
        if thermal:
            g.nusselt()
        t1 = time.perf_counter()
        if r > 0:
            times.append(t1 - t0)
    g.close()
    fields = 4 if thermal else 3
    l2 = "state stays in the 129 MB L2 across the run" if state_bytes_of(w) < 129e6 else "state > L2"
    return {"value": round(w.cells * inner / (sum(times) / len(times)) / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": fields * 8 * nx * ny, "d2h_bytes_per_step": 8 * nx * ny + (24 if thermal else 0),
            "lb_steps_per_step": inner,
            "note": "step = lb_init from %d pinned host fields + %d %s steps in one call (CUDA-graph replays) + "
                    "u_x%s to host; %s" % (fields, inner, w.scheme.upper(), " and Nu" if thermal else "", l2)}


def state_bytes_of(w):
    from paper_1505_03271_gb300 import configs as cfg
    return state_bytes(cfg, w)


# ------------------------------------------------------------------ oracle --

def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo, else the
    machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_window(w, steps, threads=None):
    """Oracle steps of a workload from its initial state: exactly `steps`
    steps (a fixed window) on `threads` OpenMP threads (default: every host
    core).  Returns the grid, the seconds the steps took and the threads."""
    import oracle as O
    O.build()
    threads = threads or os.cpu_count() or 1
    O.set_threads(threads)
    grid = dict(w.grid)
    grid.pop("store")
    r = O.RefGrid(grid["nx"], grid["ny"], grid.get("lx"), grid.get("ly"), grid.get("sx", 0),
                  grid.get("sy", 0), grid.get("stretch_x", 0.0), grid.get("stretch_y", 0.0),
                  grid.get("bcx", 0), grid.get("bcy", 0), grid.get("thermal", False))
    r.set_params(**w.params)
    kind = {0: O.INIT_TGV, 1: O.INIT_SHEAR, 2: O.INIT_POISEUILLE, 3: O.INIT_RB}[w.init["kind"]]
    r.init_preset(kind, w.init.get("u0", 0.0), w.init.get("amp", 0.0), w.init.get("mode", 1),
                  w.init.get("seed", 0))
    step = r.step_fv if w.scheme == "fv" else r.step_st
    t0 = time.perf_counter()
    step(steps)
    return r, time.perf_counter() - t0, threads


def oracle_sample(w, budget_s=15.0, steps_cap=None, threads=None):
    """Oracle steps for about budget_s seconds (one step at a time)."""
    r, _, threads = oracle_window(w, 0, threads)
    step = r.step_fv if w.scheme == "fv" else r.step_st
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s and (steps_cap is None or done < steps_cap):
        step(1)
        done += 1
    return r, done, time.perf_counter() - t0, threads


def cpu_leg(lb, w, stream, g, window, single):
    """The oracle timed on this host's cores over a fixed window of the
    workload (`window` steps on every core, `single` steps on one thread),
    and the GPU's error against it after the same window: relative L2 of u,
    and for a thermal grid the largest relative Nusselt-number error."""
    r, el, thr = oracle_window(w, window)
    _, el1, _ = oracle_window(w, single, threads=1)
    grid = dict(w.grid)
    store = grid.pop("store")
    g2 = lb.Grid(store=store, stream=stream, **grid)
    g2.init(**w.params, **w.init)
    if w.scheme == "fv":
        g2.set_fv_schedule(*g.fv_schedule())
        lb.lb_step_fv(g2.handle, window)
    else:
        lb.lb_step_st(g2.handle, window)
    _, ux, uy, _ = g2.moments()
    _, vx, vy, _ = r.moments()
    err = {"steps": window,
           "rel_l2_u": float(np.sqrt(((ux - vx) ** 2 + (uy - vy) ** 2).sum() / (vx**2 + vy**2).sum()))}
    if w.grid.get("thermal"):
        err["nu_rel_err"] = float(max(abs(a / b - 1.0) for a, b in zip(g2.nusselt(), r.nusselt())))
    g2.close()
    base = {"value": round(w.cells * window / el / 1e6, 3), "unit": "MLUPS", "cores": thr, "kind": "oracle",
            "sample": "%d %s steps of the full %dx%d grid (%.1f s)" % (window, w.scheme.upper(), w.grid["nx"],
                                                                      w.grid["ny"], el),
            "cpu_model": cpu_model(),
            "single_thread": {"value": round(w.cells * single / el1 / 1e6, 3),
                              "sample": "%d steps, full grid (%.1f s)" % (single, el1)}}
    return base, err


def run_reference(args):
    """The reference arm of this tier: the FP64 oracle, as it stands, on the
    headline workload and this host's cores.  One reference step is one
    oracle step of the full grid."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1505_03271_gb300 import configs as cfg
    w = case_workload(cfg, args.case)
    r, _, thr = oracle_window(w, 0)
    step = r.step_fv if w.scheme == "fv" else r.step_st
    for _ in range(args.warmup):
        step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(1)
    el = time.perf_counter() - t0
    v = w.cells * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w, args.gpus),
            "schedule": "FP64 oracle, one cell at a time, OpenMP over rows",
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": thr, "kind": "oracle",
                             "sample": "%d full %s steps of the %dx%d grid" % (args.steps, w.scheme.upper(),
                                                                            w.grid["nx"], w.grid["ny"]),
                             "cpu_model": cpu_model()},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


HEADLINE = "st8192"


def case_workload(cfg, name):
    """Workloads that --case selects (the default, 'st8192', is the headline:
    config 4, the largest single-GPU configuration)."""
    import paper_1505_03271_gb300 as lb
    table = {
        "st8192": lambda: cfg.st_sweep(8192, lb.LB_STORE_F32),
        "channel": lambda: cfg.channel(),
        "st4096": lambda: cfg.st_sweep(4096, lb.LB_STORE_F32),
        "st4096_f16dev": lambda: cfg.st_sweep(4096, lb.LB_STORE_F16DEV),
        "st4096_bf16dev": lambda: cfg.st_sweep(4096, lb.LB_STORE_BF16DEV),
        "st8192_f16dev": lambda: cfg.st_sweep(8192, lb.LB_STORE_F16DEV),
        "st8192_bf16dev": lambda: cfg.st_sweep(8192, lb.LB_STORE_BF16DEV),
        "fv4096": lambda: _fv_big(cfg, 4096),
        "fv2048": lambda: _fv_big(cfg, 2048),
        "rb1024": lambda: cfg.rayleigh_benard(1024, 1e8),
        "rb1024_f32": lambda: cfg.rayleigh_benard(1024, 1e8, store=lb.LB_STORE_F32),
        "rb3d_fv": lambda: cfg.rb3d_table("fv"),
        "rb3d_st": lambda: cfg.rb3d_table("st"),
    }
    return table[name]()


def describe(w):
    """What a workload is, with its sizes."""
    g = w.grid
    store = STORE_LABEL[g["store"]]
    if w.name.startswith("st") and "nz" not in g:
        return ("ST D2Q9 %dx%d periodic, Taylor-Green mode 1 + shear wave mode 2 (u0 = A = 0.01), "
                "quoted tau = 0.8, %s storage, FP32 math" % (g["nx"], g["ny"], store)
                if g["store"] != 0 else "ST D2Q9 %dx%d periodic, FP64" % (g["nx"], g["ny"]))
    if w.name.startswith("channel"):
        return ("FV channel %dx%d, tanh delta=2 walls on y, tau=0.2 (ST tau~=0.7), Re=10, %s storage, "
                "FP32 math" % (g["nx"], g["ny"], store))
    if w.name.startswith("rb") and "nz" not in g:
        return ("FV thermal Rayleigh-Benard %dx%d, Ra=1e8, Pr=1, x periodic, tanh delta=2 plates, "
                "%s storage, FP32 math" % (g["nx"], g["ny"], store))
    return w.name


def _config(w, world=1):
    """The workload fields of the JSON line, the same for both arms."""
    from paper_1505_03271_gb300 import configs as cfg
    sb = state_bytes(cfg, w)
    return {"workload": describe(w), "cells": w.cells, "scheme": w.scheme,
            "steps_per_run": w.steps,
            "l2": ("flushed: 256 MiB write between timed steps" if needs_flush(cfg, w)
                   else "state %.1f GB > 129 MB L2, no flush" % (sb / 1e9)),
            "parallelism": "replicas" if world > 1 else "single"}


def visible_gpu_index(local):
    """nvidia-smi index of this rank's GPU (the first CUDA_VISIBLE_DEVICES
    entry when it is a number)."""
    first = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(first) if first.isdigit() else local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="headline only (for profiling)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baselines")
    ap.add_argument("--case", default=HEADLINE,
                    help="workload to time: st8192 (headline), channel, st4096, st4096_f16dev, "
                         "st4096_bf16dev, fv4096, fv2048, rb1024, rb1024_f32, rb3d_fv, rb3d_st")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream")
    ap.add_argument("--roofline-sweep", default=None, metavar="N,N,...",
                    help="print the ST/FV roofline curve over these n x n grid sizes instead of the bench line")
    ap.add_argument("--serving-full", type=float, default=None, metavar="LOAD",
                    help="run the configured serving stream (2000 requests, 1e3-2e4 steps) at LOAD x the "
                         "measured one-at-a-time capacity and print its JSON line instead of the bench line")
    ap.add_argument("--serving-requests", type=int, default=160)
    ap.add_argument("--serving-rate", type=float, default=60.0, help="Poisson arrivals per second")
    ap.add_argument("--fv-schedule", default="tune",
                    help="tune (autotuner), tile, march[:rows per CTA] or pair[:rows per CTA]")
    ap.add_argument("--fv3-schedule", default="auto", choices=["auto", "plain", "staged"],
                    help="flux passes of the 3-D FV step (include/lb3.h)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global FV_SCHEDULE, FV3_SCHEDULE
    FV_SCHEDULE = args.fv_schedule
    FV3_SCHEDULE = args.fv3_schedule
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1505_03271_gb300 as lb
    from paper_1505_03271_gb300 import configs as cfg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    lb.load()
    stream = torch.cuda.current_stream().cuda_stream
    peak, peak_kind = load_peaks()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    if args.roofline_sweep:
        sizes = [int(v) for v in args.roofline_sweep.split(",")]
        with ClockSampler(visible_gpu_index(local)) as clk:
            rows = roofline_sweep(lb, torch, cfg, stream, peak, flush, sizes)
        for r in rows:
            r["peak"], r["peak_source"] = peak, f"{peak_kind} hbm_gbs"
            print(json.dumps(r), flush=True)
        print(json.dumps({"clocks": clk.summary()}), flush=True)
        return
    if args.serving_full is not None:
        from paper_1505_03271_gb300 import serving
        with ClockSampler(visible_gpu_index(local), period_ms=1000) as clk:
            res = serving.full_stream(lb, torch, load=args.serving_full)
        res["clocks"] = clk.summary()
        print(json.dumps({"serving_full": res}), flush=True)
        return
    w = case_workload(cfg, args.case)
    g = make_grid(lb, w, stream)
    fl = flush if needs_flush(cfg, w) else None

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    gpu_index = visible_gpu_index(local)
    barrier()
    with ClockSampler(gpu_index) as clk:
        ms, launches = time_steps(lb, torch, g, w.scheme, args.steps, args.warmup, fl)
    barrier()
    total_s, value = aggregate(sum(ms) * 1e-3, w.cells, args.steps, world, dist, "cuda")
    mean_ms = total_s * 1e3 / args.steps
    bpc = cfg.bytes_per_cell(w.grid["store"], w.grid.get("thermal", False), 19 if "nz" in w.grid else 9)
    dtype = "f64" if w.grid["store"] == lb.LB_STORE_F64 else "f32"
    sched = schedule_name(lb, g, w.scheme)
    tcase = {"st8192": ("st4096", 4)}.get(args.case, args.case)
    tcase, scale = tcase if isinstance(tcase, tuple) else (tcase, 1)
    traffic = measured_traffic(sched, tcase)
    rl = roofline(bpc * w.cells, mean_ms, peak, peak_kind, traffic * scale if traffic else None)
    if traffic and scale != 1:
        rl["traffic_source"] = "ncu on the %s case, scaled x%d by cells" % (tcase, scale)
    line = {"metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(mean_ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": _config(w, world), "schedule": sched,
            "gpu_launches": launches}
    full = not args.no_extra and args.case == HEADLINE
    cpu = rank == 0 and world == 1 and not args.no_cpu
    if full:
        serving = None if args.no_serving else serving_measure(lb, torch, args.serving_requests,
                                                               args.serving_rate)
        line["extra"] = extra_lines(lb, torch, cfg, stream, peak, peak_kind, flush, serving, cpu)
    line["roofline"] = rl
    line["roofline_alu"] = None if "nz" in w.grid else alu_roofline(cfg, w, mean_ms, None)
    if cpu and args.case in (HEADLINE, "channel", "rb1024"):
        window, single = {"st8192": (10, 1), "channel": (500, 50), "rb1024": (20, 2)}[args.case]
        line["cpu_baseline"], line["oracle_error"] = cpu_leg(lb, w, stream, g, window, single)
    if full:
        line["e2e"] = e2e_measure(lb, torch, w, stream, g.fv_schedule() if w.scheme == "fv" else None)
    line["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
