"""Benchmark of the lattice Boltzmann time step on GB300.

Default workload: the FV body-force channel, 256 x 512 cells, tanh wall
refinement (delta = 2) on y, FP32 arithmetic on f - w storage, Re = 10.
One bench step = one FV time step (one fused kernel launch).  The state is
9.4 MB, far below the 129 MB L2, so a 256 MiB buffer is written between timed
steps and each step is timed alone with CUDA events on the launching stream.

Extra lines in the same JSON object (not the headline): ST on 8192^2 (FP32,
BF16 and FP16 deviation storage; state larger than L2), FV on 4096^2 FP32 and
FV thermal RB 1024^2 with FP16 storage.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

    def __init__(self, gpu_index: int, period_ms: int = 100):
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
            return "3-D st push"
        if g.fv_schedule == lb.LB3_FV_STAGED:
            return "3-D fv four passes (collision; staged predictor; star; staged corrector)"
        return "3-D fv four passes (collision; predictor; star; corrector)"
    if scheme != "fv":
        if g.store == lb.LB_STORE_F64:
            return "st push, one thread per cell"
        if g.store in (lb.LB_STORE_F16DEV, lb.LB_STORE_BF16DEV) and not g.thermal:
            return "st pair (f32x2), two cells of two rows per thread"
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


def extra_lines(lb, torch, cfg, stream, peak, peak_kind, flush):
    out = {}
    # (name, workload, steps, flush, traffic case); the 8192^2 ST traffic is
    # the ncu capture of 4096^2 scaled by the cell count (ST moves every
    # cell's populations once, so its DRAM bytes grow with the cells)
    specs = [("st8192_f32", cfg.st_sweep(8192, lb.LB_STORE_F32), 20, None, ("st4096", 4)),
             ("st8192_bf16dev", cfg.st_sweep(8192, lb.LB_STORE_BF16DEV), 20, None, None),
             ("st8192_f16dev", cfg.st_sweep(8192, lb.LB_STORE_F16DEV), 20, None, ("st4096_f16dev", 4)),
             ("fv4096_f32", _fv_big(cfg, 4096), 10, None, None),
             ("fv_rb1024_f16dev", cfg.rayleigh_benard(1024, 1e8), 20, flush, "rb1024"),
             ("fv_rb1024_f32", cfg.rayleigh_benard(1024, 1e8, store=lb.LB_STORE_F32), 20, flush, None),
             ("rb3d_fv_f32", cfg.rb3d_table("fv"), 10, None, "rb3d_fv"),
             ("rb3d_st_f32", cfg.rb3d_table("st"), 20, None, "rb3d_st")]
    for name, w, k, fl, case in specs:
        g = make_grid(lb, w, stream)
        ms, _ = time_steps(lb, torch, g, w.scheme, k, 3, fl)
        mean = sum(ms) / len(ms)
        bpc = cfg.bytes_per_cell(w.grid["store"], w.grid.get("thermal", False), 19 if "nz" in w.grid else 9)
        sched = schedule_name(lb, g, w.scheme)
        case, scale = case if isinstance(case, tuple) else (case, 1)
        traffic = measured_traffic(sched, case) if case else None
        rl = roofline(bpc * w.cells, mean, peak, peak_kind, traffic * scale if traffic else None)
        if traffic and scale != 1:
            rl["traffic_source"] = "ncu on the %s case, scaled x%d by cells" % (case, scale)
        out[name] = {"mlups": round(w.cells / (mean * 1e-3) / 1e6, 1), "ms_per_step": round(mean, 5),
                     "bytes_per_cell": bpc, "schedule": sched,
                     "roofline": rl,
                     "roofline_alu": None if "nz" in w.grid else alu_roofline(cfg, w, mean, None),
                     "cells": w.cells, "l2": "flushed" if fl is not None else "state > L2"}
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


def e2e_measure(lb, torch, w, stream, reps=3, inner=1000):
    """Through the public API with host buffers: per iteration, upload rho, ux,
    uy from pinned host memory (lb_init FIELDS), advance `inner` FV steps,
    read u_x back to host (lb_moments)."""
    nx, ny = w.grid["nx"], w.grid["ny"]
    grid = dict(w.grid)
    store = grid.pop("store")
    g = lb.Grid(store=store, stream=stream, **grid)
    pin = lambda: torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    rho, ux, uy, out = pin(), pin(), pin(), pin()
    from paper_1505_03271_gb300 import configs as cfg
    xi = cfg.faces(ny, w.grid["ly"], w.grid["sy"], w.grid["stretch_y"])
    yc = 0.5 * (xi[1:] + xi[:-1])
    rho[:] = 1.0
    ux[:] = (4 * w.init["u0"] * yc * (w.grid["ly"] - yc) / w.grid["ly"] ** 2)[:, None]
    uy[:] = 0.0

    def timed(graph_steps):
        g.set_graph_steps(graph_steps)
        times = []
        for r in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.init(**w.params, kind=lb.LB_INIT_FIELDS, rho=rho, ux=ux, uy=uy)
            lb.lb_step_fv(g.handle, inner)
            lb.lb_moments(g.handle, None, out, None, None)
            t1 = time.perf_counter()
            if r > 0:
                times.append(t1 - t0)
        return round(w.cells * inner / min(times) / 1e6, 1)

    plain = timed(0)
    graph_steps = 32
    v = timed(graph_steps)
    g.close()
    return {"value": v, "unit": "MLUPS",
            "h2d_bytes_per_step": 3 * 8 * nx * ny, "d2h_bytes_per_step": 8 * nx * ny,
            "lb_steps_per_step": inner, "graph_steps": graph_steps, "value_plain_launches": plain,
            "note": "step = lb_init from pinned host rho,ux,uy + %d FV steps (replays of a %d-step "
                    "CUDA graph) + u_x to host" % (inner, graph_steps)}


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


def oracle_sample(w, budget_s=15.0, steps_cap=None, threads=None):
    """Oracle FV/ST steps on the workload for about budget_s seconds, on
    `threads` OpenMP threads (default: every host core)."""
    import oracle as O
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
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s and (steps_cap is None or done < steps_cap):
        step(1)
        done += 1
    el = time.perf_counter() - t0
    return r, done, el, threads


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1505_03271_gb300 import configs as cfg
    w = cfg.channel()
    import oracle as O
    O.build()
    O.set_threads(os.cpu_count() or 1)
    grid = dict(w.grid)
    grid.pop("store")
    r = O.RefGrid(grid["nx"], grid["ny"], grid["lx"], grid["ly"], 0, grid["sy"], 0.0,
                  grid["stretch_y"], 0, grid["bcy"], False)
    r.set_params(**w.params)
    r.init_preset(O.INIT_POISEUILLE, w.init["u0"])
    # each reference step: one oracle FV step of the full channel
    for _ in range(args.warmup):
        r.step_fv(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.step_fv(1)
    el = time.perf_counter() - t0
    v = w.cells * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w),
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": O.get_threads(),
                             "kind": "oracle", "sample": "%d full FV steps of the channel" % args.steps,
                             "cpu_model": cpu_model()},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def case_workload(cfg, name):
    """Workloads that --case selects (the default, 'channel', is the headline)."""
    import paper_1505_03271_gb300 as lb
    table = {
        "channel": lambda: cfg.channel(),
        "st8192": lambda: cfg.st_sweep(8192, lb.LB_STORE_F32),
        "st4096": lambda: cfg.st_sweep(4096, lb.LB_STORE_F32),
        "st4096_f16dev": lambda: cfg.st_sweep(4096, lb.LB_STORE_F16DEV),
        "fv4096": lambda: _fv_big(cfg, 4096),
        "fv2048": lambda: _fv_big(cfg, 2048),
        "rb1024": lambda: cfg.rayleigh_benard(1024, 1e8),
        "rb3d_fv": lambda: cfg.rb3d_table("fv"),
        "rb3d_st": lambda: cfg.rb3d_table("st"),
    }
    return table[name]()


def _config(w, case="channel"):
    if case != "channel":
        return {"workload": w.name, "cells": w.cells, "scheme": w.scheme,
                "store": w.grid["store"], "thermal": bool(w.grid.get("thermal", False)),
                "l2": "flushed: 256 MiB write between timed steps"}
    return {"workload": "FV channel %dx%d, tanh delta=2 walls on y, tau=0.2 (ST tau~=0.7), Re=10, "
                        "FP32 math on f-w storage" % (w.grid["nx"], w.grid["ny"]),
            "cells": w.cells, "scheme": "fv semi-implicit + Heun + QUICK",
            "dt": round(w.params["dt"], 6), "l2": "flushed: 256 MiB write between timed steps"}


def visible_gpu_index(local):
    """nvidia-smi index of this rank's GPU (the first CUDA_VISIBLE_DEVICES
    entry when it is a number)."""
    first = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(first) if first.isdigit() else local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="headline only (for profiling)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--case", default="channel",
                    help="workload to time: channel (headline), st8192, st4096, st4096_f16dev, "
                         "fv4096, fv2048, rb1024, rb3d_fv, rb3d_st (3-D Table rb grids)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream")
    ap.add_argument("--roofline-sweep", default=None, metavar="N,N,...",
                    help="print the ST/FV roofline curve over these n x n grid sizes instead of the bench line")
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
    if args.roofline_sweep:
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        sizes = [int(v) for v in args.roofline_sweep.split(",")]
        with ClockSampler(visible_gpu_index(local)) as clk:
            rows = roofline_sweep(lb, torch, cfg, stream, peak, flush, sizes)
        for r in rows:
            r["peak"], r["peak_source"] = peak, f"{peak_kind} hbm_gbs"
            print(json.dumps(r), flush=True)
        print(json.dumps({"clocks": clk.summary()}), flush=True)
        return
    w = case_workload(cfg, args.case)
    g = make_grid(lb, w, stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    gpu_index = visible_gpu_index(local)
    barrier()
    with ClockSampler(gpu_index) as clk:
        ms, launches = time_steps(lb, torch, g, w.scheme, args.steps, args.warmup, flush)
    barrier()
    total_s, value = aggregate(sum(ms) * 1e-3, w.cells, args.steps, world, dist, "cuda")
    mean_ms = total_s * 1e3 / args.steps
    bpc = cfg.bytes_per_cell(w.grid["store"], w.grid.get("thermal", False), 19 if "nz" in w.grid else 9)
    dtype = "f64" if w.grid["store"] == lb.LB_STORE_F64 else "f32"
    line = {"metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(mean_ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": _config(w, args.case), "gpu_launches": launches,
            "roofline": roofline(bpc * w.cells, mean_ms, peak, peak_kind,
                                 measured_traffic(schedule_name(lb, g, w.scheme), args.case)),
            "clocks": clk.summary()}
    line["roofline_alu"] = None if "nz" in w.grid else alu_roofline(cfg, w, mean_ms, line["clocks"])
    line["config"]["parallelism"] = "replicas" if world > 1 else "single"
    line["config"]["schedule"] = schedule_name(lb, g, w.scheme)
    if not args.no_extra and args.case == "channel":
        line["e2e"] = e2e_measure(lb, torch, w, stream)
        line["extra"] = extra_lines(lb, torch, cfg, stream, peak, peak_kind, flush)
        if not args.no_serving:
            line["extra"]["serving"] = serving_measure(lb, torch, args.serving_requests, args.serving_rate)
    if rank == 0 and world == 1 and not args.no_cpu and args.case == "channel":
        import oracle as O
        O.build()
        r, done, el, thr = oracle_sample(w, budget_s=15.0)
        _, done1, el1, _ = oracle_sample(w, budget_s=5.0, threads=1)
        # error of the GPU against the oracle after the same number of steps
        g2 = make_grid(lb, w, stream, tune=False)
        g2.set_fv_schedule(*g.fv_schedule())
        lb.lb_step_fv(g2.handle, done)
        _, ux, uy, _ = g2.moments()
        _, vx, vy, _ = r.moments()
        err = float(np.sqrt(((ux - vx) ** 2 + (uy - vy) ** 2).sum() / (vx**2 + vy**2).sum()))
        line["cpu_baseline"] = {"value": round(w.cells * done / el / 1e6, 3), "unit": "MLUPS",
                                "cores": thr, "kind": "oracle",
                                "sample": "%d FV steps of the full channel (%.1f s)" % (done, el),
                                "cpu_model": cpu_model(),
                                "single_thread": {"value": round(w.cells * done1 / el1 / 1e6, 3),
                                                  "sample": "%d FV steps of the full channel (%.1f s)"
                                                            % (done1, el1)}}
        line["oracle_error"] = {"rel_l2_u": err, "steps": done}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
