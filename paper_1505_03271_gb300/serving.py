"""Serving workload and drivers (host logic): a stream of independent
Rayleigh-Benard FV requests, as in the paper's parameter studies (Sec. IV:
several grids and Rayleigh numbers), run through the continuous-batching
server or one at a time.

Request recipe (seeded): square cell of N x N, N uniform in
{64, 128, 256, 512, 1024}, H = L = N, x periodic, tanh plates (delta = 2);
Ra log-uniform in [1e4, 1e8], Pr = 1, parameters by `configs.rb_params`;
FV time step dt = 0.9 min(dx_min, 8 tau); step count uniform in
[steps_lo, steps_hi]; seeded 1e-3 perturbation (seed = request id).
Arrivals are a Poisson process of rate `rate` per second.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import LB_AXIS_TANH, LB_BC_WALLS, LB_INIT_RB, LB_STORE_F16DEV
from . import configs as cfg

SIZES = (64, 128, 256, 512, 1024)


@dataclass
class Request:
    rid: int
    arrival: float
    n: int
    Ra: float
    nsteps: int
    params: dict

    @property
    def cells(self):
        return self.n * self.n

    def grid_kwargs(self):
        return dict(nx=self.n, ny=self.n, lx=float(self.n), ly=float(self.n), sy=LB_AXIS_TANH,
                    stretch_y=2.0, bcy=LB_BC_WALLS)


def make_requests(count: int, rate: float, steps_lo: int = 50, steps_hi: int = 1000,
                  seed_arrivals: int = 1, seed_params: int = 2, sizes=SIZES):
    ra = np.random.default_rng(seed_arrivals)
    rp = np.random.default_rng(seed_params)
    t = np.cumsum(ra.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        n = int(rp.choice(sizes))
        Ra = float(10 ** rp.uniform(4.0, 8.0))
        steps = int(rp.integers(steps_lo, steps_hi + 1))
        p = cfg.rb_params(Ra, 1.0, float(n))
        dt = cfg.fv_dt(cfg.min_cell(n, float(n), LB_AXIS_TANH, 2.0), min(p.tau, p.tau_g))
        params = dict(tau=p.tau, tau_g=p.tau_g, dt=dt, beta=p.beta, grav=p.grav, T0=p.T0,
                      T_bot=p.T_bot, T_top=p.T_top)
        out.append(Request(i + 1, float(t[i]), n, Ra, steps, params))
    return out


def _percentiles(x):
    x = np.asarray(x, dtype=float)
    if x.size == 0:
        return None, None
    return float(np.percentile(x, 50)), float(np.percentile(x, 99))


def run_server(lb, requests, store=LB_STORE_F16DEV, steps_per_launch=50, hbm_budget=200 << 30, policy=None):
    """Submit each request at its arrival time (server clock), pump until all
    are done.  Returns per-request results and aggregate figures."""
    s = lb.Server(store=store, thermal=True, hbm_budget=hbm_budget, steps_per_launch=steps_per_launch,
                  policy=policy)
    pending = list(requests)
    results = {}
    t_start = s.clock()
    while pending or len(results) < len(requests):
        now = s.clock() - t_start
        while pending and pending[0].arrival <= now:
            r = pending.pop(0)
            s.submit(r.rid, r.nsteps, **r.grid_kwargs(), kind=LB_INIT_RB, amp=1e-3, seed=r.rid,
                     **r.params)
        active, queued = s.pump()
        for res in s.results():
            results[res["id"]] = res
        if active == 0 and queued == 0 and pending:
            wait = pending[0].arrival - (s.clock() - t_start)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    s.close()
    return summarize(requests, results, t_start)


def summarize(requests, results, t_start=0.0):
    ok = [r for r in requests if results[r.rid]["status"] == 0]
    unstable = sum(1 for r in requests if results[r.rid]["status"] == 5)
    tts = [results[r.rid]["t_done"] - results[r.rid]["t_submit"] for r in requests]
    done = max(results[r.rid]["t_done"] for r in requests)
    first = min(results[r.rid]["t_submit"] for r in requests)
    work = sum(r.cells * results[r.rid]["steps"] for r in requests)
    p50, p99 = _percentiles(tts)
    return {"requests": len(requests), "ok": len(ok), "unstable": unstable,
            "cell_updates": int(work), "wall_s": done - first,
            "mlups": work / max(done - first, 1e-9) / 1e6, "tts_p50_s": p50, "tts_p99_s": p99,
            "results": results}


def run_sequential(lb, torch, requests, store=LB_STORE_F16DEV):
    """The same requests one at a time with the plain single-grid path, in
    arrival order; a request starts when it has arrived and the previous one
    is done."""
    results = {}
    t0 = time.perf_counter()
    clock = 0.0
    for r in requests:
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        start = time.perf_counter() - t0
        g = lb.Grid(thermal=True, store=store, **r.grid_kwargs())
        g.init(kind=LB_INIT_RB, amp=1e-3, seed=r.rid, **r.params)
        status = 0
        nu = (0.0, 0.0, 0.0)
        try:
            g.step_fv(r.nsteps)
            g.conservation()
            nu = g.nusselt()
        except lb.LBError as e:
            status = e.status
        g.close()
        end = time.perf_counter() - t0
        results[r.rid] = {"id": r.rid, "status": status, "steps": r.nsteps, "t_submit": r.arrival,
                          "t_admit": start, "t_done": end, "nu_vol": nu[0], "nu_bot": nu[1],
                          "nu_top": nu[2]}
        clock = end
    return summarize(requests, results)


def mean_work(steps_lo: int = 1000, steps_hi: int = 20000, sizes=SIZES) -> float:
    """Expected cell updates of one request of the stream: E[N^2] E[steps]."""
    return float(np.mean([n * n for n in sizes])) * 0.5 * (steps_lo + steps_hi)


def sequential_capacity(lb, torch, sample: int = 10, steps_lo: int = 1000, steps_hi: int = 20000,
                        store=LB_STORE_F16DEV) -> float:
    """Requests per second the one-at-a-time path sustains on the full
    stream's request mix: a seeded sample of requests (seeds 5 and 6, not the
    stream's), each of every size, run back to back; capacity = measured
    cell updates per second / the stream's mean work per request."""
    pool = make_requests(20 * len(SIZES), 1e9, steps_lo, steps_hi, seed_arrivals=5, seed_params=6)
    per = max(1, sample // len(SIZES))
    reqs = []
    for n in SIZES:  # the same number of each size, as in the stream
        reqs += [r for r in pool if r.n == n][:per]
    res = run_sequential(lb, torch, [Request(r.rid, 0.0, r.n, r.Ra, r.nsteps, r.params) for r in reqs], store)
    return res["mlups"] * 1e6 / mean_work(steps_lo, steps_hi)


def full_stream(lb, torch, load: float = 0.8, count: int = 2000, steps_lo: int = 1000, steps_hi: int = 20000,
                capacity: float | None = None, store=LB_STORE_F16DEV):
    """The configured serving stream: `count` requests with the full step
    range, Poisson arrivals at `load` times the measured one-at-a-time
    capacity, through the arrival-order server and one at a time."""
    from . import LB_SERVE_ARRIVAL
    cap = capacity if capacity is not None else sequential_capacity(lb, torch, steps_lo=steps_lo, steps_hi=steps_hi)
    rate = load * cap
    reqs = make_requests(count, rate, steps_lo, steps_hi)
    srv = run_server(lb, reqs, store=store, policy=LB_SERVE_ARRIVAL)
    seq = run_sequential(lb, torch, reqs, store)
    keep = ("requests", "ok", "unstable", "cell_updates", "wall_s", "mlups", "tts_p50_s", "tts_p99_s")
    diffs = [abs(srv["results"][r.rid]["nu_vol"] - seq["results"][r.rid]["nu_vol"]) for r in reqs
             if srv["results"][r.rid]["status"] == 0 and seq["results"][r.rid]["status"] == 0]
    return {"requests": count, "steps": [steps_lo, steps_hi], "load": load,
            "capacity_req_per_s": cap, "rate_req_per_s": rate,
            "server_arrival": {k: srv[k] for k in keep}, "sequential": {k: seq[k] for k in keep},
            "max_abs_nu_vol_diff": max(diffs) if diffs else None}
