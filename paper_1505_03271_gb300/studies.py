"""Accuracy and stability studies of Secs. III and V, run through the library.

  * ``viscosity_error``: relative error of the viscosity measured from the
    decay of the [1, 64] shear wave, nu_num against tau c_s^2, for FV and ST
    as a function of tau (Fig. KOL; FV with dt = 1 for tau >= 0.13 and 0.1
    below, ST with dt = 1).
  * ``poiseuille_unit_dx``: the Re = 10 Poiseuille error at fixed dx = 1
    (L = N) for FV and ST on uniform grids (Fig. POI).
  * ``poiseuille_vs_n``: relative L2 error of the Re = 10 Poiseuille profile
    against the parabola for a fixed channel width L = 64 and a varying
    number of cells N (Fig. POI2), for FV on uniform, tanh, sinh and
    Chebyshev grids and for ST on the uniform lattice.
  * ``poiseuille_vs_spacing``: the same at fixed N = 64 for a varying mean
    spacing <dx> = L/N, with the forcing rescaled to keep Re = 10 (Fig. POI3).
  * ``dt_max``: the largest stable FV time step as a function of tau for the
    Euler, semi-implicit and Heun schemes on the decaying [1, 64] shear wave
    (Fig. KOL3).
  * ``predictability_horizon``: the step at which two runs of the chaotic
    1024^2 Ra = 1e8 cell that start one ulp apart (one population of one
    cell) part by 1e-3 in a Nusselt number, in FP64 and in FP32.
  * ``rb3d_stats``: the 3-D Rayleigh-Benard runs of Table rb with FV (sinh z
    grid) and ST (uniform), time- and plane-averaged profiles T_m(z),
    T_rms(z), k_m(z) and Nu(z), and the cells inside the thermal boundary
    layer (Sec. IV, Figs. cfrT, cfrT2, cfrE, cfrLB).

Conventions (readings of the paper):
  * tau = 0.5 (physical) for the Poiseuille studies: the paper puts the best
    viscosity accuracy, and dt ~ 2 tau at dx ~ 1, there.  nu = tau/3,
    U = Re nu / L, a_x = 8 nu U / L^2, started on the parabola.
  * FV: dt = 0.9 min(dx_min, 8 tau) on every grid.  Grid stretchings are the
    paper's s1 = 0.98 (tanh, delta = atanh 0.98) and s2 = 6.5 (sinh).
  * ST at N cells over L runs in lattice units with dx = dt = L/N (the
    acoustic scaling of FV's unit lattice speeds): tau_lat = tau N / L, the
    same U (Mach number) and Re.
  * Steady state: each run lasts `relax` decay times of the slowest viscous
    mode, L^2 / (pi^2 nu), from the exact parabola; the remaining transient
    is exp(-relax) of the discretisation error.
  * Error: (sum (u_x - U)^2 dy / sum U^2 dy)^(1/2) over cell centres (the
    discrete L2 norm of Sec. III B).
  * Stability: the shear wave u_x = A sin(2 pi y / 64), A = 1e-5, plus 1e-6
    w_a Gaussian noise on every population (seed 1), is unstable when its
    kinetic energy grows tenfold or turns non-finite within 3000 steps;
    dt_max by bisection on [0.01, 4].

Independent runs are stepped concurrently, each grid on its own CUDA stream.
Run ``python -m paper_1505_03271_gb300.studies`` on a GPU to print the tables
as JSON lines.
"""
from __future__ import annotations

import json
import math
import sys
from dataclasses import dataclass

import numpy as np

from . import (LB_AXIS_CHEB, LB_AXIS_SINH, LB_AXIS_TANH, LB_AXIS_UNIFORM, LB_BC_WALLS, LB_FV_EULER,
               LB_FV_HEUN, LB_FV_SEMI, LB_INIT_POISEUILLE, LB_INIT_SHEAR, LB_STORE_F64)
from . import configs as cfg

TANH_DELTA = math.atanh(0.98)
SINH_S2 = 6.5
FV_GRIDS = {"uniform": (LB_AXIS_UNIFORM, 0.0), "tanh": (LB_AXIS_TANH, TANH_DELTA),
            "sinh": (LB_AXIS_SINH, SINH_S2), "cheb": (LB_AXIS_CHEB, 0.0)}
SCHEMES = {"euler": LB_FV_EULER, "semi": LB_FV_SEMI, "heun": LB_FV_HEUN}
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@dataclass(frozen=True)
class Poiseuille:
    """One steady Poiseuille run: method "st" or "fv-<grid>"."""
    method: str
    n: int
    L: float
    tau: float = 0.5
    Re: float = 10.0
    relax: float = 5.0

    def spec(self):
        nu = self.tau * cfg.CS2
        U = self.Re * nu / self.L
        if self.method == "st":
            dx = self.L / self.n
            tau_l = self.tau / dx
            nu_l = tau_l * cfg.CS2
            grid = dict(nx=1, ny=self.n, lx=1.0, ly=float(self.n), bcy=LB_BC_WALLS)
            params = dict(tau=tau_l, dt=1.0, ax=8.0 * nu_l * U / self.n**2)
            steps = int(math.ceil(self.relax * self.n**2 / (math.pi**2 * nu_l)))
            xi = np.arange(self.n + 1, dtype=float)
            return grid, params, U, steps, xi, float(self.n), "st"
        sp, st = FV_GRIDS[self.method.split("-", 1)[1]]
        grid = dict(nx=1, ny=self.n, lx=1.0, ly=self.L, sy=sp, stretch_y=st, bcy=LB_BC_WALLS)
        xi = cfg.faces(self.n, self.L, sp, st)
        dt = cfg.fv_dt(float(np.diff(xi).min()), self.tau)
        params = dict(tau=self.tau, dt=dt, ax=8.0 * nu * U / self.L**2)
        steps = int(math.ceil(self.relax * self.L**2 / (math.pi**2 * nu) / dt))
        return grid, params, U, steps, xi, self.L, "fv"

    def error(self, ux, xi, L, U):
        y = 0.5 * (xi[1:] + xi[:-1])
        dy = np.diff(xi)
        ref = 4.0 * U * y * (L - y) / L**2
        return float(np.sqrt(((ux - ref) ** 2 * dy).sum() / (ref**2 * dy).sum()))


def _run_concurrent(lb, torch, jobs, start, advance, finish, streams=8, chunk=256, after_round=None):
    """Step independent jobs round-robin, each on its own stream.
    start(job, stream) -> state with .remaining; advance(state, k) enqueues
    k steps; after_round(state), if given, runs once every active job has
    been advanced (it may synchronise); finish(state) -> result."""
    pending = list(jobs)
    active, out = [], {}
    while pending or active:
        while pending and len(active) < streams:
            job = pending.pop(0)
            s = torch.cuda.Stream()
            active.append((job, s, start(job, s.cuda_stream)))
        for job, s, st in active:
            k = min(chunk, st.remaining)
            if k > 0:
                advance(st, k)
                st.remaining -= k
        if after_round is not None:
            for job, s, st in active:
                after_round(st)
        for item in [a for a in active if a[2].remaining == 0]:
            job, s, st = item
            out[job] = finish(st)
            active.remove(item)
    return out


class _State:
    pass


def run_poiseuille(lb, torch, cases, streams=8):
    """Relative L2 error of each Poiseuille case (FP64 storage)."""
    def start(c, stream):
        grid, params, U, steps, xi, L, scheme = c.spec()
        st = _State()
        st.g = lb.Grid(store=LB_STORE_F64, stream=stream, **grid)
        st.g.init(kind=LB_INIT_POISEUILLE, u0=U, **params)
        st.scheme, st.remaining, st.c = scheme, steps, c
        st.aux = (U, steps, xi, L, params["dt"])
        return st

    def advance(st, k):
        (st.g.step_st if st.scheme == "st" else st.g.step_fv)(k)

    def finish(st):
        U, steps, xi, L, dt = st.aux
        _, ux, _, _ = st.g.moments()
        st.g.close()
        return {"method": st.c.method, "n": st.c.n, "L": st.c.L, "mean_dx": st.c.L / st.c.n,
                "U": U, "dt": dt, "steps": steps, "err": st.c.error(ux[:, 0], xi, L, U)}

    return _run_concurrent(lb, torch, cases, start, advance, finish, streams)


def viscosity_error(lb, torch, taus=(0.02, 0.05, 0.08, 0.1, 0.13, 0.2, 0.3, 0.5, 0.7, 1.0, 1.5, 2.0),
                    n=64, amp=1e-4, periods=0.25):
    """nu_num from the kinetic energy decay k(t) = k0 exp(-2 nu k^2 t) of the
    shear wave u_x = A sin(2 pi y / n) (Sec. III A), a least-squares fit of
    ln k over `periods` energy decay times; error |nu_num / (tau c_s^2) - 1|."""
    kw2 = (2 * math.pi / n) ** 2
    rows = []
    for scheme in ("fv", "st"):
        for tau in taus:
            nu = tau * cfg.CS2
            dt = 1.0 if (scheme == "st" or tau >= 0.13) else 0.1
            T = periods / (2 * nu * kw2)
            nsamp = 20
            steps = max(1, int(round(T / dt / nsamp)))
            g = lb.Grid(1, n, lx=1.0, ly=float(n), store=LB_STORE_F64)
            g.init(tau=tau, dt=dt, kind=LB_INIT_SHEAR, amp=amp)
            ts, ks = [], []
            for s in range(nsamp + 1):
                if s:
                    (g.step_fv if scheme == "fv" else g.step_st)(steps)
                _, ux, uy, _ = g.moments()
                ts.append(s * steps * dt)
                ks.append(0.5 * float((ux * ux + uy * uy).sum()))
            g.close()
            slope = np.polyfit(np.array(ts), np.log(np.array(ks)), 1)[0]
            nu_num = -slope / (2 * kw2)
            rows.append({"scheme": scheme, "tau": tau, "dt": dt, "nu": nu, "nu_num": nu_num,
                         "err": abs(nu_num / nu - 1)})
    return rows


def poiseuille_unit_dx(lb, torch, ns=(8, 16, 32, 64, 128, 256)):
    """Fig. POI: channel width L = N at dx = 1, Re = 10, tau = 0.5."""
    cases = []
    for n in ns:
        cases.append(Poiseuille("st", n, float(n)))
        cases.append(Poiseuille("fv-uniform", n, float(n)))
    res = run_poiseuille(lb, torch, cases)
    return [res[c] for c in cases]


def poiseuille_vs_n(lb, torch, ns=(8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256), cheb_max=128):
    cases = []
    for n in ns:
        cases.append(Poiseuille("st", n, 64.0))
        for gname in FV_GRIDS:
            if gname == "cheb" and n > cheb_max:
                continue
            cases.append(Poiseuille("fv-" + gname, n, 64.0))
    res = run_poiseuille(lb, torch, cases)
    return [res[c] for c in cases]


def poiseuille_vs_spacing(lb, torch, mean_dx=(0.25, 0.5, 1, 2, 4, 8, 16), n=64, cheb_max=8):
    cases = []
    for d in mean_dx:
        cases.append(Poiseuille("st", n, n * float(d)))
        for gname in FV_GRIDS:
            if gname == "cheb" and d > cheb_max:
                continue
            cases.append(Poiseuille("fv-" + gname, n, n * float(d)))
    res = run_poiseuille(lb, torch, cases)
    return [res[c] for c in cases]


def _shear_state(lb, scheme, tau, dt, stream, n=64, seed=1):
    g = lb.Grid(1, n, lx=1.0, ly=float(n), store=LB_STORE_F64, stream=stream).set_fv_scheme(scheme)
    g.init(tau=tau, dt=dt, kind=LB_INIT_SHEAR, amp=1e-5)
    f, _ = g.get_pops()
    rng = np.random.default_rng(seed)
    g.set_pops(f + 1e-6 * W[:, None, None] * rng.standard_normal(f.shape))
    return g


def _energy(g):
    _, ux, uy, _ = g.moments()
    return float((ux**2 + uy**2).sum())


def stable_many(lb, torch, probes, steps=3000, check=100, streams=16):
    """Stability verdict of each (scheme, tau, dt) probe."""
    def start(p, stream):
        scheme, tau, dt = p
        st = _State()
        st.g = _shear_state(lb, SCHEMES[scheme], tau, dt, stream)
        st.k0 = _energy(st.g)
        st.ok = True
        st.remaining = steps
        return st

    def advance(st, k):
        if st.ok:
            st.g.step_fv(k)

    def after_round(st):
        if not st.ok:
            return
        try:
            e = _energy(st.g)
        except lb.LBError:
            e = float("nan")
        if not math.isfinite(e) or e > 10 * st.k0:
            st.ok = False
            st.remaining = 0

    def finish(st):
        st.g.close()
        return st.ok

    return _run_concurrent(lb, torch, probes, start, advance, finish, streams, chunk=check,
                           after_round=after_round)


def dt_max(lb, torch, taus=(0.03, 0.05, 0.08, 0.125, 0.2, 0.3, 0.5, 0.7, 1.0, 1.5),
           schemes=("euler", "semi", "heun"), lo=0.01, hi=4.0, iters=9):
    """Largest stable dt by bisection for every (scheme, tau), all pairs
    bisected together."""
    keys = [(s, t) for s in schemes for t in taus]
    bounds = {k: [lo, hi] for k in keys}
    for _ in range(iters):
        probes = [(s, t, 0.5 * sum(bounds[(s, t)])) for s, t in keys]
        verdict = stable_many(lb, torch, probes)
        for (s, t, dt) in probes:
            bounds[(s, t)][0 if verdict[(s, t, dt)] else 1] = dt
    return [{"scheme": s, "tau": t, "dt_max": round(bounds[(s, t)][0], 4)} for s, t in keys]


def _ddz(z, f):
    """Second-order derivative at the nodes of a stretched grid: the
    3-point Lagrange derivative, central in the bulk, forward/backward at
    the first and last node (the post-processing of Sec. IV)."""
    n = len(z)
    d = np.zeros(n)
    for k in range(n):
        m = min(max(k, 1), n - 2)
        z0, z1, z2 = z[m - 1], z[m], z[m + 1]
        x = z[k]
        d[k] = (f[m - 1] * (2 * x - z1 - z2) / ((z0 - z1) * (z0 - z2)) +
                f[m] * (2 * x - z0 - z2) / ((z1 - z0) * (z1 - z2)) +
                f[m + 1] * (2 * x - z0 - z1) / ((z2 - z0) * (z2 - z1)))
    return d


def _ddz_weights(z):
    """Rows (m - 1, m, m + 1) and weights of _ddz at every node, for arrays."""
    n = len(z)
    m = np.clip(np.arange(n), 1, n - 2)
    z0, z1, z2, x = z[m - 1], z[m], z[m + 1], z
    w = np.stack([(2 * x - z1 - z2) / ((z0 - z1) * (z0 - z2)), (2 * x - z0 - z2) / ((z1 - z0) * (z1 - z2)),
                  (2 * x - z0 - z1) / ((z2 - z0) * (z2 - z1))], axis=1)
    return m, w


def _grad(f, dx, dy, mz, wz):
    """Gradient of a field [nz, ny, nx]: central differences in the periodic
    x and y, the stretched-grid 3-point derivative in z."""
    gx = (np.roll(f, -1, axis=2) - np.roll(f, 1, axis=2)) / (2.0 * dx)
    gy = (np.roll(f, -1, axis=1) - np.roll(f, 1, axis=1)) / (2.0 * dy)
    gz = (wz[:, 0, None, None] * f[mz - 1] + wz[:, 1, None, None] * f[mz] + wz[:, 2, None, None] * f[mz + 1])
    return gx, gy, gz


def _turnover(series, spacing):
    """Large-eddy turnover time: the first zero crossing of the
    autocorrelation of a time series sampled every `spacing` (Sec. IV), by
    linear interpolation; None if it never crosses."""
    x = np.asarray(series, dtype=float)
    x = x - x.mean()
    var = float((x * x).mean())
    if var <= 0:
        return None
    n = len(x)
    c = np.array([float((x[: n - l] * x[l:]).mean()) / var for l in range(n // 2)])
    for l in range(1, len(c)):
        if c[l] <= 0.0:
            return spacing * (l - 1 + c[l - 1] / (c[l - 1] - c[l]))
    return None


def rb3d_stats(lb, torch, scheme, tff_total=300.0, tff_avg=200.0, samples=100, store=None):
    """Table rb run with `scheme` ("fv" or "st"): tff_total free-fall times
    H / sqrt(beta g dT H), statistics over the last tff_avg of them from
    `samples` equally spaced snapshots (Sec. IV, Figs. cfrT, cfrT2, cfrE,
    cfrLB).
      Nu(z) = (<u_z (T - T0)> - kappa d<T>/dz) / (kappa dT / H);
      lambda_T = dT / (2 dT_m/dz at the plate);
      eps_u = nu sum_ij (d_j u_i)^2, eps_T = kappa sum_j (d_j T)^2 and the
      Bolgiano length L_B = (beta g)^(-3/2) <eps_u>^(5/4) <eps_T>^(-3/4);
      the large-eddy turnover time from the zero crossing of the
      autocorrelation of the total kinetic energy, and t_tot over it."""
    w = cfg.rb3d_table(scheme) if store is None else cfg.rb3d_table(scheme, store=store)
    gk = dict(w.grid)
    st = gk.pop("store")
    p = w.params
    H, dT = gk["lz"], p["T_bot"] - p["T_top"]
    bg = p["beta"] * p["grav"]
    tff = H / math.sqrt(bg * dT * H)
    dt = p["dt"]
    steps_total = int(round(tff_total * tff / dt))
    steps_avg = int(round(tff_avg * tff / dt))
    every = max(1, steps_avg // samples)
    g = lb.Grid3(store=st, **gk).init(**p, **w.init)
    step = g.step_fv if scheme == "fv" else g.step_st
    xi = cfg.faces(gk["nz"], H, gk.get("sz", 0), gk.get("stretch_z", 0.0))
    zc = 0.5 * (xi[1:] + xi[:-1])
    dzc = np.diff(xi)
    dx, dy = gk["lx"] / gk["nx"], gk["ly"] / gk["ny"]
    mz, wz = _ddz_weights(zc)
    kappa = p["tau_g"] * cfg.CS2
    nu = p["tau"] * cfg.CS2
    acc = {k: np.zeros(gk["nz"]) for k in ("T", "T2", "k", "uzT", "eu", "eT")}
    nus, energy = [], []
    step(steps_total - steps_avg)
    n = 0
    for _ in range(steps_avg // every):
        step(every)
        rho, ux, uy, uz, T = g.moments()
        acc["T"] += T.mean(axis=(1, 2))
        acc["T2"] += (T * T).mean(axis=(1, 2))
        kz = 0.5 * (ux * ux + uy * uy + uz * uz).mean(axis=(1, 2))
        acc["k"] += kz
        energy.append(float((kz * dzc).sum()))
        acc["uzT"] += (uz * (T - p["T0"])).mean(axis=(1, 2))
        eu = np.zeros_like(T)
        for comp in (ux, uy, uz):
            for gcomp in _grad(comp, dx, dy, mz, wz):
                eu += gcomp * gcomp
        acc["eu"] += nu * eu.mean(axis=(1, 2))
        eT = sum(gcomp * gcomp for gcomp in _grad(T, dx, dy, mz, wz))
        acc["eT"] += kappa * eT.mean(axis=(1, 2))
        nus.append(g.nusselt())
        n += 1
    g.close()
    Tm = acc["T"] / n
    Trms = np.sqrt(np.maximum(acc["T2"] / n - Tm * Tm, 0.0))
    km = acc["k"] / n
    nu_z = (acc["uzT"] / n - kappa * _ddz(zc, Tm)) / (kappa * dT / H)
    eps_u, eps_T = acc["eu"] / n, acc["eT"] / n
    LB = bg ** -1.5 * eps_u ** 1.25 * eps_T ** -0.75
    turn = _turnover(energy, every * dt / tff)
    nus = np.array(nus)
    nu_bot = float(nus[:, 1].mean())
    lam = H / (2.0 * nu_bot)
    lower = zc < 0.1 * H
    mid = int(np.argmin(np.abs(zc - 0.5 * H)))
    return {"scheme": scheme, "cells": w.cells, "nz": gk["nz"], "H": H, "dt": dt, "tff": tff,
            "steps": steps_total, "samples": n, "nu_vol": float(nus[:, 0].mean()), "nu_bot": nu_bot,
            "nu_top": float(nus[:, 2].mean()), "nu_vol_std": float(nus[:, 0].std()),
            "lambda_T": lam, "cells_in_bl": int((zc < lam).sum()), "z1": float(zc[0]),
            "nu_z_mean": float(nu_z.mean()), "nu_z_wall_dev": float(np.abs(nu_z[lower] - nu_z.mean()).max()),
            "turnover_tff": turn, "t_tot_over_turnover": (tff_total / turn) if turn else None,
            "LB_over_H_wall": float(LB[0] / H), "LB_over_H_mid": float(LB[mid] / H),
            "zc_over_H": [round(float(v), 5) for v in zc / H], "T_m": [round(float(v), 6) for v in Tm],
            "T_rms": [round(float(v), 6) for v in Trms], "k_m": [float(f"{v:.4e}") for v in km],
            "nu_z": [round(float(v), 4) for v in nu_z], "LB_over_H": [float(f"{v:.4e}") for v in LB / H],
            "eps_u": [float(f"{v:.4e}") for v in eps_u], "eps_T": [float(f"{v:.4e}") for v in eps_T]}


def rb3d(lb, torch, tff_total=300.0, tff_avg=200.0, samples=100):
    return [rb3d_stats(lb, torch, s, tff_total, tff_avg, samples) for s in ("fv", "st")]


def rb3d_long(lb, torch):
    """The same comparison over 600 free-fall times (statistics over the
    last 500, a snapshot every 2): beyond the paper's twelve large-eddy
    turnover times for both schemes."""
    return rb3d(lb, torch, 600.0, 500.0, 250)


def _nudge_one_cell(g, rel=None):
    """Change population 5 of one cell (a third of the way across, mid
    height) by the smallest step its storage keeps: one ulp of the FP64
    value, or, for 32-bit storage, the smallest power-of-two step that
    survives the round trip.  Returns the absolute change."""
    f, gg = g.get_pops()
    j, i = f.shape[1] // 2, f.shape[2] // 3
    v = f[5, j, i]
    step = float(np.nextafter(v, np.inf) - v)
    while True:
        f2 = f.copy()
        f2[5, j, i] = v + step
        g.set_pops(f2, gg)
        back = g.get_pops()[0][5, j, i]
        if back != v:
            return float(back - v)
        step *= 2.0


def predictability_horizon(lb, torch, n=1024, Ra=1e8, chunk=2000, max_steps=2000000, budget_s=420.0,
                           tol=1e-3, stores=("f64", "f32")):
    """Predictability horizon t_h of the chaotic RB cell (config 3): for each
    storage in `stores`, two runs of the same start, one of them with a
    single population of one cell changed by the smallest step the storage
    keeps (one ulp in FP64); t_h is the first sampled step at which a
    Nusselt number (volume or either plate) of the pair differs by more than
    `tol` relatively.  The pairs advance together, `chunk` steps at a time,
    until every pair has parted, max_steps, or budget_s seconds; a pair that
    has not parted reports a lower bound."""
    import time
    from . import STORE_NAMES
    pairs = {}
    for name in stores:
        w = cfg.rayleigh_benard(n, Ra, store=STORE_NAMES[name])
        grid = dict(w.grid)
        grid.pop("store")
        a = lb.Grid(store=STORE_NAMES[name], **grid).init(**w.params, **w.init)
        b = lb.Grid(store=STORE_NAMES[name], **grid).init(**w.params, **w.init)
        delta = _nudge_one_cell(b)
        pairs[name] = {"grids": (a, b), "delta": delta, "t_h": None, "last": 0.0}
    dt = w.params["dt"]
    t0 = time.perf_counter()
    steps = 0
    hist = []
    while steps < max_steps and time.perf_counter() - t0 < budget_s:
        live = [k for k, v in pairs.items() if v["t_h"] is None]
        if not live:
            break
        for k in live:
            for g in pairs[k]["grids"]:
                g.step_fv(chunk)
        steps += chunk
        row = {"step": steps}
        for k in live:
            a, b = pairs[k]["grids"]
            na, nb = a.nusselt(), b.nusselt()
            d = max(abs(x / y - 1.0) for x, y in zip(nb, na))
            pairs[k]["last"] = d
            row["d_" + k] = d
            row["nu_" + k] = [round(v, 6) for v in na]
            if d > tol:
                pairs[k]["t_h"] = steps
        hist.append(row)
        print(json.dumps({"horizon_progress": row}), file=sys.stderr, flush=True)
    out = {"grid": "%d^2, Ra=%g, tanh plates, dt=%.6g" % (n, Ra, dt), "tol": tol, "sampled_every": chunk,
           "seconds": round(time.perf_counter() - t0, 1)}
    for k, v in pairs.items():
        for g in v["grids"]:
            g.close()
        out[k] = {"nudge": v["delta"], "t_h_steps": v["t_h"],
                  "t_h_lower_bound": None if v["t_h"] else max(r["step"] for r in hist if "d_" + k in r),
                  "last_rel_diff": v["last"]}
    out["history"] = hist[:: max(1, len(hist) // 40)] + hist[-1:]
    return out


def main(argv=None):
    import time

    import torch

    from . import load
    import paper_1505_03271_gb300 as lb
    argv = sys.argv[1:] if argv is None else argv
    which = set(argv) or {"kol3", "poi2", "poi3"}
    load()
    for name, fn in (("kol", viscosity_error), ("poi", poiseuille_unit_dx), ("kol3", dt_max),
                     ("poi2", poiseuille_vs_n), ("poi3", poiseuille_vs_spacing), ("rb3d", rb3d),
                     ("rb3d_long", rb3d_long), ("horizon", predictability_horizon)):
        if name in which:
            t0 = time.perf_counter()
            rows = fn(lb, torch)
            print(json.dumps({"study": name, "seconds": round(time.perf_counter() - t0, 1), "rows": rows}),
                  flush=True)


if __name__ == "__main__":
    main()
