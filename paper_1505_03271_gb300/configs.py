"""Parameter rules and the synthetic workloads (host logic only).

Conventions (readings of the paper listed in the design notes):
  * ``tau`` handed to the library is the physical relaxation time,
    nu = tau c_s^2 (Sec. II).  The lattice relaxation time of the streaming
    scheme at dt = 1 is tau~ = tau + 1/2, so a quoted "tau = 0.8" of an ST
    run means tau = 0.3 here.
  * FV time step on a stretched grid: dt = 0.9 min(dx_min, 8 tau); the paper
    gives the stability limit only at dx = 1 (Sec. III C).
  * Rayleigh-Benard: free-fall velocity U = sqrt(beta g dT H) = 0.1 (the LB
    rule of thumb of Sec. IV), Ra = beta g dT H^3 / (nu kappa), Pr = nu/kappa,
    dT = 1 with plates at T0 +- 1/2 and T0 = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import (LB_AXIS_CHEB, LB_AXIS_SINH, LB_AXIS_TANH, LB_AXIS_UNIFORM, LB_BC_PERIODIC, LB_BC_WALLS, LB_INIT_POISEUILLE,
               LB_INIT_RB, LB_INIT_TGV, LB_STORE_F16DEV, LB_STORE_F32, LB_STORE_F64)

CS2 = 1.0 / 3.0


def tau_from_st_tau(tau_tilde_st: float) -> float:
    """Physical tau from the ST relaxation time at dt = 1 (tau~ = tau + 1/2)."""
    return tau_tilde_st - 0.5


def faces(n: int, L: float, spacing: int, stretch: float) -> np.ndarray:
    """Face coordinates of Eq. (grids), as the library builds them: uniform;
    tanh with delta = stretch; sinh with s2 = stretch (even n); Chebyshev
    xi_i = L/2 (1 - cos(i pi / n))."""
    i = np.arange(n + 1)
    if spacing == LB_AXIS_TANH:
        xi = 0.5 * L * (1.0 + np.tanh((2.0 * i / n - 1.0) * stretch) / np.tanh(stretch))
    elif spacing == LB_AXIS_SINH:
        amp = 0.5 * L / np.sinh(0.5 * stretch)
        xi = np.where(2 * i <= n, amp * np.sinh(stretch * i / n), L - amp * np.sinh(stretch * (n - i) / n))
    elif spacing == LB_AXIS_CHEB:
        xi = 0.5 * L * (1.0 - np.cos(np.pi * i / n))
    else:
        xi = L * i / n
    xi[0], xi[-1] = 0.0, L
    return xi


def min_cell(n: int, L: float, spacing: int, stretch: float) -> float:
    return float(np.diff(faces(n, L, spacing, stretch)).min())


def fv_dt(dx_min: float, tau: float, safety: float = 0.9) -> float:
    return safety * min(dx_min, 8.0 * tau)


@dataclass
class RBParams:
    tau: float
    tau_g: float
    beta: float
    grav: float
    T0: float
    T_bot: float
    T_top: float

    @property
    def nu(self):
        return self.tau * CS2

    @property
    def kappa(self):
        return self.tau_g * CS2


def rb_params(Ra: float, Pr: float, H: float, U_ff: float = 0.1, T0: float = 1.0,
              dT: float = 1.0, grav: float = 1.0) -> RBParams:
    """nu = U H sqrt(Pr/Ra), kappa = nu / Pr, beta g dT = U^2 / H."""
    nu = U_ff * H * math.sqrt(Pr / Ra)
    kappa = nu / Pr
    beta = U_ff**2 / (H * dT * grav)
    return RBParams(tau=nu / CS2, tau_g=kappa / CS2, beta=beta, grav=grav, T0=T0,
                    T_bot=T0 + 0.5 * dT, T_top=T0 - 0.5 * dT)


def rayleigh(p: RBParams, H: float) -> float:
    return p.beta * p.grav * (p.T_bot - p.T_top) * H**3 / (p.nu * p.kappa)


@dataclass
class Workload:
    """A grid description plus parameters and an initial condition."""
    name: str
    grid: dict
    params: dict
    init: dict
    steps: int
    scheme: str
    notes: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.grid["nx"] * self.grid["ny"] * self.grid.get("nz", 1)


def tgv64(scheme: str = "st") -> Workload:
    """64x64 periodic TGV, FP64, quoted tau = 0.8 (tau = 0.3), u0 = 0.01,
    t = 1000 (ST: dt = 1; FV: dt = 0.5, stable in 2-D at this tau)."""
    dt = 1.0 if scheme == "st" else 0.5
    return Workload("tgv64_" + scheme,
                    dict(nx=64, ny=64, store=LB_STORE_F64),
                    dict(tau=tau_from_st_tau(0.8), dt=dt),
                    dict(kind=LB_INIT_TGV, u0=0.01), int(round(1000 / dt)), scheme)


def channel(u_max: float | None = None, store: int = LB_STORE_F32, nx: int = 256,
            ny: int = 512, steps: int = 20000) -> Workload:
    """Body-force channel, 256 x 512, walls on y with tanh delta = 2, quoted
    tau = 0.7 (tau = 0.2, nu = 1/15), a_x = 8 nu U / L^2, started on the
    parabola.  Default U from Re = 10 (Sec. III B)."""
    tau = tau_from_st_tau(0.7)
    nu = tau * CS2
    L = float(ny)
    U = u_max if u_max is not None else 10.0 * nu / L
    dt = fv_dt(min_cell(ny, L, LB_AXIS_TANH, 2.0), tau)
    return Workload("channel_%dx%d" % (nx, ny),
                    dict(nx=nx, ny=ny, lx=float(nx), ly=L, sy=LB_AXIS_TANH, stretch_y=2.0,
                         bcy=LB_BC_WALLS, store=store),
                    dict(tau=tau, dt=dt, ax=8.0 * nu * U / L**2),
                    dict(kind=LB_INIT_POISEUILLE, u0=U), steps, "fv", dict(U=U, Re=U * L / nu))


def rayleigh_benard(n: int = 1024, Ra: float = 1e8, Pr: float = 1.0, store: int = LB_STORE_F16DEV,
                    steps: int = 2000, seed: int = 1234, amp: float = 1e-3) -> Workload:
    """Square RB cell, x periodic uniform, plates on y with tanh delta = 2."""
    H = float(n)
    p = rb_params(Ra, Pr, H)
    dt = fv_dt(min_cell(n, H, LB_AXIS_TANH, 2.0), min(p.tau, p.tau_g))
    return Workload("rb%d_Ra%.0e" % (n, Ra),
                    dict(nx=n, ny=n, lx=H, ly=H, sy=LB_AXIS_TANH, stretch_y=2.0, bcy=LB_BC_WALLS,
                         thermal=True, store=store),
                    dict(tau=p.tau, dt=dt, tau_g=p.tau_g, beta=p.beta, grav=p.grav, T0=p.T0,
                         T_bot=p.T_bot, T_top=p.T_top),
                    dict(kind=LB_INIT_RB, amp=amp, seed=seed), steps, "fv")


def rb3d_table(scheme: str = "fv", store: int = LB_STORE_F32, steps: int = 20, seed: int = 1234,
               amp: float = 1e-3) -> Workload:
    """The 3-D Rayleigh-Benard runs of Table rb (Sec. IV): Ra = 2.5e6, Pr = 1,
    aspect ratio 2 on 128 x 128 x 64 cells, x and y periodic, plates on z.
    FV: H = 640, L = 1280, dt = 4, tau = tau_g = 0.5, beta = 1.325e-4, sinh
    z grid with s2 = 4 (the paper gives no 3-D stretching; its 2-D s2 = 6.5
    makes the wall cell 2.5 and dt = 4 diverges, s2 = 3..5 are stable).  ST: H = 64, L = 128,
    dt = 1, tau = tau_g = 0.05, beta = 1.325e-3, uniform.  dT = 2, g = 1,
    plates at T0 +- 1 with T0 = 2 (only beta g dT enters).  Conductive,
    barometric start with a seeded 1e-3 dT perturbation."""
    fv = scheme == "fv"
    H, L = (640.0, 1280.0) if fv else (64.0, 128.0)
    grid = dict(nx=128, ny=128, nz=64, lx=L, ly=L, lz=H, bcz=LB_BC_WALLS, thermal=True, store=store)
    if fv:
        grid.update(sz=LB_AXIS_SINH, stretch_z=4.0)
    tau = 0.5 if fv else 0.05
    params = dict(tau=tau, tau_g=tau, dt=4.0 if fv else 1.0, beta=1.325e-4 if fv else 1.325e-3, grav=1.0,
                  T0=2.0, T_bot=3.0, T_top=1.0)
    return Workload("rb3d_%s_128x128x64" % scheme, grid, params, dict(kind=LB_INIT_RB, amp=amp, seed=seed),
                    steps, scheme, dict(Ra=params["beta"] * 2.0 * H**3 / (tau * CS2) ** 2))


def st_sweep(n: int = 8192, store: int = LB_STORE_F32, steps: int = 500) -> Workload:
    """Periodic n x n ST: TGV mode 1 (u0 = 0.01) plus shear wave mode 2 (0.01),
    quoted tau = 0.8."""
    return Workload("st%d" % n, dict(nx=n, ny=n, store=store),
                    dict(tau=tau_from_st_tau(0.8), dt=1.0),
                    dict(kind=LB_INIT_TGV, u0=0.01, amp=0.01, mode=2), steps, "st")


def flops_per_cell(scheme: str, thermal: bool) -> int:
    """Algorithmic FP32 operations per cell update (an FMA counts 2), from
    the formulas the step evaluates, each shared subexpression once and
    each QUICK face once (a face belongs to two cells).  Halo recomputation
    in the kernels is not counted.

    Per evaluation of the cell macro routine (Sec. II, Eq. (F2)):
      moments rho, j (18), 1/rho (1), u = j/rho + dt/2 a (4)            23
      equilibrium: u^2 (3), c.u of the diagonals (4), 1 - 1.5u^2 (2),
        w rho (3), 5 per moving population, 1 for the rest one          53
      Guo force: u.a (3), 6 per moving population, 1 for the rest one   52
      advected field h = f + dt/(2 tau~)(f_eq - f) + dt/2 F, 5 x 9       45
      f + Coll (reusing f_eq - f), 4 x 9 (only at time level n)         36
    Per flux evaluation (Eq. (fv), Sec. II B 3): 12 face values (6
    populations move in x, 6 in y) of 5 each = 60; 12 differences scaled
    by 1/dx (2 each) and 4 sums for the diagonals = 28.
    FV (Eq. (semi-heun)): 209 + 88 + 16 (predictor) + 173 + 88 + 24
    (corrector) = 598.  The thermal populations add T (8), the buoyant
    a_y (2), g_eq = (T/rho) f_eq (10), h^g (27), g + Coll_g (18) at time
    level n, the same less Coll_g at the starred level (47), two more
    flux evaluations (176) and the two updates (40): 328, so 926.
    ST (Eq. (ST)): moments, equilibrium, force and the post-collision
    value f + (f_eq - f)/tau~ + (1 - 1/(2 tau~)) F (45) = 173; thermal adds
    T, a_y, g_eq and the g collision (47): 220."""
    if scheme == "fv":
        return 926 if thermal else 598
    return 220 if thermal else 173


def fp32_peak_tflops(sms: int, sm_mhz: float) -> float:
    """Non-tensor FP32 peak: 128 FP32 lanes per SM, one FMA (2 flops) per
    lane per clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def bytes_per_cell(store: int, thermal: bool, q: int = 9) -> int:
    """Compulsory HBM bytes per cell update: every population read and
    written once (q = 9 for D2Q9, 19 for D3Q19; twice that with thermal)."""
    from . import STORE_BYTES
    return 2 * (2 * q if thermal else q) * STORE_BYTES[store]
