"""One FV step (Eqs. (semi), (semi-heun)) on a 4 x 5 grid recomputed in exact
rational arithmetic, independently of the oracle's C code, for the Heun
scheme and for the two single-stage schemes (the predictor alone, and
explicit Euler on plain populations, Eq. (euler)), with periodic axes,
walls, thermal plates and the fixed-density boundary: the same readings,
written out again with Python fractions from the equations, and compared with
the oracle's FP64 step.  This is a cross-check of the implementation details
(indices, ghost cells, upwind node choice, face weights, signs), not a pin of
the readings, which the other oracle tests pin.

The oracle's own face coordinates, exact binary fractions of its doubles,
define the grid, so a stretched wall-normal axis can be checked exactly."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from tests import inputs

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
W = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
INV = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def _lagrange(pos, x):
    out = []
    for k in range(3):
        num, den = Fr(1), Fr(1)
        for m in range(3):
            if m != k:
                num *= x - pos[m]
                den *= pos[k] - pos[m]
        out.append(num / den)
    return out


class Exact:
    """Rational FV step on an nx x ny grid, x periodic, y periodic or walls."""

    def __init__(self, xi_x, xi_y, walls, thermal, p):
        self.xi = [xi_x, xi_y]
        self.n = [len(xi_x) - 1, len(xi_y) - 1]
        self.walls = [False, walls]
        self.th = thermal
        self.p = p
        self.c = [[(a[i] + a[i + 1]) / 2 for i in range(len(a) - 1)] for a in self.xi]
        self.d = [[a[i + 1] - a[i] for i in range(len(a) - 1)] for a in self.xi]

    def pos(self, ax, i):
        n, c, xi = self.n[ax], self.c[ax], self.xi[ax]
        if 0 <= i < n:
            return c[i]
        if not self.walls[ax]:
            q = i // n
            return c[i - q * n] + q * (xi[n] - xi[0])
        return 2 * xi[0] - c[-i - 1] if i < 0 else 2 * xi[n] - c[2 * n - 1 - i]

    def macro(self, f, g):
        p = self.p
        rho = sum(f)
        jx = sum(CX[a] * f[a] for a in range(9))
        jy = sum(CY[a] * f[a] for a in range(9))
        T = sum(g) if self.th else Fr(0)
        ax, ay = p["ax"], p["ay"] + (p["bg"] * (T - p["T0"]) if self.th else 0)
        ux, uy = jx / rho + p["dt"] / 2 * ax, jy / rho + p["dt"] / 2 * ay
        return rho, ux, uy, T, ax, ay

    def eval(self, F, G):
        """h, h_g (dicts over cells) and Coll, Coll_g of a state."""
        p, dt = self.p, self.p["dt"]
        tt, ttg = p["tau"] + dt / 2, p["tau_g"] + dt / 2
        h, hg, co, cog = {}, {}, {}, {}
        for (i, j), f in F.items():
            g = G[(i, j)] if self.th else None
            rho, ux, uy, T, ax, ay = self.macro(f, g)
            uu = ux * ux + uy * uy
            hh, cc, hgg, cgg = [], [], [], []
            for a in range(9):
                cu = CX[a] * ux + CY[a] * uy
                feq = W[a] * rho * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu)
                fa = W[a] * rho * ((3 * (CX[a] - ux) + 9 * cu * CX[a]) * ax + (3 * (CY[a] - uy) + 9 * cu * CY[a]) * ay)
                # the plain population of Appendix A: f = f~ + dt/(2 tau + dt)(f~_eq - f~)
                # + dt/2 F, with the tilded equilibrium f~_eq = f_eq - dt/2 F (2 tau + dt = 2 tau~)
                hh.append(f[a] + dt / (2 * tt) * ((feq - dt / 2 * fa) - f[a]) + dt / 2 * fa)
                cc.append(dt / tt * (feq - f[a]) + dt * (1 - dt / (2 * tt)) * fa)
                if self.th:
                    geq = T / rho * feq
                    hgg.append(g[a] + dt / (2 * ttg) * (geq - g[a]))
                    cgg.append(dt / ttg * (geq - g[a]))
            h[(i, j)], co[(i, j)] = hh, cc
            if self.th:
                hg[(i, j)], cog[(i, j)] = hgg, cgg
        return h, hg, co, cog

    def value(self, h, a, i, j, thermal):
        """h_a at any (i, j) with at most one index outside the grid."""
        nx, ny = self.n
        if 0 <= j < ny:
            return h[(i % nx, j)][a]
        if not self.walls[1]:
            return h[(i % nx, j % ny)][a]
        k = -j if j < 0 else j - ny + 1  # ghost layer 1 or 2
        src = (i % nx, k - 1 if j < 0 else ny - k)
        v = h[src][INV[a]]
        if thermal:
            Tw = self.p["T_bot"] if j < 0 else self.p["T_top"]
            return 2 * W[a] * Tw - v
        return v

    def advect(self, h, thermal):
        nx, ny = self.n
        out = {}
        for (i, j) in h:
            res = []
            for a in range(9):
                v = Fr(0)
                for ax, cv in ((0, CX[a]), (1, CY[a])):
                    if cv == 0:
                        continue
                    m = i if ax == 0 else j
                    faces = []
                    for fc in (m, m + 1):
                        n0 = fc - 2 if cv > 0 else fc - 1
                        wts = _lagrange([self.pos(ax, n0 + k) for k in range(3)], self.xi[ax][fc])
                        nodes = [(n0 + k, j) if ax == 0 else (i, n0 + k) for k in range(3)]
                        faces.append(sum(w_ * self.value(h, a, x, y, thermal) for w_, (x, y) in zip(wts, nodes)))
                    v += cv * (faces[1] - faces[0]) / self.d[ax][m]
                res.append(v)
            out[(i, j)] = res
        return out

    def step(self, F, G):
        dt = self.p["dt"]
        h, hg, co, cog = self.eval(F, G)
        A = self.advect(h, False)
        Ag = self.advect(hg, True) if self.th else None
        Fs = {c: [F[c][a] - dt * A[c][a] + co[c][a] for a in range(9)] for c in F}
        Gs = {c: [G[c][a] - dt * Ag[c][a] + cog[c][a] for a in range(9)] for c in F} if self.th else None
        h2, hg2, _, _ = self.eval(Fs, Gs)
        A2 = self.advect(h2, False)
        Ag2 = self.advect(hg2, True) if self.th else None
        Fn = {c: [F[c][a] - dt / 2 * (A[c][a] + A2[c][a]) + co[c][a] for a in range(9)] for c in F}
        Gn = ({c: [G[c][a] - dt / 2 * (Ag[c][a] + Ag2[c][a]) + cog[c][a] for a in range(9)] for c in F}
              if self.th else None)
        return Fn, Gn


@pytest.mark.parametrize("walls,stretch,thermal", [(False, 0.0, False), (True, 1.5, False), (True, 1.5, True)])
def test_fv_step_exact(oracle, walls, stretch, thermal):
    nx, ny = 4, 5
    sy = oracle.TANH if stretch else oracle.UNIFORM
    kw = dict(tau=0.3, dt=0.25, ax=2e-3, ay=-1e-3)
    if thermal:
        kw.update(tau_g=0.2, beta=0.05, grav=1.0, T0=1.0, T_bot=1.25, T_top=0.75)
    r = oracle.RefGrid(nx, ny, ly=5.0, sy=sy, stretch_y=stretch, bcy=oracle.WALLS if walls else oracle.PERIODIC,
                       thermal=thermal).set_params(**kw)
    f = inputs.random_populations(nx, ny, seed=21, amp=0.3)
    g = inputs.random_populations(nx, ny, seed=22, amp=0.3) if thermal else None
    r.set_pops(f, g)
    xi_x, xi_y = r.face_coords()
    p = {k: Fr(v) for k, v in kw.items()}
    p.setdefault("tau_g", p["tau"])
    p["bg"] = p.get("beta", Fr(0)) * p.get("grav", Fr(0))
    ex = Exact([Fr(v) for v in xi_x], [Fr(v) for v in xi_y], walls, thermal, p)
    F = {(i, j): [Fr(f[a, j, i]) for a in range(9)] for i in range(nx) for j in range(ny)}
    G = {(i, j): [Fr(g[a, j, i]) for a in range(9)] for i in range(nx) for j in range(ny)} if thermal else None
    Fn, Gn = ex.step(F, G)
    r.step_fv(1)
    fr, gr = r.get_pops()
    ref = np.array([[[float(Fn[(i, j)][a]) for i in range(nx)] for j in range(ny)] for a in range(9)])
    assert np.abs(fr - ref).max() < 1e-14
    if thermal:
        refg = np.array([[[float(Gn[(i, j)][a]) for i in range(nx)] for j in range(ny)] for a in range(9)])
        assert np.abs(gr - refg).max() < 1e-14


class ExactSingleStage(Exact):
    """The two single-stage FV schemes of Sec. II B 2 on the same grid."""

    def semi(self, F, G):
        """Eq. (semi) alone: f~ - dt A[h] + Coll, the Heun predictor."""
        dt = self.p["dt"]
        h, hg, co, cog = self.eval(F, G)
        A = self.advect(h, False)
        Fn = {c: [F[c][a] - dt * A[c][a] + co[c][a] for a in range(9)] for c in F}
        if not self.th:
            return Fn, None
        Ag = self.advect(hg, True)
        return Fn, {c: [G[c][a] - dt * Ag[c][a] + cog[c][a] for a in range(9)] for c in F}

    def euler(self, F, G):
        """Eq. (euler) on plain populations: the advected field is f itself,
        u = sum c f / rho with no half-step shift, and the source is
        dt/tau (f_eq - f) + dt F (g: dt/tau_g (g_eq - g))."""
        p, dt = self.p, self.p["dt"]
        src, srcg = {}, {}
        for (i, j), f in F.items():
            rho = sum(f)
            T = sum(G[(i, j)]) if self.th else Fr(0)
            ax, ay = p["ax"], p["ay"] + (p["bg"] * (T - p["T0"]) if self.th else 0)
            ux = sum(CX[a] * f[a] for a in range(9)) / rho
            uy = sum(CY[a] * f[a] for a in range(9)) / rho
            uu = ux * ux + uy * uy
            s, sg = [], []
            for a in range(9):
                cu = CX[a] * ux + CY[a] * uy
                feq = W[a] * rho * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu)
                fa = W[a] * rho * ((3 * (CX[a] - ux) + 9 * cu * CX[a]) * ax + (3 * (CY[a] - uy) + 9 * cu * CY[a]) * ay)
                s.append(dt / p["tau"] * (feq - f[a]) + dt * fa)
                if self.th:
                    sg.append(dt / p["tau_g"] * (T / rho * feq - G[(i, j)][a]))
            src[(i, j)] = s
            if self.th:
                srcg[(i, j)] = sg
        A = self.advect(F, False)
        Fn = {c: [F[c][a] - dt * A[c][a] + src[c][a] for a in range(9)] for c in F}
        if not self.th:
            return Fn, None
        Ag = self.advect(G, True)
        return Fn, {c: [G[c][a] - dt * Ag[c][a] + srcg[c][a] for a in range(9)] for c in F}


@pytest.mark.parametrize("scheme", ["semi", "euler"])
@pytest.mark.parametrize("walls,stretch,thermal", [(False, 0.0, False), (True, 1.5, False), (True, 1.5, True)])
def test_fv_single_stage_steps_exact(oracle, scheme, walls, stretch, thermal):
    nx, ny = 4, 5
    sy = oracle.TANH if stretch else oracle.UNIFORM
    kw = dict(tau=0.3, dt=0.25, ax=2e-3, ay=-1e-3)
    if thermal:
        kw.update(tau_g=0.2, beta=0.05, grav=1.0, T0=1.0, T_bot=1.25, T_top=0.75)
    r = oracle.RefGrid(nx, ny, ly=5.0, sy=sy, stretch_y=stretch, bcy=oracle.WALLS if walls else oracle.PERIODIC,
                       thermal=thermal)
    r.set_scheme(oracle.FV_SEMI if scheme == "semi" else oracle.FV_EULER).set_params(**kw)
    f = inputs.random_populations(nx, ny, seed=23, amp=0.3)
    g = inputs.random_populations(nx, ny, seed=24, amp=0.3) if thermal else None
    r.set_pops(f, g)
    xi_x, xi_y = r.face_coords()
    p = {k: Fr(v) for k, v in kw.items()}
    p.setdefault("tau_g", p["tau"])
    p["bg"] = p.get("beta", Fr(0)) * p.get("grav", Fr(0))
    ex = ExactSingleStage([Fr(v) for v in xi_x], [Fr(v) for v in xi_y], walls, thermal, p)
    F = {(i, j): [Fr(f[a, j, i]) for a in range(9)] for i in range(nx) for j in range(ny)}
    G = {(i, j): [Fr(g[a, j, i]) for a in range(9)] for i in range(nx) for j in range(ny)} if thermal else None
    Fn, Gn = ex.semi(F, G) if scheme == "semi" else ex.euler(F, G)
    r.step_fv(1)
    fr, gr = r.get_pops()
    ref = np.array([[[float(Fn[(i, j)][a]) for i in range(nx)] for j in range(ny)] for a in range(9)])
    assert np.abs(fr - ref).max() < 1e-14
    if thermal:
        refg = np.array([[[float(Gn[(i, j)][a]) for i in range(nx)] for j in range(ny)] for a in range(9)])
        assert np.abs(gr - refg).max() < 1e-14


class ExactBC(ExactSingleStage):
    """The same steps with each axis periodic, walls, or a fixed-density
    boundary (Sec. II B 5): a density ghost takes the same population of the
    node it mirrors, scaled by rho_g / rho_k with rho_g = 2 rho_S - rho_k (the
    face lies midway between the two centres)."""

    def __init__(self, xi_x, xi_y, kinds, rho_bc, p):
        super().__init__(xi_x, xi_y, False, False, p)
        self.kinds = kinds
        self.walls = [k != "periodic" for k in kinds]  # ghost centres are mirrored
        self.rho_bc = rho_bc

    def value(self, h, a, i, j, thermal):
        idx = [i, j]
        for ax in (0, 1):
            n, t = self.n[ax], idx[ax]
            if 0 <= t < n:
                continue
            if self.kinds[ax] == "periodic":
                idx[ax] = t % n
                return h[tuple(idx)][a]
            k = -t if t < 0 else t - n + 1
            idx[ax] = k - 1 if t < 0 else n - k
            src = h[tuple(idx)]
            if self.kinds[ax] == "walls":
                return src[INV[a]]
            rho_s = self.rho_bc[ax][0 if t < 0 else 1]
            rho_k = sum(src)
            return (2 * rho_s - rho_k) / rho_k * src[a]
        return h[(i, j)][a]


@pytest.mark.parametrize("scheme", ["heun", "semi", "euler"])
@pytest.mark.parametrize("kinds,stretch", [(("density", "periodic"), (1.5, 0.0)),
                                           (("periodic", "density"), (0.0, 0.0)),
                                           (("density", "walls"), (0.0, 1.5))],
                         ids=["x-density-tanh", "y-density", "x-density-y-walls"])
def test_fv_density_boundary_step_exact(oracle, scheme, kinds, stretch):
    nx, ny = 5, 4
    code = {"periodic": oracle.PERIODIC, "walls": oracle.WALLS, "density": oracle.DENSITY}
    sp = [oracle.TANH if s else oracle.UNIFORM for s in stretch]
    kw = dict(tau=0.3, dt=0.25, ax=2e-3, ay=-1e-3)
    r = oracle.RefGrid(nx, ny, lx=5.0, ly=4.0, sx=sp[0], sy=sp[1], stretch_x=stretch[0], stretch_y=stretch[1],
                       bcx=code[kinds[0]], bcy=code[kinds[1]])
    r.set_scheme({"heun": oracle.FV_HEUN, "semi": oracle.FV_SEMI, "euler": oracle.FV_EULER}[scheme])
    r.set_params(**kw).set_boundary_density(rho_x0=1.03, rho_x1=0.98, rho_y0=1.01, rho_y1=0.97)
    f = inputs.random_populations(nx, ny, seed=25, amp=0.3)
    r.set_pops(f)
    xi_x, xi_y = r.face_coords()
    p = {k: Fr(v) for k, v in kw.items()}
    p["tau_g"], p["bg"] = p["tau"], Fr(0)
    rho_bc = [(Fr(1.03), Fr(0.98)), (Fr(1.01), Fr(0.97))]
    ex = ExactBC([Fr(v) for v in xi_x], [Fr(v) for v in xi_y], kinds, rho_bc, p)
    F = {(i, j): [Fr(f[a, j, i]) for a in range(9)] for i in range(nx) for j in range(ny)}
    Fn = {"heun": ex.step, "semi": ex.semi, "euler": ex.euler}[scheme](F, None)[0]
    r.step_fv(1)
    fr = r.get_pops()[0]
    ref = np.array([[[float(Fn[(i, j)][a]) for i in range(nx)] for j in range(ny)] for a in range(9)])
    assert np.abs(fr - ref).max() < 1e-14
