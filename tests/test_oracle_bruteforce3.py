"""One D3Q19 FV step (Eqs. (semi), (semi-heun); QUICK faces of Sec. II B 3 on
each axis line; double-reflection walls of Sec. II B 5, the thermal field
anti-reflected at the plates) recomputed in exact rational arithmetic from
the equations, independently of the oracle's C code, and compared with the
oracle's FP64 step on small grids with all three axes active at once.

The projection tests of test_oracle_3d.py pin the 3-D oracle through the
2-D one, two axes at a time; this check reaches what they cannot: a state
that varies along all three axes, walls on two axes of one grid, and the
velocity order of include/lb3.h.  The oracle's own face coordinates (exact
binary fractions of its doubles) define the stretched axes."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from tests import inputs

# include/lb3.h: 0 rest; 1, 2 = +-x; 3, 4 = +-y; 5, 6 = +-z; then the edge
# velocities in opposite pairs (xy, xz, yz planes)
C3 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
      (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
      (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
W3 = [Fr(1, 3)] + [Fr(1, 18)] * 6 + [Fr(1, 36)] * 12
INV3 = [C3.index(tuple(-v for v in c)) for c in C3]


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


class Exact3:
    """Rational FV step on an nx x ny x nz grid; each axis periodic or walls."""

    def __init__(self, xi, walls, thermal, p):
        self.xi = xi                                   # face coordinates per axis
        self.n = [len(a) - 1 for a in xi]
        self.walls = walls
        self.th = thermal
        self.p = p
        self.c = [[(a[i] + a[i + 1]) / 2 for i in range(len(a) - 1)] for a in xi]
        self.d = [[a[i + 1] - a[i] for i in range(len(a) - 1)] for a in xi]

    def pos(self, ax, i):
        """Centre of cell index i on an axis: a fluid cell, a periodic image or
        a ghost mirrored about the wall face."""
        n, c, xi = self.n[ax], self.c[ax], self.xi[ax]
        if 0 <= i < n:
            return c[i]
        if not self.walls[ax]:
            q = i // n
            return c[i - q * n] + q * (xi[n] - xi[0])
        return 2 * xi[0] - c[-i - 1] if i < 0 else 2 * xi[n] - c[2 * n - 1 - i]

    def eval(self, F, G):
        p, dt = self.p, self.p["dt"]
        tt, ttg = p["tau"] + dt / 2, p["tau_g"] + dt / 2
        h, hg, co, cog = {}, {}, {}, {}
        for cell, f in F.items():
            rho = sum(f)
            j = [sum(C3[a][x] * f[a] for a in range(19)) for x in range(3)]
            T = sum(G[cell]) if self.th else Fr(0)
            acc = [p["ax"], p["ay"], p["az"] + (p["bg"] * (T - p["T0"]) if self.th else 0)]
            u = [j[x] / rho + dt / 2 * acc[x] for x in range(3)]
            uu = sum(v * v for v in u)
            ua = sum(u[x] * acc[x] for x in range(3))
            hh, cc, hgg, cgg = [], [], [], []
            for a in range(19):
                cu = sum(C3[a][x] * u[x] for x in range(3))
                ca = sum(C3[a][x] * acc[x] for x in range(3))
                feq = W3[a] * rho * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu)
                fa = W3[a] * rho * (3 * (ca - ua) + 9 * cu * ca)
                # the plain population of Appendix A: f = f~ + dt/(2 tau + dt)(f~_eq - f~)
                # + dt/2 F, with the tilded equilibrium f~_eq = f_eq - dt/2 F (2 tau + dt = 2 tau~)
                hh.append(f[a] + dt / (2 * tt) * ((feq - dt / 2 * fa) - f[a]) + dt / 2 * fa)
                cc.append(dt / tt * (feq - f[a]) + dt * (1 - dt / (2 * tt)) * fa)
                if self.th:
                    g = G[cell][a]
                    geq = T / rho * feq
                    hgg.append(g + dt / (2 * ttg) * (geq - g))
                    cgg.append(dt / ttg * (geq - g))
            h[cell], co[cell] = hh, cc
            if self.th:
                hg[cell], cog[cell] = hgg, cgg
        return h, hg, co, cog

    def value(self, h, a, idx, thermal):
        """h_a at a cell index with at most one coordinate outside the grid."""
        idx = list(idx)
        for ax in range(3):
            n = self.n[ax]
            if 0 <= idx[ax] < n:
                continue
            if not self.walls[ax]:
                idx[ax] %= n
                return h[tuple(idx)][a]
            lo = idx[ax] < 0
            idx[ax] = -idx[ax] - 1 if lo else 2 * n - 1 - idx[ax]
            v = h[tuple(idx)][INV3[a]]
            if thermal:
                Tw = self.p["T_bot"] if lo else self.p["T_top"]
                return 2 * W3[a] * Tw - v
            return v
        return h[tuple(idx)][a]

    def advect(self, h, thermal):
        out = {}
        for cell in h:
            res = []
            for a in range(19):
                v = Fr(0)
                for ax in range(3):
                    cv = C3[a][ax]
                    if cv == 0:
                        continue
                    m = cell[ax]
                    phi = []
                    for fc in (m, m + 1):
                        n0 = fc - 2 if cv > 0 else fc - 1
                        wts = _lagrange([self.pos(ax, n0 + k) for k in range(3)], self.xi[ax][fc])
                        s = Fr(0)
                        for k in range(3):
                            idx = list(cell)
                            idx[ax] = n0 + k
                            s += wts[k] * self.value(h, a, idx, thermal)
                        phi.append(s)
                    v += cv * (phi[1] - phi[0]) / self.d[ax][m]
                res.append(v)
            out[cell] = res
        return out

    def step(self, F, G):
        dt = self.p["dt"]
        h, hg, co, cog = self.eval(F, G)
        A = self.advect(h, False)
        Ag = self.advect(hg, True) if self.th else None
        Fs = {c: [F[c][a] - dt * A[c][a] + co[c][a] for a in range(19)] for c in F}
        Gs = {c: [G[c][a] - dt * Ag[c][a] + cog[c][a] for a in range(19)] for c in F} if self.th else None
        h2, hg2, _, _ = self.eval(Fs, Gs)
        A2 = self.advect(h2, False)
        Ag2 = self.advect(hg2, True) if self.th else None
        Fn = {c: [F[c][a] - dt / 2 * (A[c][a] + A2[c][a]) + co[c][a] for a in range(19)] for c in F}
        Gn = ({c: [G[c][a] - dt / 2 * (Ag[c][a] + Ag2[c][a]) + cog[c][a] for a in range(19)] for c in F}
              if self.th else None)
        return Fn, Gn


def test_lattice_order_matches_header(oracle):
    cx, cy, cz, w, inv = oracle.lattice3()
    assert [tuple(v) for v in zip(cx, cy, cz)] == C3
    assert np.array_equal(w, np.array([float(x) for x in W3]))
    assert list(inv) == INV3


CASES = [
    # flow: x periodic, walls on y (tanh) and z (sinh), a body force along all three axes
    dict(n=(3, 4, 4), L=(3.0, 4.0, 4.0), sp=("UNIFORM", "TANH", "SINH"), st=(0.0, 1.5, 3.0),
         walls=(False, True, True), thermal=False),
    # flow: walls on x only, stretched x, periodic y and z
    dict(n=(4, 3, 3), L=(4.0, 3.0, 3.0), sp=("TANH", "UNIFORM", "UNIFORM"), st=(1.2, 0.0, 0.0),
         walls=(True, False, False), thermal=False),
    # thermal: x and y periodic, plates on a sinh z grid, buoyancy along z
    dict(n=(3, 3, 4), L=(3.0, 3.0, 4.0), sp=("UNIFORM", "UNIFORM", "SINH"), st=(0.0, 0.0, 3.0),
         walls=(False, False, True), thermal=True),
]


@pytest.mark.parametrize("case", CASES, ids=["flow-yz-walls", "flow-x-walls", "thermal-plates"])
def test_fv3_step_exact(oracle, case):
    nx, ny, nz = case["n"]
    th = case["thermal"]
    sp = [getattr(oracle, s) for s in case["sp"]]
    kw = dict(tau=0.3, dt=0.25, ax=2e-3, ay=-1e-3, az=1.5e-3)
    if th:
        kw.update(tau_g=0.2, beta=0.05, grav=1.0, T0=1.0, T_bot=1.25, T_top=0.75)
    bc = [oracle.WALLS if w else oracle.PERIODIC for w in case["walls"]]
    r = oracle.RefGrid3(nx, ny, nz, lx=case["L"][0], ly=case["L"][1], lz=case["L"][2], sx=sp[0], sy=sp[1],
                        sz=sp[2], stretch_x=case["st"][0], stretch_y=case["st"][1], stretch_z=case["st"][2],
                        bcx=bc[0], bcy=bc[1], bcz=bc[2], thermal=th).set_params(**kw)
    f = inputs.random_populations3(nx, ny, nz, seed=31, amp=0.3)
    g = inputs.random_populations3(nx, ny, nz, seed=32, amp=0.3) if th else None
    r.set_pops(f, g)
    xi = [[Fr(v) for v in oracle.faces(n, L, s, t)] for n, L, s, t in zip(case["n"], case["L"], sp, case["st"])]
    p = {k: Fr(v) for k, v in kw.items()}
    p.setdefault("tau_g", p["tau"])
    p["bg"] = p.get("beta", Fr(0)) * p.get("grav", Fr(0))
    ex = Exact3(xi, case["walls"], th, p)
    cells = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    F = {c: [Fr(f[a, c[2], c[1], c[0]]) for a in range(19)] for c in cells}
    G = {c: [Fr(g[a, c[2], c[1], c[0]]) for a in range(19)] for c in cells} if th else None
    Fn, Gn = ex.step(F, G)
    r.step_fv(1)
    fr, gr = r.get_pops()
    ref = np.zeros((19, nz, ny, nx))
    for (i, j, k), v in Fn.items():
        ref[:, k, j, i] = [float(x) for x in v]
    assert np.abs(fr - ref).max() < 1e-14
    if th:
        refg = np.zeros((19, nz, ny, nx))
        for (i, j, k), v in Gn.items():
            refg[:, k, j, i] = [float(x) for x in v]
        assert np.abs(gr - refg).max() < 1e-14
