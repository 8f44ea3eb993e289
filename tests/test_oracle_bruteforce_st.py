"""ST steps (Eq. (ST) at dt = dx = 1) recomputed in exact rational
arithmetic from the equation, independently of the oracle's C code, and
compared with the oracle's FP64 steps, for D2Q9 and D3Q19.

Each cell collides (BGK relaxation with tau~ = tau + 1/2 toward f_eq(rho, u)
at the force-corrected velocity, plus (1 - 1/(2 tau~)) times the Guo force of
Eq. (F2); g relaxes with tau_g~ toward (T/rho) f_eq) and pushes every
population to the neighbour c_a away.  A population that would leave through
a wall comes back to its own cell reversed (half-way bounce-back); the
thermal one comes back as 2 w_a T_wall minus itself (anti-bounce-back, the
isothermal plate).  The states vary along every axis, so a wrong neighbour
offset, a transposed velocity component or a wrong wall rule in any plane
shows up; the 3-D cases reach the xz-plane edge velocities, which the
projection tests onto the 2-D oracle cannot."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from tests import inputs

# include/lb.h order: rest; +x, +y, -x, -y; then the diagonals
C2 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W2 = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
# include/lb3.h order: rest; +-x, +-y, +-z; then the edges in opposite pairs
C3 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
      (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
      (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
W3 = [Fr(1, 3)] + [Fr(1, 18)] * 6 + [Fr(1, 36)] * 12


def st_step(F, G, n, walls, C, W, p):
    """One exact ST step.  F, G: dicts cell -> populations; the last axis
    carries gravity and, where it has walls, the plates (T_bot below)."""
    Q, D = len(C), len(n)
    inv = [C.index(tuple(-v for v in c)) for c in C]
    tt, ttg = p["tau"] + Fr(1, 2), p["tau_g"] + Fr(1, 2)
    th = G is not None
    Fn = {c: [None] * Q for c in F}
    Gn = {c: [None] * Q for c in F} if th else None
    for cell, f in F.items():
        rho = sum(f)
        T = sum(G[cell]) if th else Fr(0)
        acc = list(p["a"])
        if th:
            acc[-1] += p["bg"] * (T - p["T0"])
        u = [sum(C[a][x] * f[a] for a in range(Q)) / rho + acc[x] / 2 for x in range(D)]
        uu = sum(v * v for v in u)
        ua = sum(u[x] * acc[x] for x in range(D))
        for a in range(Q):
            cu = sum(C[a][x] * u[x] for x in range(D))
            ca = sum(C[a][x] * acc[x] for x in range(D))
            feq = W[a] * rho * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu)
            force = W[a] * rho * (3 * (ca - ua) + 9 * cu * ca)
            post = f[a] + (feq - f[a]) / tt + (1 - 1 / (2 * tt)) * force
            gpost = G[cell][a] + (T / rho * feq - G[cell][a]) / ttg if th else None
            dest, wall_T, out = [], None, False
            for x in range(D):
                t = cell[x] + C[a][x]
                if 0 <= t < n[x]:
                    dest.append(t)
                elif not walls[x]:
                    dest.append(t % n[x])
                else:
                    out = True
                    if th and x == D - 1:
                        wall_T = p["T_bot"] if t < 0 else p["T_top"]
                    dest.append(cell[x])
            if out:
                Fn[cell][inv[a]] = post
                if th:
                    Gn[cell][inv[a]] = -gpost + 2 * W[a] * wall_T
            else:
                Fn[tuple(dest)][a] = post
                if th:
                    Gn[tuple(dest)][a] = gpost
    return Fn, Gn


def _params(kw, D):
    p = {k: Fr(v) for k, v in kw.items() if k not in ("ax", "ay", "az")}
    p["a"] = [Fr(kw.get(k, 0.0)) for k in ("ax", "ay", "az")[:D]]
    p.setdefault("tau_g", p["tau"])
    p["bg"] = p.get("beta", Fr(0)) * p.get("grav", Fr(0))
    return p


def test_lattice_orders(oracle):
    cx, cy, w, inv = oracle.lattice()
    assert [tuple(v) for v in zip(cx, cy)] == C2
    assert np.array_equal(w, np.array([float(x) for x in W2]))
    cx, cy, cz, w, inv = oracle.lattice3()
    assert [tuple(v) for v in zip(cx, cy, cz)] == C3


CASES2 = [
    dict(n=(5, 4), walls=(False, False), thermal=False),
    dict(n=(4, 5), walls=(False, True), thermal=False),
    dict(n=(4, 3), walls=(True, True), thermal=False),   # a closed box: corners bounce both ways
    dict(n=(4, 5), walls=(False, True), thermal=True),
]


@pytest.mark.parametrize("case", CASES2, ids=["periodic", "y-walls", "box", "thermal-plates"])
def test_st2_steps_exact(oracle, case):
    (nx, ny), walls, th = case["n"], case["walls"], case["thermal"]
    kw = dict(tau=0.3, dt=1.0, ax=2e-3, ay=-1e-3)
    if th:
        kw.update(tau_g=0.2, beta=0.05, grav=1.0, T0=1.0, T_bot=1.25, T_top=0.75)
    bc = [oracle.WALLS if w else oracle.PERIODIC for w in walls]
    r = oracle.RefGrid(nx, ny, bcx=bc[0], bcy=bc[1], thermal=th).set_params(**kw)
    f = inputs.random_populations(nx, ny, seed=41, amp=0.3)
    g = inputs.random_populations(nx, ny, seed=42, amp=0.3) if th else None
    r.set_pops(f, g)
    kw.pop("dt")
    p = _params(kw, 2)
    F = {(i, j): [Fr(f[a, j, i]) for a in range(9)] for j in range(ny) for i in range(nx)}
    G = {(i, j): [Fr(g[a, j, i]) for a in range(9)] for j in range(ny) for i in range(nx)} if th else None
    for _ in range(2):
        F, G = st_step(F, G, (nx, ny), walls, C2, W2, p)
    r.step_st(2)
    fr, gr = r.get_pops()
    ref = np.array([[[float(F[(i, j)][a]) for i in range(nx)] for j in range(ny)] for a in range(9)])
    assert np.abs(fr - ref).max() < 1e-14
    if th:
        refg = np.array([[[float(G[(i, j)][a]) for i in range(nx)] for j in range(ny)] for a in range(9)])
        assert np.abs(gr - refg).max() < 1e-14


CASES3 = [
    dict(n=(3, 4, 3), walls=(False, False, False), thermal=False),
    dict(n=(3, 4, 4), walls=(False, True, True), thermal=False),
    dict(n=(4, 3, 3), walls=(True, False, False), thermal=False),
    dict(n=(3, 3, 4), walls=(False, False, True), thermal=True),
]


@pytest.mark.parametrize("case", CASES3, ids=["periodic", "yz-walls", "x-walls", "thermal-plates"])
def test_st3_step_exact(oracle, case):
    (nx, ny, nz), walls, th = case["n"], case["walls"], case["thermal"]
    kw = dict(tau=0.3, dt=1.0, ax=2e-3, ay=-1e-3, az=1.5e-3)
    if th:
        kw.update(tau_g=0.2, beta=0.05, grav=1.0, T0=1.0, T_bot=1.25, T_top=0.75)
    bc = [oracle.WALLS if w else oracle.PERIODIC for w in walls]
    r = oracle.RefGrid3(nx, ny, nz, bcx=bc[0], bcy=bc[1], bcz=bc[2], thermal=th).set_params(**kw)
    f = inputs.random_populations3(nx, ny, nz, seed=43, amp=0.3)
    g = inputs.random_populations3(nx, ny, nz, seed=44, amp=0.3) if th else None
    r.set_pops(f, g)
    kw.pop("dt")
    p = _params(kw, 3)
    cells = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    F = {c: [Fr(f[a, c[2], c[1], c[0]]) for a in range(19)] for c in cells}
    G = {c: [Fr(g[a, c[2], c[1], c[0]]) for a in range(19)] for c in cells} if th else None
    F, G = st_step(F, G, (nx, ny, nz), walls, C3, W3, p)
    r.step_st(1)
    fr, gr = r.get_pops()
    ref = np.zeros((19, nz, ny, nx))
    for (i, j, k), v in F.items():
        ref[:, k, j, i] = [float(x) for x in v]
    assert np.abs(fr - ref).max() < 1e-14
    if th:
        refg = np.zeros((19, nz, ny, nx))
        for (i, j, k), v in G.items():
            refg[:, k, j, i] = [float(x) for x in v]
        assert np.abs(gr - refg).max() < 1e-14
