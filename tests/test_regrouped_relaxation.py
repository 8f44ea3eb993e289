"""The regrouped relaxation the paired kernels compute (collide_units and
PairMom::relax_f), checked as an identity against the BGK update with the
Guo force written term by term (Sec. II A, Eq. (F2)), in exact rational
arithmetic on D2Q9:

    d_a + k1 (feq_a - f_a) + k2 F_a
      = (1 - k1) d_a + k1 w_a rho' + w_a rho (S +- D),

with d = f - w rho_r the stored deviation, rho' = sum d = rho - rho_r,
cu3 = 3 c_a.u, t = 3 c_a.a, C0 = k1 (-1.5 u.u) + k2 (-3 u.a),
g = (k1/2) cu3 + k2 t, S = cu3 g + C0, D = g + (k1/2) cu3, the sign + for a
and - for the opposite population.  The GPU parity tests check the kernels;
this pins the algebra they share, so that a dropped term or a wrong sign in
the derivation fails here without a GPU."""
from fractions import Fraction as Fr
import random

import pytest

C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
INV = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def textbook(f, rho_r, k1, k2, ax, ay, hf):
    """d_a + k1 (feq_a - f_a) + k2 F_a with f_eq and F written out."""
    rho = sum(f)
    ux = sum(c[0] * x for c, x in zip(C, f)) / rho + hf * ax
    uy = sum(c[1] * x for c, x in zip(C, f)) / rho + hf * ay
    out = []
    for a, (cx, cy) in enumerate(C):
        cu = cx * ux + cy * uy
        uu = ux * ux + uy * uy
        ca = cx * ax + cy * ay
        ua = ux * ax + uy * ay
        feq = W[a] * rho * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu)
        F = W[a] * rho * (3 * (ca - ua) + 9 * cu * ca)
        out.append(f[a] - W[a] * rho_r + k1 * (feq - f[a]) + k2 * F)
    return out


def regrouped(f, rho_r, k1, k2, ax, ay, hf):
    """The same from the stored deviations, per pair of opposite populations."""
    d = [x - w * rho_r for x, w in zip(f, W)]
    rp = sum(d)
    rho = rp + rho_r
    ux = sum(c[0] * x for c, x in zip(C, d)) / rho + hf * ax
    uy = sum(c[1] * x for c, x in zip(C, d)) / rho + hf * ay
    C0 = k1 * Fr(-3, 2) * (ux * ux + uy * uy) + k2 * (-3) * (ux * ax + uy * ay)
    out = [None] * 9
    out[0] = (1 - k1) * d[0] + k1 * W[0] * rp + W[0] * rho * C0
    for a in (1, 2, 5, 6):
        b = INV[a]
        cx, cy = C[a]
        cu3 = 3 * (cx * ux + cy * uy)
        t = 3 * (cx * ax + cy * ay)
        g = k1 / 2 * cu3 + k2 * t
        S = cu3 * g + C0
        D = g + k1 / 2 * cu3
        out[a] = (1 - k1) * d[a] + k1 * W[a] * rp + W[a] * rho * (S + D)
        out[b] = (1 - k1) * d[b] + k1 * W[b] * rp + W[b] * rho * (S - D)
    return out


def _rand(rng, scale):
    return Fr(rng.randint(-1000, 1000), 1000) * scale


@pytest.mark.parametrize("seed", range(6))
def test_regrouped_relaxation_is_the_bgk_guo_update(seed):
    rng = random.Random(seed)
    # populations near a base state rho_r (1 on flow grids, barometric rows otherwise)
    rho_r = 1 + _rand(rng, Fr(1, 10))
    f = [w * rho_r + _rand(rng, Fr(1, 20)) for w in W]
    ax, ay = _rand(rng, Fr(1, 100)), _rand(rng, Fr(1, 100))
    # (k1, k2): the ST / f~ + Coll pair (om, 1 - om/2) and the advected-field pair (om/2, its force part)
    om = Fr(rng.randint(200, 1900), 1000)
    for k1, k2 in ((om, 1 - om / 2), (om / 2, Fr(1, 2) * (1 - om / 2))):
        assert regrouped(f, rho_r, k1, k2, ax, ay, Fr(1, 2)) == textbook(f, rho_r, k1, k2, ax, ay, Fr(1, 2))


def test_a_dropped_term_is_seen():
    """The identity is tight: dropping the odd part's force term breaks it."""
    rng = random.Random(7)
    f = [w + _rand(rng, Fr(1, 20)) for w in W]
    ax, ay, om = Fr(1, 300), Fr(-1, 500), Fr(3, 2)
    k1, k2 = om, 1 - om / 2
    good = textbook(f, Fr(1), k1, k2, ax, ay, Fr(1, 2))
    assert regrouped(f, Fr(1), k1, k2, ax, ay, Fr(1, 2)) == good
    assert regrouped(f, Fr(1), k1, 0, ax, ay, Fr(1, 2)) != good
