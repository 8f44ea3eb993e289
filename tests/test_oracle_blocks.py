"""Pins of the oracle's building blocks against facts fixed by the paper or by
the mathematics (moment identities, closed forms, published constants)."""
import os

import numpy as np
import pytest

from tests import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_lattice_isotropy(oracle):
    """D2Q9 weights and velocities: the moment identities that make the
    second-order equilibrium reproduce Navier-Stokes (Sec. II)."""
    cx, cy, w, inv = oracle.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj->ij", w, c, c), np.eye(2) / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj,ak->ijk", w, c, c, c), 0.0, atol=1e-15)
    d = np.eye(2)
    iso4 = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
            + np.einsum("il,jk->ijkl", d, d)) / 9.0
    assert np.allclose(np.einsum("a,ai,aj,ak,al->ijkl", w, c, c, c, c), iso4, atol=1e-15)
    # inv(a) reverses the velocity and keeps the weight (Sec. II B 5)
    assert np.array_equal(cx[inv], -cx) and np.array_equal(cy[inv], -cy)
    assert np.array_equal(w[inv], w) and np.array_equal(inv[inv], np.arange(9))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_equilibrium_moments(oracle, seed):
    """sum f_eq = rho, sum c f_eq = rho u, sum c c f_eq = rho (u u + I/3)."""
    rho, ux, uy = 1.0 + 0.1 * inputs.random_vector(1, seed)[0], *inputs.random_vector(2, seed + 7, -0.1, 0.1)
    cx, cy, w, _ = oracle.lattice()
    feq = oracle.equilibrium(rho, ux, uy)
    u = np.array([ux, uy])
    c = np.stack([cx, cy], 1)
    assert np.isclose(feq.sum(), rho, rtol=1e-14)
    assert np.allclose(feq @ c, rho * u, rtol=1e-13, atol=1e-16)
    P = np.einsum("a,ai,aj->ij", feq, c, c)
    assert np.allclose(P, rho * (np.outer(u, u) + np.eye(2) / 3.0), rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("seed", [4, 5])
def test_guo_force_moments(oracle, seed):
    """Eq. (F2): sum F = 0, sum c F = rho a (stated in Sec. II B 4), and Guo's
    second moment sum c c F = rho (u a + a u)."""
    rho = 1.0 + 0.1 * inputs.random_vector(1, seed)[0]
    ux, uy, ax, ay = inputs.random_vector(4, seed + 11, -0.1, 0.1)
    cx, cy, _, _ = oracle.lattice()
    c = np.stack([cx, cy], 1)
    F = oracle.guo_force(rho, ux, uy, ax, ay)
    u, a = np.array([ux, uy]), np.array([ax, ay])
    assert abs(F.sum()) < 1e-15
    assert np.allclose(F @ c, rho * a, rtol=1e-13, atol=1e-17)
    S = np.einsum("a,ai,aj->ij", F, c, c)
    assert np.allclose(S, rho * (np.outer(u, a) + np.outer(a, u)), rtol=1e-12, atol=1e-17)


def test_guo_force_reduces_to_simple_force_at_rest(oracle):
    """At u = 0, Eq. (F2) equals the simple force Eq. (F1): w c.(rho a)/c_s^2."""
    cx, cy, w, _ = oracle.lattice()
    F = oracle.guo_force(1.3, 0.0, 0.0, 0.02, -0.01)
    assert np.allclose(F, w * (cx * 0.02 + cy * -0.01) * 1.3 * 3.0, rtol=1e-14, atol=1e-18)


def test_faces_uniform_and_tanh(oracle):
    """Eq. (grids): uniform faces i L/N; the tanh grid spans [0, L], is
    symmetric, monotone, and with the paper's s1 (delta = atanh s1) its
    smallest/largest cell ratio approaches sech^2(delta) for large N."""
    assert np.allclose(oracle.faces(8, 4.0), np.arange(9) * 0.5, atol=1e-15)
    for n in (16, 512, 1024):
        xi = oracle.faces(n, 3.0, oracle.TANH, 2.0)
        assert xi[0] == 0.0 and xi[-1] == 3.0
        assert np.allclose(xi + xi[::-1], 3.0, atol=1e-12)
        assert np.all(np.diff(xi) > 0)
    d = np.diff(oracle.faces(4096, 1.0, oracle.TANH, 2.0))
    assert abs(d.min() / d.max() - 1.0 / np.cosh(2.0) ** 2) < 2e-3
    # the paper's own stretching s1 = 0.98 is delta = atanh(0.98)
    xi = oracle.faces(64, 64.0, oracle.TANH, np.arctanh(0.98))
    assert np.isclose(xi[1], 32.0 * (1 + np.tanh((2 / 64 - 1) * np.arctanh(0.98)) / 0.98), rtol=1e-12)


def test_faces_sinh(oracle):
    """Eq. (grids) sinh branches meet at L/2 for even N and mirror each other."""
    for n in (8, 64):
        xi = oracle.faces(n, 2.0, oracle.SINH, 6.5)
        assert np.isclose(xi[n // 2], 1.0, atol=1e-14)
        assert np.allclose(xi + xi[::-1], 2.0, atol=1e-13)
        assert np.all(np.diff(xi) > 0)


def test_faces_chebyshev(oracle):
    """Chebyshev faces xi_i = L/2 (1 - cos(i pi / N)) (Eq. (grids), read with
    i in place of i - 1/2 so the faces reach both walls): the cell widths
    have the closed form L sin((2i + 1) pi / (2N)) sin(pi / (2N))."""
    for n in (8, 11, 64):
        xi = oracle.faces(n, 64.0, oracle.CHEB, 0.0)
        assert xi[0] == 0.0 and xi[-1] == 64.0
        assert np.allclose(xi + xi[::-1], 64.0, atol=1e-12)
        i = np.arange(n)
        d = 64.0 * np.sin((2 * i + 1) * np.pi / (2 * n)) * np.sin(np.pi / (2 * n))
        assert np.allclose(np.diff(xi), d, rtol=1e-12, atol=1e-13)


def test_quick_uniform_weights(oracle):
    """Leonard's QUICK coefficients on a uniform grid (Sec. II B 3)."""
    ref = np.array([float(v) for v in _golden("quick_uniform.txt")[0]])
    assert np.allclose(oracle.lagrange3([-1.0, 0.0, 1.0], 0.5), ref, atol=1e-15)
    # negative direction: upwind node is i+1; nodes (i, i+1, i+2) at face i+1/2
    assert np.allclose(oracle.lagrange3([0.0, 1.0, 2.0], 0.5), ref[::-1], atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_lagrange_exact_on_quadratics(oracle, seed):
    """The 3-node interpolant reproduces any parabola exactly at any face,
    on arbitrarily stretched node positions (the meaning of the gammas)."""
    r = inputs.random_vector(6, seed)
    pos = np.sort(r[:3]) + np.array([0.0, 0.3, 0.6])
    x = pos[1] + 0.4 * (pos[2] - pos[1])
    a, b, c = r[3:]
    w = oracle.lagrange3(pos, x)
    assert np.isclose(w.sum(), 1.0, atol=1e-13)
    assert np.isclose(w @ (a + b * pos + c * pos**2), a + b * x + c * x**2, atol=1e-12)


def test_splitmix_published_outputs(oracle):
    """The counter generator's first output equals SplitMix64's published one."""
    for seed, out in _golden("splitmix64.txt"):
        expect = (int(out) >> 11) / 2.0**53
        assert oracle.splitmix_uniform(int(seed), 0) == expect


def test_table_rb_rayleigh_number(oracle):
    """Table rb: Ra = beta g dT H^3 / (nu kappa) with nu = tau c_s^2 gives
    2.5e6 for both rows only if the table's tau is the physical one."""
    for name, H, L, dt, tau, tau_g, dT, beta, g, ttot in _golden("table_rb.txt"):
        H, tau, tau_g, dT, beta, g = map(float, (H, tau, tau_g, dT, beta, g))
        Ra = beta * g * dT * H**3 / ((tau / 3.0) * (tau_g / 3.0))
        assert abs(Ra / 2.5e6 - 1.0) < 1e-3, name
