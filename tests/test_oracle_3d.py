"""Pins of the D3Q19 oracle (the lattice of the paper's 3-D runs, Sec. II B 5
and Sec. IV).

The strongest pin is a projection: summed over one velocity component, the
D3Q19 weights, equilibrium and Guo force are exactly D2Q9's when the flow does
not depend on that axis, and every step (streaming, QUICK fluxes, walls,
collision) commutes with the sum.  A 3-D run of such a flow, projected onto
the other two axes, must therefore equal the two-dimensional oracle, which
is pinned on its own.  Running the projection in the (y, z) plane exercises
the z plates, the stretched z grid and buoyancy along z.  Besides: the
lattice's moment identities, equilibrium and force moments, exact mass
conservation, the 3-D Taylor-Green decay rate and the conduction state."""
import numpy as np
import pytest

from tests import inputs

D2 = dict(cx=np.array([0, 1, 0, -1, 0, 1, -1, -1, 1]), cy=np.array([0, 0, 1, 0, -1, 1, 1, -1, -1]))


def _d2_index(u, v):
    for b in range(9):
        if D2["cx"][b] == u and D2["cy"][b] == v:
            return b
    raise AssertionError


def _projection(oracle, plane):
    """Matrix P[b, a]: D3Q19 population a contributes to D2Q9 population b
    of the plane ("xy": drop c_z, "yz": drop c_x, map (c_y, c_z) -> (x, y))."""
    cx, cy, cz, _, _ = oracle.lattice3()
    P = np.zeros((9, 19))
    for a in range(19):
        u, v = (cx[a], cy[a]) if plane == "xy" else (cy[a], cz[a])
        P[_d2_index(u, v), a] = 1.0
    return P


def test_d3q19_lattice_moments(oracle):
    """sum w = 1, sum w c = 0, sum w c_i c_j = delta_ij / 3, the odd third
    moments vanish and sum w c_i c_j c_k c_l = (delta delta + ...) / 9;
    inv(a) reverses c_a."""
    cx, cy, cz, w, inv = oracle.lattice3()
    c = np.stack([cx, cy, cz], 1).astype(float)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj->ij", w, c, c), np.eye(3) / 3, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj,ak->ijk", w, c, c, c), 0.0, atol=1e-15)
    d = np.eye(3)
    iso = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)) / 9
    assert np.allclose(np.einsum("a,ai,aj,ak,al->ijkl", w, c, c, c, c), iso, atol=1e-15)
    assert np.array_equal(c[inv], -c)


@pytest.mark.parametrize("seed", range(3))
def test_d3q19_equilibrium_and_force_moments(oracle, seed):
    """sum f_eq = rho, sum c f_eq = rho u, sum c c f_eq = rho (u u + I/3);
    sum F = 0, sum c F = rho a, sum c c F = rho (a u + u a) (Eq. (F2))."""
    r = inputs.random_vector(7, seed)
    rho, u, a = 1 + 0.1 * r[0], 0.05 * r[1:4], 1e-3 * r[4:7]
    cx, cy, cz, _, _ = oracle.lattice3()
    c = np.stack([cx, cy, cz], 1).astype(float)
    feq = oracle.equilibrium3(rho, *u)
    assert np.isclose(feq.sum(), rho, atol=1e-15)
    assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj->ij", feq, c, c), rho * (np.outer(u, u) + np.eye(3) / 3), atol=1e-15)
    F = oracle.guo_force3(rho, *u, *a)
    assert abs(F.sum()) < 1e-17
    assert np.allclose(c.T @ F, rho * a, atol=1e-17)
    assert np.allclose(np.einsum("a,ai,aj->ij", F, c, c), rho * (np.outer(a, u) + np.outer(u, a)), atol=1e-17)


def _rb2d(oracle, nx, ny, **kw):
    return oracle.RefGrid(nx, ny, **kw)


@pytest.mark.parametrize("scheme", ["st", "fv"])
def test_projection_xy_equals_d2q9(oracle, scheme):
    """z-independent flow on a periodic box (nz = 2): the c_z-summed 3-D
    state follows the 2-D oracle step for step (forced, x periodic, y walls;
    the FV run on a tanh y grid)."""
    nx, ny, nz = 9, 8, 2
    sy, st = (0, 0.0) if scheme == "st" else (1, 1.5)
    dt = 1.0 if scheme == "st" else 0.2
    kw = dict(tau=0.3, dt=dt, ax=1e-4, ay=-2e-4)
    g3 = oracle.RefGrid3(nx, ny, nz, sy=sy, stretch_y=st, bcy=oracle.WALLS).set_params(**kw)
    g2 = oracle.RefGrid(nx, ny, sy=sy, stretch_y=st, bcy=oracle.WALLS).set_params(**kw)
    rho, ux, uy, _ = inputs.random_fields(nx, ny, seed=4, u_amp=0.03, rho_amp=0.02)
    g2.init_fields(rho, ux, uy)
    rep = lambda a: np.broadcast_to(a, (nz, ny, nx)).copy()
    g3.init_fields(rep(rho), rep(ux), rep(uy))
    P = _projection(oracle, "xy")
    for _ in range(3):
        (g3.step_st if scheme == "st" else g3.step_fv)(2)
        (g2.step_st if scheme == "st" else g2.step_fv)(2)
        f3 = g3.get_pops()[0]
        proj = np.einsum("ba,akji->kbji", P, f3)
        assert np.abs(proj[0] - g2.get_pops()[0]).max() < 1e-14
        assert np.abs(proj[1] - proj[0]).max() < 1e-15


@pytest.mark.parametrize("scheme", ["st", "fv"])
def test_projection_yz_thermal_plates(oracle, scheme):
    """x-independent Rayleigh-Benard state (nx = 1): projected onto (y, z) it
    follows the 2-D oracle with (x, y) = (y, z): plates, anti-reflected
    thermal ghosts, buoyancy along z and (FV) a sinh z grid."""
    ny, nz = 10, 8
    sz, st = (0, 0.0) if scheme == "st" else (2, 4.0)
    dt = 1.0 if scheme == "st" else 0.1
    kw = dict(tau=0.2, tau_g=0.25, dt=dt, beta=2e-3, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)
    g3 = oracle.RefGrid3(1, ny, nz, lx=1.0, sz=sz, stretch_z=st, bcz=oracle.WALLS, thermal=True)
    g3.set_params(**kw)
    g2 = oracle.RefGrid(ny, nz, sy=sz, stretch_y=st, bcy=oracle.WALLS, thermal=True)
    g2.set_params(tau=kw["tau"], tau_g=kw["tau_g"], dt=dt, beta=2e-3, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)
    rho, uy, uz, T = inputs.random_fields(ny, nz, seed=9, u_amp=0.02, rho_amp=0.02, T_amp=0.3)
    g2.init_fields(rho, uy, uz, T)
    ex = lambda a: a[:, :, None].copy()
    g3.init_fields(ex(rho), np.zeros((nz, ny, 1)), ex(uy), ex(uz), ex(T))
    P = _projection(oracle, "yz")
    for _ in range(3):
        (g3.step_st if scheme == "st" else g3.step_fv)(3)
        (g2.step_st if scheme == "st" else g2.step_fv)(3)
        f3, t3 = g3.get_pops()
        f2, t2 = g2.get_pops()
        assert np.abs(np.einsum("ba,akj->bkj", P, f3[..., 0]) - f2).max() < 1e-14
        assert np.abs(np.einsum("ba,akj->bkj", P, t3[..., 0]) - t2).max() < 1e-14
    nu3, nu2 = g3.nusselt(), g2.nusselt()
    assert np.allclose(nu3, nu2, rtol=1e-12, atol=1e-12)


def test_fv_mass_conservation_3d(oracle):
    """The flux form conserves sum V rho to rounding with walls on two axes
    and a stretched grid."""
    g = oracle.RefGrid3(5, 6, 8, sy=1, stretch_y=2.0, sz=2, stretch_z=5.0, bcy=oracle.WALLS, bcz=oracle.WALLS)
    g.set_params(tau=0.3, dt=0.05, ax=1e-4)
    g.set_pops(inputs.random_populations3(5, 6, 8, seed=3, amp=0.1))
    m0 = g.conservation()[0]
    g.step_fv(10)
    assert abs(g.conservation()[0] - m0) < 1e-13 * m0


@pytest.mark.parametrize("scheme", ["st", "fv"])
def test_taylor_green_3d_decay(oracle, scheme):
    """3-D Taylor-Green vortex at low Reynolds number decays at
    nu (kx^2 + ky^2 + kz^2) = 3 nu k^2 (amplitude): measured between t = 10
    and t = 50 (after the start-up transient), within 2 % on 24^3 (1.1 %
    ST, 1.4 % FV; 2.6 % and 3.0 % on 16^3, second-order convergence)."""
    oracle.set_threads(4)
    n, tau, u0 = 24, 0.3, 1e-3
    dt = 1.0 if scheme == "st" else 0.5
    g = oracle.RefGrid3(n, n, n).set_params(tau=tau, dt=dt).init_preset(oracle.INIT_TGV, u0=u0)
    x = (np.arange(n) + 0.5) * 2 * np.pi / n
    mode = np.sin(x)[None, None, :] * np.cos(x)[None, :, None] * np.cos(x)[:, None, None]
    step = g.step_st if scheme == "st" else g.step_fv
    step(int(round(10 / dt)))
    a0 = (g.moments()[1] * mode).sum()
    step(int(round(40 / dt)))
    a1 = (g.moments()[1] * mode).sum()
    rate = -np.log(a1 / a0) / 40.0
    assert abs(rate / (tau / 3 * 3 * (2 * np.pi / n) ** 2) - 1) < 0.02


def test_conduction_state_3d(oracle):
    """Rest state with the linear conductive profile between isothermal
    plates (beta = 0, below onset) on a sinh z grid is an exact steady state
    of both schemes: T stays linear and every Nusselt number is 1."""
    for scheme, sz, dt in (("st", 0, 1.0), ("fv", 2, 0.1)):
        kw = dict(tau=0.2, tau_g=0.2, dt=dt, T0=1.0, T_bot=1.5, T_top=0.5)
        g = oracle.RefGrid3(4, 3, 12, lz=12.0, sz=sz, stretch_z=4.0, bcz=oracle.WALLS, thermal=True)
        g.set_params(**kw).init_preset(oracle.INIT_RB, amp=0.0)
        (g.step_st if scheme == "st" else g.step_fv)(200)
        _, ux, uy, uz, T = g.moments()
        assert max(np.abs(ux).max(), np.abs(uy).max(), np.abs(uz).max()) < 1e-13
        xi = oracle.faces(12, 12.0, sz, 4.0)
        zc = 0.5 * (xi[1:] + xi[:-1])
        assert np.allclose(T, (1.0 + (0.5 - zc / 12.0))[:, None, None], atol=1e-12)
        assert np.allclose(g.nusselt(), 1.0, atol=1e-10)


def test_plate_nusselt_exact_on_quadratic_profiles_3d(oracle):
    """As in two dimensions: on T(z) = T_bot + b z + c z^2 meeting both plate
    temperatures, the plate Nusselt numbers equal -H T'(0)/dT and
    -H T'(H)/dT to rounding, on a sinh z grid; at rest Nu_vol = 1."""
    nx, ny, nz, H = 3, 2, 12, 12.0
    T_bot, T_top, c = 1.5, 0.5, 2e-3
    b = (T_top - T_bot - c * H * H) / H
    g = oracle.RefGrid3(nx, ny, nz, lz=H, sz=oracle.SINH, stretch_z=3.0, bcz=oracle.WALLS, thermal=True)
    g.set_params(tau=0.2, dt=0.1, tau_g=0.2, beta=1e-3, grav=1.0, T0=1.0, T_bot=T_bot, T_top=T_top)
    xi = oracle.faces(nz, H, oracle.SINH, 3.0)
    zc = 0.5 * (xi[1:] + xi[:-1])
    shape = (nz, ny, nx)
    T = np.broadcast_to((T_bot + b * zc + c * zc * zc)[:, None, None], shape).copy()
    g.init_fields(np.ones(shape), np.zeros(shape), np.zeros(shape), np.zeros(shape), T)
    nu_vol, nu_bot, nu_top = g.nusselt()
    dT = T_bot - T_top
    assert nu_vol == pytest.approx(1.0, abs=1e-14)
    assert nu_bot == pytest.approx(-H * b / dT, rel=1e-12)
    assert nu_top == pytest.approx(-H * (b + 2 * c * H) / dT, rel=1e-12)
