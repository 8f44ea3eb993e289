"""Pins of the oracle's ST and FV steps: exact invariants, closed-form flows,
symmetries and convergence order, each chosen so that a plausible mistake
(dropped term, wrong sign, swapped axis, wrong factor) fails one of them."""
import numpy as np
import pytest

from tests import inputs

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
ROT = np.array([0, 2, 3, 4, 1, 6, 7, 8, 5])      # c_a rotated by +90 degrees
MIRX = np.array([0, 3, 2, 1, 4, 6, 5, 8, 7])     # c_x -> -c_x
MIRY = np.array([0, 1, 4, 3, 2, 8, 7, 6, 5])     # c_y -> -c_y


def _grid(O, nx, ny, **kw):
    return O.RefGrid(nx, ny, **kw)


def _step(g, scheme, n=1):
    return g.step_st(n) if scheme == "st" else g.step_fv(n)


@pytest.mark.parametrize("scheme", ["st", "fv"])
def test_uniform_state_collision(oracle, scheme):
    """On a spatially uniform state advection vanishes and one step is the
    collision alone: mass is unchanged, momentum gains exactly dt rho a
    (Eqs. (ST), (semi-heun) with Eq. (F2)), and without force the
    non-equilibrium part decays by (1 - dt/tau~), tau~ = tau + dt/2."""
    dt = 1.0 if scheme == "st" else 0.4
    f1 = inputs.random_populations(1, 1, seed=3, amp=0.2)[:, 0, 0]
    f = np.broadcast_to(f1[:, None, None], (9, 3, 3)).copy()
    ax, ay, tau = 1e-3, -2e-3, 0.35
    g = _grid(oracle, 3, 3).set_params(tau=tau, dt=dt, ax=ax, ay=ay).set_pops(f)
    rho = f1.sum()
    p0 = np.array([CX @ f1, CY @ f1])
    _step(g, scheme)
    fn = g.get_pops()[0][:, 1, 1]
    assert np.isclose(fn.sum(), rho, rtol=0, atol=1e-15)
    assert np.allclose([CX @ fn, CY @ fn], p0 + dt * rho * np.array([ax, ay]), rtol=0, atol=1e-15)
    # relaxation rate without force
    g = _grid(oracle, 3, 3).set_params(tau=tau, dt=dt).set_pops(f)
    ux, uy = p0 / rho
    feq = oracle.equilibrium(rho, ux, uy)
    _step(g, scheme)
    fn = g.get_pops()[0][:, 1, 1]
    assert np.allclose(fn - feq, (1 - dt / (tau + dt / 2)) * (f1 - feq), rtol=0, atol=1e-15)


@pytest.mark.parametrize("scheme,sy,bcy", [("st", 0, 0), ("st", 0, 1), ("fv", 0, 0),
                                           ("fv", 1, 0), ("fv", 0, 1), ("fv", 1, 1)])
def test_mass_conservation(oracle, scheme, sy, bcy):
    """Global mass sum V rho is conserved to rounding: the flux form of
    Eq. (fv) telescopes, periodic faces cancel, and the double-reflection
    ghosts make the wall flux vanish (mirror-symmetric QUICK weights)."""
    nx, ny = 7, 10
    g = _grid(oracle, nx, ny, sy=sy, stretch_y=2.0, bcy=bcy)
    g.set_params(tau=0.3, dt=1.0 if scheme == "st" else 0.05, ax=1e-4)
    g.set_pops(inputs.random_populations(nx, ny, seed=11, amp=0.1))
    m0 = g.conservation()[0]
    _step(g, scheme, 20)
    assert abs(g.conservation()[0] / m0 - 1.0) < 1e-13


def test_periodic_momentum_balance(oracle):
    """Periodic FV grid: the flux terms cancel globally, so total momentum
    grows by exactly dt * (sum V rho) * a per step."""
    nx, ny = 6, 8
    g = _grid(oracle, nx, ny, sy=1, stretch_y=1.5).set_params(tau=0.4, dt=0.1, ax=2e-4, ay=-1e-4)
    g.set_pops(inputs.random_populations(nx, ny, seed=5, amp=0.1))
    m, px, py, _ = g.conservation()
    g.step_fv(5)
    m1, px1, py1, _ = g.conservation()
    assert np.isclose(px1 - px, 5 * 0.1 * m * 2e-4, rtol=1e-10, atol=1e-16)
    assert np.isclose(py1 - py, 5 * 0.1 * m * -1e-4, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_fv_pure_advection_order(oracle, axis):
    """With collisions switched off (tau -> infinity) every population obeys
    d_t f + c.grad f = 0.  The FV step transports a sine wave in the
    direction of c_a (sign check).  On node values the QUICK flux divergence
    (Sec. II B 3) has the Fourier symbol i k (1 - (k dx)^2 / 24) + O(dx^3):
    the wave keeps its amplitude and lags by k^3 dx^2 t / 24, so the error is
    second order with exactly that constant (other flux schemes differ:
    central -1/6, linear upwind +1/12, first-order upwind diffusive)."""
    L, t_end, eps = 16.0, 4.0, 0.01
    errs = []
    for n in (16, 32, 64):
        dx = L / n
        dt = 0.05 * dx
        if axis == "x":
            g = _grid(oracle, n, 1, lx=L, ly=1.0)
        else:
            g = _grid(oracle, 1, n, lx=1.0, ly=L)
        g.set_params(tau=1e12, dt=dt)
        s = (np.arange(n) + 0.5) * dx
        prof = 1 + eps * np.sin(2 * np.pi * s / L)
        f = W[:, None] * prof[None, :]
        f = f[:, None, :] if axis == "x" else f[:, :, None]
        g.set_pops(f)
        g.step_fv(int(round(t_end / dt)))
        out = g.get_pops()[0].reshape(9, n)
        c = CX if axis == "x" else CY
        exact = W[:, None] * (1 + eps * np.sin(2 * np.pi * (s[None, :] - c[:, None] * t_end) / L))
        errs.append(np.abs(out - exact).max())
    order = np.log2(errs[1] / errs[2])
    assert 1.9 < order < 2.2, (errs, order)
    # largest error: populations 1/3 (weight 1/9), phase lag k^3 dx^2 t / 24
    k = 2 * np.pi / L
    predicted = eps * (1 / 9) * k**3 * (L / 64) ** 2 * t_end / 24
    assert abs(errs[2] / predicted - 1) < 0.05, (errs[2], predicted)


def _tgv_amplitude(ux, xc, yc, L):
    k = 2 * np.pi / L
    mode = -np.cos(k * xc)[None, :] * np.sin(k * yc)[:, None]
    return float((ux * mode).sum() / (mode * mode).sum())


@pytest.mark.parametrize("scheme,dt,tol", [("st", 1.0, 0.01), ("fv", 0.5, 0.02)])
def test_taylor_green_decay(oracle, scheme, dt, tol):
    """Decaying Taylor-Green vortex on the 64x64 periodic grid, BGK tau~ =
    0.8 at dt = 1 (nu = 0.1): the amplitude follows exp(-2 nu k^2 t), with
    nu = (tau~ - dt/2) c_s^2 (Sec. II A).  FV uses dt = 0.5 at the same
    physical tau = 0.3 and reaches the same time t = 1000."""
    g = _grid(oracle, 64, 64).set_params(tau=0.3, dt=dt)
    g.init_preset(oracle.INIT_TGV, u0=0.01)
    xc, yc = g.centers()
    a0 = _tgv_amplitude(g.moments()[1], xc, yc, 64)
    _step(g, scheme, int(round(1000 / dt)))
    a1 = _tgv_amplitude(g.moments()[1], xc, yc, 64)
    expect = np.exp(-2 * 0.1 * (2 * np.pi / 64) ** 2 * 1000)
    assert abs(a1 / a0 / expect - 1) < tol


@pytest.mark.parametrize("scheme,tau,dt,tol", [("st", 0.5, 1.0, 0.01), ("fv", 0.5, 1.0, 0.02),
                                               ("fv", 0.1, 0.1, 0.02)])
def test_shear_wave_viscosity(oracle, scheme, tau, dt, tol):
    """Sec. III A: k_tot(t) = 1/4 A^2 L^2 exp(-2 (2 pi/L)^2 nu t) on the
    [1, 64] domain; the fitted nu matches tau c_s^2."""
    g = _grid(oracle, 1, 64, lx=1.0, ly=64.0).set_params(tau=tau, dt=dt)
    g.init_preset(oracle.INIT_SHEAR, amp=0.01, mode=1)
    ts, ks = [], []
    nsub = int(round(20 / dt))
    for k in range(10):
        _step(g, scheme, nsub)
        r, ux, uy, _ = g.moments()
        ts.append((k + 1) * nsub * dt)
        ks.append(0.5 * (r * (ux**2 + uy**2)).sum())
    slope = np.polyfit(ts, np.log(ks), 1)[0]
    nu = -slope / (2 * (2 * np.pi / 64) ** 2)
    assert abs(nu / (tau / 3) - 1) < tol


@pytest.mark.parametrize("scheme,sy", [("st", 0), ("fv", 1)])
def test_poiseuille_from_rest(oracle, scheme, sy):
    """Body-force-driven channel between no-slip walls (Sec. III B): started
    from rest, the flow settles on the parabola U(y) = 4 U y (L - y)/L^2 with
    a_x = 8 nu U / L^2 (the amplitude pins the force factor (1 - dt/2tau~))."""
    ny, U, tau = 16, 0.01, 0.5
    nu = tau / 3
    g = _grid(oracle, 2, ny, sy=sy, stretch_y=2.0, bcy=1)
    xi = g.face_coords()[1]
    dt = 1.0 if scheme == "st" else 0.9 * np.diff(xi).min()
    g.set_params(tau=tau, dt=dt, ax=8 * nu * U / ny**2)
    g.init_fields()
    _step(g, scheme, int(round(6000 / dt)))
    ux = g.moments()[1][:, 0]
    yc = g.centers()[1]
    Ue = 4 * U * yc * (ny - yc) / ny**2
    dy = np.diff(xi)
    err = np.sqrt(((ux - Ue) ** 2 * dy).sum() / (Ue**2 * dy).sum())
    assert err < 1e-2


def _rotate(f):
    """Rotate a [9, n, n] population field by +90 degrees about the centre."""
    n = f.shape[1]
    out = np.empty_like(f)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for a in range(9):
        out[ROT[a], i, n - 1 - j] = f[a, j, i]
    return out


@pytest.mark.parametrize("scheme", ["st", "fv"])
def test_rotation_equivariance(oracle, scheme):
    """Rotating the state by 90 degrees commutes with the step (square
    periodic uniform grid): catches swapped axes and x/y-asymmetric signs."""
    n = 8
    f = inputs.random_populations(n, n, seed=21, amp=0.2)
    dt = 1.0 if scheme == "st" else 0.3
    a = _grid(oracle, n, n).set_params(tau=0.4, dt=dt).set_pops(f)
    b = _grid(oracle, n, n).set_params(tau=0.4, dt=dt).set_pops(_rotate(f))
    _step(a, scheme, 3)
    _step(b, scheme, 3)
    assert np.allclose(_rotate(a.get_pops()[0]), b.get_pops()[0], rtol=0, atol=1e-14)


@pytest.mark.parametrize("scheme,sy", [("st", 0), ("fv", 0), ("fv", 1)])
def test_wall_mirror_symmetry(oracle, scheme, sy):
    """Mirroring y about the channel centre (walls, symmetric tanh grid) and x
    commutes with the step, force included: catches one-sided wall errors."""
    nx, ny = 5, 12
    f = inputs.random_populations(nx, ny, seed=8, amp=0.2)
    dt = 1.0 if scheme == "st" else 0.05
    mir = np.empty_like(f)
    for a in range(9):
        mir[MIRY[MIRX[a]]] = f[a, ::-1, ::-1]
    A = _grid(oracle, nx, ny, sy=sy, stretch_y=2.0, bcy=1).set_params(tau=0.3, dt=dt, ax=1e-4, ay=2e-4)
    B = _grid(oracle, nx, ny, sy=sy, stretch_y=2.0, bcy=1).set_params(tau=0.3, dt=dt, ax=-1e-4, ay=-2e-4)
    A.set_pops(f)
    B.set_pops(mir)
    _step(A, scheme, 4)
    _step(B, scheme, 4)
    fa, fb = A.get_pops()[0], B.get_pops()[0]
    back = np.empty_like(fa)
    for a in range(9):
        back[MIRY[MIRX[a]]] = fa[a, ::-1, ::-1]
    assert np.allclose(back, fb, rtol=0, atol=1e-14)


def test_fv_translation_invariance(oracle):
    """Shifting a periodic uniform state by one cell shifts the result."""
    f = inputs.random_populations(6, 5, seed=2, amp=0.2)
    A = _grid(oracle, 6, 5).set_params(tau=0.3, dt=0.2).set_pops(f)
    B = _grid(oracle, 6, 5).set_params(tau=0.3, dt=0.2).set_pops(np.roll(f, 1, axis=2))
    A.step_fv(3)
    B.step_fv(3)
    assert np.allclose(np.roll(A.get_pops()[0], 1, axis=2), B.get_pops()[0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_init_fields_roundtrip(oracle, seed):
    """Initial populations f~ = f_eq - dt/2 F (Appendix A) give back the
    prescribed rho and u through rho = sum f~, u = sum c f~/rho + dt/2 a."""
    rho, ux, uy, T = inputs.random_fields(5, 4, seed, T_amp=0.1)
    g = _grid(oracle, 5, 4, thermal=True).set_params(tau=0.3, dt=0.7, ax=1e-3, beta=0.01, grav=1.0)
    g.init_fields(rho, ux, uy, T)
    r, vx, vy, t = g.moments()
    assert np.allclose(r, rho, rtol=1e-15) and np.allclose(t, T, rtol=1e-15)
    assert np.allclose(vx, ux, atol=1e-16) and np.allclose(vy, uy, atol=1e-16)


@pytest.mark.parametrize("scheme,sy", [("st", 0), ("fv", 0), ("fv", 1)])
def test_conduction_state_is_steady(oracle, scheme, sy):
    """Fluid at rest with a linear temperature between isothermal plates
    (Sec. IV, below onset, beta = 0): the profile is an exact steady state of
    both schemes and every Nusselt number equals 1."""
    g = _grid(oracle, 3, 16, sy=sy, stretch_y=2.0, bcy=1, thermal=True)
    dt = 1.0 if scheme == "st" else 0.1
    g.set_params(tau=0.2, dt=dt, tau_g=0.2, T0=1.0, T_bot=1.5, T_top=0.5)
    g.init_preset(oracle.INIT_RB, amp=0.0)
    _step(g, scheme, 300)
    for nu in g.nusselt():
        assert abs(nu - 1.0) < 1e-10
    T = g.moments()[3][:, 0]
    yc = g.centers()[1]
    assert np.allclose(T, 1.0 + (0.5 - yc / 16.0), atol=1e-12)


def test_heat_conservation_periodic(oracle):
    """Periodic thermal FV grid: sum V T is conserved (sum g_eq = T)."""
    g = _grid(oracle, 6, 6, thermal=True).set_params(tau=0.3, dt=0.2, tau_g=0.25, beta=0.01, grav=1.0)
    g.set_pops(inputs.random_populations(6, 6, 3, amp=0.1), inputs.random_populations(6, 6, 4, amp=0.1))
    e0 = g.conservation()[3]
    g.step_fv(10)
    assert abs(g.conservation()[3] / e0 - 1) < 1e-13


def test_rb_preset_perturbation_is_seeded(oracle):
    """The RB preset adds amp*dT*(2U-1) with U from the counter generator."""
    g = _grid(oracle, 4, 6, bcy=1, thermal=True).set_params(tau=0.1, tau_g=0.1, T0=1.0, T_bot=1.5,
                                                            T_top=0.5)
    g.init_preset(oracle.INIT_RB, amp=1e-3, seed=1234)
    T = g.moments()[3]
    yc = g.centers()[1]
    for j in range(6):
        for i in range(4):
            U = oracle.splitmix_uniform(1234, j * 4 + i)
            assert np.isclose(T[j, i], 1.0 + (0.5 - yc[j] / 6) + 1e-3 * (2 * U - 1), rtol=0, atol=1e-15)


def _rb_rest_grid(O, sy, bg, ny=24, dt=1.0, rho="barometric"):
    """RB cell between plates at T0 -/+ dT/2 (dT = 1), no perturbation; beta g
    = bg.  rho="uniform" restarts the same conductive T with rho = 1, the
    start the barometric density exists to replace (Sec. IV)."""
    g = _grid(O, 3, ny, ly=float(ny), sy=sy, stretch_y=2.0, bcy=1, thermal=True)
    g.set_params(tau=0.2, dt=dt, tau_g=0.2, beta=bg, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)
    g.init_preset(O.INIT_RB, amp=0.0)
    if rho == "uniform":
        r, ux, uy, T = g.moments()
        g.init_fields(np.ones_like(r), np.zeros_like(ux), np.zeros_like(uy), T)
    return g


@pytest.mark.parametrize("sy", [0, 1])
def test_rb_barometric_density_solves_hydrostatics(oracle, sy):
    """The RB preset's density (Sec. IV, barometric equation) is the solution
    of c_s^2 d(ln rho)/dy = a_y = beta g (T_c - T0) with the conductive
    T_c = T0 + dT (1/2 - y/H), normalised to sum V rho = sum V.  ln rho is
    then quadratic in y, so its difference quotient between neighbouring
    centres equals the ODE's right-hand side at their midpoint exactly.  A
    sign error, a missing 1/c_s^2 = 3, or the wrong normalisation each fails
    one assertion; so does an asymmetric profile (rho(y) = rho(H - y))."""
    ny, bg = 24, 1e-3
    g = _rb_rest_grid(oracle, sy, bg, ny=ny)
    rho, ux, uy, T = g.moments()
    yc = g.centers()[1]
    assert np.ptp(rho, axis=1).max() == 0.0
    r = rho[:, 0]
    ybar = 0.5 * (yc[1:] + yc[:-1])
    dq = np.diff(np.log(r)) / np.diff(yc)
    assert np.allclose(dq, 3.0 * bg * (0.5 - ybar / ny), rtol=0, atol=1e-12)
    assert np.allclose(r, r[::-1], rtol=0, atol=1e-15)
    assert abs(g.conservation()[0] / (3.0 * ny) - 1.0) < 1e-14
    assert np.abs(ux).max() < 1e-16 and np.abs(uy).max() < 1e-16


def test_rb_barometric_start_is_at_rest_st(oracle):
    """ST from the barometric conductive state (Sec. IV: the barometric start
    avoids pressure waves at start-up).  The lattice's hydrostatic balance
    differs from the continuum one only at second order in beta g, so after
    100 steps the spurious velocity is O((beta g)^2): ten times weaker beta g
    leaves it at least 50 times smaller, and it stays 1e4 times below that of
    the uniform-density start, whose imbalance rho a is first order.  Every
    Nusselt number stays 1 to the same order."""
    out = {}
    for bg in (1e-3, 1e-4):
        for rho in ("barometric", "uniform"):
            g = _rb_rest_grid(oracle, 0, bg, rho=rho)
            g.step_st(100)
            _, ux, uy, _ = g.moments()
            out[bg, rho] = (max(np.abs(ux).max(), np.abs(uy).max()), g.nusselt())
    assert out[1e-3, "barometric"][0] < 3e-8
    assert out[1e-4, "barometric"][0] < 3e-10
    assert out[1e-3, "barometric"][0] > 50 * out[1e-4, "barometric"][0]
    for bg in (1e-3, 1e-4):
        assert out[bg, "barometric"][0] < 1e-4 * out[bg, "uniform"][0]
        assert out[bg, "uniform"][0] > 0.5 * bg
        for nu in out[bg, "barometric"][1]:
            assert abs(nu - 1.0) < 5.0 * bg * bg


@pytest.mark.parametrize("sy", [0, 1])
def test_rb_barometric_start_is_at_rest_fv_interior(oracle, sy):
    """FV (Heun) from the barometric conductive state, uniform and tanh
    plates.  The double-reflection ghosts mirror rho evenly, so the wall
    cells see a first-order density kink (Sec. II B 5 calls the wall rule
    first order); one step reaches four rows into the fluid (two QUICK
    stages of two rows each).  Beyond those rows one step leaves only the
    O((beta g)^2) residual of QUICK on ln rho quadratic, 1e4 times below the
    uniform-density start's dt * a."""
    ny, dt = 24, 0.1
    res = {}
    for bg in (1e-3, 1e-4):
        for rho in ("barometric", "uniform"):
            g = _rb_rest_grid(oracle, sy, bg, ny=ny, dt=dt, rho=rho)
            g.step_fv(1)
            _, ux, uy, _ = g.moments()
            assert np.abs(ux).max() < 1e-18
            res[bg, rho] = np.abs(uy[4:ny - 4]).max()
    assert res[1e-3, "barometric"] < 2e-9
    assert res[1e-3, "barometric"] > 50 * res[1e-4, "barometric"]
    for bg in (1e-3, 1e-4):
        assert res[bg, "barometric"] < 1e-4 * res[bg, "uniform"]
        assert res[bg, "uniform"] > 0.2 * dt * bg


@pytest.mark.parametrize("dt", [0.5, 0.25])
def test_hydrostatic_column_stays_at_rest(oracle, dt):
    """A column between walls under a uniform body force a_y, started in
    hydrostatic balance (c_s^2 d rho/dy = rho a_y): a fluid at rest under
    gravity stays at rest.  In the middle quarter of the column (away from
    the first-order wall layers of Sec. II B 5) the FV state settles at
    |u_y| below 1e-4 |a_y|, independent of dt.  This pins the force part of the advected field:
    with the plain population of Appendix A, (dt/2)(1 - dt/(2 tau~)) F, the
    advected mass flux sum c h equals rho u; with dt/2 F it would carry an
    extra dt^2 rho a / (4 tau~), and the steady column would drift at
    u_y = -dt^2 a_y / (4 tau~) (1.4e-4 at dt = 0.5 here)."""
    ny, tau, ay = 32, 0.2, -1e-3
    g = _grid(oracle, 3, ny, ly=float(ny), bcy=1).set_params(tau=tau, dt=dt, ay=ay)
    yc = g.centers()[1]
    rho = np.exp(3 * ay * (yc - ny / 2))[:, None] * np.ones((ny, 3))
    g.init_fields(rho, np.zeros_like(rho), np.zeros_like(rho), None)
    g.step_fv(int(12000 / dt))
    uy = g.moments()[2][:, 0]
    literal = -dt * dt * ay / (4 * (tau + dt / 2))
    assert np.abs(uy[12:20]).max() < 1e-4 * abs(ay)
    assert np.abs(uy[12:20]).max() < 0.01 * abs(literal)


def _golden_rb():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "rb_ra1e4.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            Ra, Pr, Ar, Nu, tol = map(float, line.split())
            return Ra, Pr, Ar, Nu, tol


def test_rb_ra1e4_nusselt(oracle):
    """Sec. IV: 2-D Rayleigh-Benard at Ra = 1e4, Pr = 1, Ar = 2.02 settles on a
    steady roll pair with Nu ~= 2.66 (the Clever & Busse value the paper
    compares to).  ST oracle, H = 32, 0.9 diffusive times; every Nusselt
    number (volume, both plates) within the stated tolerance."""
    from paper_1505_03271_gb300 import configs as cfg
    Ra, Pr, Ar, Nu_ref, tol = _golden_rb()
    H = 32
    nx = int(round(Ar * H))
    p = cfg.rb_params(Ra, Pr, float(H))
    g = oracle.RefGrid(nx, H, lx=float(nx), ly=float(H), bcy=oracle.WALLS, thermal=True)
    g.set_params(tau=p.tau, dt=1.0, tau_g=p.tau_g, beta=p.beta, grav=p.grav, T0=p.T0, T_bot=p.T_bot,
                 T_top=p.T_top)
    g.init_preset(oracle.INIT_RB, amp=1e-2, seed=3)
    g.step_st(int(0.9 * H * H / p.kappa))
    for nu in g.nusselt():
        assert abs(nu - Nu_ref) < tol, g.nusselt()


@pytest.mark.parametrize("sy,stretch", [(0, 0.0), (1, 2.0)], ids=["uniform", "tanh"])
def test_plate_nusselt_exact_on_quadratic_profiles(oracle, sy, stretch):
    """The plate Nusselt numbers (Sec. IV post-processing: the quadratic
    through the wall value and the first two cell centres) are exact on any
    temperature profile T(y) = T_bot + b y + c y^2 that meets both plate
    temperatures, where a first-order one-sided gradient would be off by
    c y_0.  With the fluid at rest the volume Nusselt number is exactly 1."""
    nx, ny, H = 3, 12, 12.0
    T_bot, T_top, c = 1.5, 0.5, 2e-3
    b = (T_top - T_bot - c * H * H) / H
    g = oracle.RefGrid(nx, ny, ly=H, sy=sy, stretch_y=stretch, bcy=1, thermal=True)
    g.set_params(tau=0.2, dt=0.1, tau_g=0.2, beta=1e-3, grav=1.0, T0=1.0, T_bot=T_bot, T_top=T_top)
    yc = g.centers()[1]
    T = np.repeat((T_bot + b * yc + c * yc * yc)[:, None], nx, axis=1)
    g.init_fields(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), T)
    nu_vol, nu_bot, nu_top = g.nusselt()
    dT = T_bot - T_top
    assert nu_vol == pytest.approx(1.0, abs=1e-14)
    assert nu_bot == pytest.approx(-H * b / dT, rel=1e-12)
    assert nu_top == pytest.approx(-H * (b + 2 * c * H) / dT, rel=1e-12)
    # the curvature matters at this size: a first-order gradient would miss it
    assert abs((T[0, 0] - T_bot) / yc[0] - b) > 1e-3 * abs(b)
