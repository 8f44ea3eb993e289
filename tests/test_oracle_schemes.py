"""Pins of the oracle's three FV time integrations (Sec. II B 2): explicit
Euler on the plain populations (Eq. (euler)), the semi-implicit collision
alone (Eq. (semi)) and with the Heun corrector (Eq. (semi-heun)).

Each scheme is pinned by what the paper states or the mathematics fixes:
the local relaxation factor and its stability region (Euler stable only for
dt <= 2 tau, the semi-implicit form for every dt), the order of accuracy in
time, exact mass conservation, and the ordering of the stability limits of
Fig. KOL3 on the decaying shear wave."""
import numpy as np
import pytest

from tests import inputs

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _uniform(oracle, scheme, tau, dt, ax=0.0, ay=0.0):
    f1 = inputs.random_populations(1, 1, seed=3, amp=0.2)[:, 0, 0]
    f = np.broadcast_to(f1[:, None, None], (9, 3, 3)).copy()
    g = oracle.RefGrid(3, 3).set_scheme(scheme).set_params(tau=tau, dt=dt, ax=ax, ay=ay)
    g.set_pops(f)
    return g, f1


@pytest.mark.parametrize("scheme", ["euler", "semi", "heun"])
def test_uniform_state_relaxation(oracle, scheme):
    """On a uniform state the flux divergence vanishes and one step is the
    source alone.  Euler relaxes f - f_eq by (1 - dt/tau) with the physical
    tau; the tilded schemes by (1 - dt/tau~), tau~ = tau + dt/2.  Momentum
    gains exactly dt rho a in all three (sum c F = rho a; the Euler moments
    carry no dt/2 shift)."""
    sch = {"euler": oracle.FV_EULER, "semi": oracle.FV_SEMI, "heun": oracle.FV_HEUN}[scheme]
    tau, dt, ax, ay = 0.35, 0.3, 1e-3, -2e-3
    g, f1 = _uniform(oracle, sch, tau, dt, ax, ay)
    rho = f1.sum()
    p0 = np.array([CX @ f1, CY @ f1])
    g.step_fv(1)
    fn = g.get_pops()[0][:, 1, 1]
    assert np.isclose(fn.sum(), rho, rtol=0, atol=1e-15)
    assert np.allclose([CX @ fn, CY @ fn], p0 + dt * rho * np.array([ax, ay]), rtol=0, atol=1e-15)
    g, f1 = _uniform(oracle, sch, tau, dt)
    feq = oracle.equilibrium(rho, *(p0 / rho))
    g.step_fv(1)
    fn = g.get_pops()[0][:, 1, 1]
    factor = 1 - dt / tau if scheme == "euler" else 1 - dt / (tau + dt / 2)
    assert np.allclose(fn - feq, factor * (f1 - feq), rtol=0, atol=1e-15)


def test_local_stability_regions(oracle):
    """Without advection Euler is stable only for dt <= 2 tau, while the
    semi-implicit collision is stable for every dt (Sec. II B 2): at
    dt = 2.5 tau the Euler non-equilibrium part grows by 1.5 per step, the
    semi-implicit one shrinks by 2/3 at dt = 10 tau."""
    tau = 0.2
    for scheme, dt, factor in ((oracle.FV_EULER, 2.5 * tau, -1.5), (oracle.FV_SEMI, 10 * tau, -2.0 / 3.0)):
        g, f1 = _uniform(oracle, scheme, tau, dt)
        rho = f1.sum()
        feq = oracle.equilibrium(rho, CX @ f1 / rho, CY @ f1 / rho)
        g.step_fv(4)
        fn = g.get_pops()[0][:, 1, 1]
        assert np.allclose(fn - feq, factor**4 * (f1 - feq), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("scheme", ["euler", "semi"])
@pytest.mark.parametrize("sy,bcy", [(0, 0), (1, 1)])
def test_single_stage_mass_conservation(oracle, scheme, sy, bcy):
    """The single-stage schemes keep the flux form: sum V rho is conserved to
    rounding with periodic faces and with double-reflection walls."""
    sch = oracle.FV_EULER if scheme == "euler" else oracle.FV_SEMI
    nx, ny = 7, 10
    g = oracle.RefGrid(nx, ny, sy=sy, stretch_y=2.0, bcy=bcy).set_scheme(sch)
    g.set_params(tau=0.3, dt=0.05, ax=1e-4)
    g.set_pops(inputs.random_populations(nx, ny, seed=11, amp=0.1))
    m0 = g.conservation()[0]
    g.step_fv(20)
    assert abs(g.conservation()[0] - m0) <= 1e-13 * abs(m0)


def _decay_rate(oracle, scheme, tau, dt, T=16.0, n=32):
    r = oracle.RefGrid(1, n, lx=1.0, ly=float(n)).set_scheme(scheme).set_params(tau=tau, dt=dt)
    r.init_preset(oracle.INIT_SHEAR, amp=1e-4)
    mode = np.sin(2 * np.pi * (np.arange(n) + 0.5) / n)
    a0 = r.moments()[1][:, 0] @ mode
    steps = int(round(T / dt))
    r.step_fv(steps)
    a1 = r.moments()[1][:, 0] @ mode
    return -np.log(a1 / a0) / (steps * dt)


@pytest.mark.parametrize("scheme,order", [("euler", 1), ("semi", 1), ("heun", 2)])
def test_time_order(oracle, scheme, order):
    """Decay rate of the shear wave u_x = A sin(2 pi y / L) at dt, dt/2, dt/4,
    dt/8: successive differences shrink by 2 for the first-order schemes
    (Euler; the semi-implicit collision with Euler advection) and approach 4
    for the Heun corrector (trapezoidal advection and collision).  The rate
    itself tends to nu k^2 up to the QUICK spatial error."""
    sch = {"euler": oracle.FV_EULER, "semi": oracle.FV_SEMI, "heun": oracle.FV_HEUN}[scheme]
    oracle.set_threads(1)
    tau = 0.3
    rates = np.array([_decay_rate(oracle, sch, tau, dt) for dt in (0.2, 0.1, 0.05, 0.025)])
    d = np.diff(rates)
    ratios = d[:-1] / d[1:]
    if order == 1:
        assert np.all(np.abs(ratios - 2.0) < 0.1), ratios
    else:
        assert 3.3 < ratios[-1] < 4.4 and ratios[-1] > ratios[0], ratios
    nuk2 = tau / 3 * (2 * np.pi / 32) ** 2
    assert abs(rates[-1] / nuk2 - 1) < 0.03


def _stable(oracle, scheme, tau, dt, steps=3000, n=64):
    """[1, 64] shear wave of amplitude 1e-5 with 1e-6 noise on every
    population (the linear stability of the decaying flow); unstable when
    the kinetic energy grows tenfold or turns non-finite within `steps`
    steps."""
    r = oracle.RefGrid(1, n, lx=1.0, ly=float(n)).set_scheme(scheme).set_params(tau=tau, dt=dt)
    r.init_preset(oracle.INIT_SHEAR, amp=1e-5)
    f, _ = r.get_pops()
    rng = np.random.default_rng(1)
    r.set_pops(f + 1e-6 * W[:, None, None] * rng.standard_normal(f.shape))
    k0 = None
    for _ in range(steps // 100):
        r.step_fv(100)
        _, ux, uy, _ = r.moments()
        k = float((ux**2 + uy**2).sum())
        k0 = k if k0 is None else k0
        if not np.isfinite(k) or k > 10 * k0:
            return False
    return True


@pytest.mark.parametrize("tau,dt,expect", [
    (0.25, 0.45, {"euler": False, "semi": True, "heun": True}),
    (0.25, 0.65, {"euler": False, "semi": False, "heun": True}),
    (0.125, 1.2, {"semi": False, "heun": True}),
    (0.5, 1.2, {"euler": False, "semi": False, "heun": True}),
    (0.25, 0.3, {"euler": True, "semi": True, "heun": True}),
])
def test_stability_ordering(oracle, tau, dt, expect):
    """Fig. KOL3: Euler is bounded by 2 tau and is narrower still with
    advection, the semi-implicit form is still limited by tau, and the Heun
    corrector allows dt > 1 for tau >= 1/8 (dt = 1.2 here)."""
    oracle.set_threads(1)
    sch = {"euler": oracle.FV_EULER, "semi": oracle.FV_SEMI, "heun": oracle.FV_HEUN}
    for name, want in expect.items():
        assert _stable(oracle, sch[name], tau, dt) == want, (name, tau, dt)


def test_scheme_switch_semantics(oracle):
    """The Euler state holds plain populations: initialised at f_eq (no
    -dt/2 F shift), moments without the dt/2 a shift, and the ST step
    refuses it."""
    r = oracle.RefGrid(4, 4).set_scheme(oracle.FV_EULER).set_params(tau=0.5, dt=1.0, ax=1e-3)
    r.init_preset(oracle.INIT_SHEAR, amp=0.01)
    f, _ = r.get_pops()
    rho, ux, uy, _ = r.moments()
    assert np.allclose(np.einsum("a,ayx->yx", CX, f) / f.sum(0), ux, rtol=0, atol=1e-15)
    with pytest.raises(ValueError):
        r.step_st(1)
    h = oracle.RefGrid(4, 4).set_params(tau=0.5, dt=1.0, ax=1e-3)
    h.init_preset(oracle.INIT_SHEAR, amp=0.01)
    fh, _ = h.get_pops()
    assert np.allclose(np.einsum("a,ayx->yx", CX, fh) / fh.sum(0) + 0.5e-3, h.moments()[1], rtol=0, atol=1e-15)
    with pytest.raises(ValueError):
        r.set_scheme(7)
