"""Pins of the oracle's fixed-density boundary (Sec. II B 5): ghost densities
extrapolated linearly through the imposed face value, ghost populations the
mirrored node's rescaled by the density ratio.

  * one step from a uniform rest state moves exactly the mass the QUICK face
    values of the ghosts imply (a closed form on the uniform grid);
  * a uniform state at the imposed density is a fixed point;
  * a channel driven by a density difference reaches the steady state of the
    same channel driven by the equivalent body force c_s^2 d(rho)/L, with a
    linear density that extrapolates to the imposed face values."""
import numpy as np
import pytest


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("scheme", ["euler", "semi"])
def test_one_step_mass_flux(oracle, axis, scheme):
    """Uniform rest state rho0, density rho_S on the low face of one axis
    (rho0 on the high one).  At rest h_a = w_a rho0 and the ghosts hold
    w_a (2 rho_S - rho0); on the uniform grid the QUICK face values are
    w (5 rho_g + 3 rho0)/8 (c > 0) and w (3 rho_g + 5 rho0)/8 (c < 0), and the
    D2Q9 weights moving each way sum to 1/6, so one single-stage step adds
    dt * L_other * (rho_S - rho0) / 12 of mass."""
    sch = oracle.FV_EULER if scheme == "euler" else oracle.FV_SEMI
    nx, ny, dt, rho_s = (8, 5, 0.3, 1.02) if axis == "x" else (5, 8, 0.3, 1.02)
    kw = dict(bcx=oracle.DENSITY) if axis == "x" else dict(bcy=oracle.DENSITY)
    r = oracle.RefGrid(nx, ny, **kw).set_scheme(sch).set_params(tau=0.5, dt=dt)
    if axis == "x":
        r.set_boundary_density(rho_x0=rho_s)
    else:
        r.set_boundary_density(rho_y0=rho_s)
    r.init_fields()
    m0 = r.conservation()[0]
    r.step_fv(1)
    other = ny if axis == "x" else nx
    assert abs(r.conservation()[0] - m0 - dt * other * (rho_s - 1.0) / 12.0) < 1e-14


@pytest.mark.parametrize("scheme", ["euler", "semi", "heun"])
def test_imposed_density_is_a_fixed_point(oracle, scheme):
    """A uniform rest state at the imposed density stays put: the ghosts
    copy the nodes (ratio 1) and every flux cancels."""
    sch = {"euler": oracle.FV_EULER, "semi": oracle.FV_SEMI, "heun": oracle.FV_HEUN}[scheme]
    r = oracle.RefGrid(6, 7, bcx=oracle.DENSITY, bcy=oracle.WALLS, sy=oracle.TANH, stretch_y=1.5)
    r.set_scheme(sch).set_params(tau=0.4, dt=0.1).set_boundary_density(1.03, 1.03)
    r.init_fields(rho=np.full((7, 6), 1.03))
    f0, _ = r.get_pops()
    r.step_fv(20)
    assert np.abs(r.get_pops()[0] - f0).max() < 1e-15


def test_pressure_driven_channel(oracle):
    """Steady channel between no-slip walls on y, driven by rho_in - rho_out
    = 2e-3 across L_x = 32: the same profile as the body-force channel with
    a_x = c_s^2 (rho_in - rho_out) / L_x to the compressibility order
    (relative 2e-3), the mass flux constant along x, and the centre-line
    density linear, reaching the imposed values at the faces."""
    oracle.set_threads(1)
    nx, ny, tau, dt, drho = 32, 16, 0.5, 0.9, 2e-3
    grad = drho / 3.0 / nx
    p = oracle.RefGrid(nx, ny, bcx=oracle.DENSITY, bcy=oracle.WALLS).set_params(tau=tau, dt=dt)
    p.set_boundary_density(1 + drho / 2, 1 - drho / 2)
    xc = np.arange(nx) + 0.5
    p.init_fields(rho=np.broadcast_to(1 + drho / 2 - drho * xc / nx, (ny, nx)).copy())
    f = oracle.RefGrid(nx, ny, bcy=oracle.WALLS).set_params(tau=tau, dt=dt, ax=grad)
    f.init_fields()
    p.step_fv(3000)
    f.step_fv(3000)
    rp, up, vp, _ = p.moments()
    _, uf, _, _ = f.moments()
    assert np.abs(up[:, nx // 2] - uf[:, nx // 2]).max() < 2e-3 * uf.max()
    flux = (rp * up).sum(0)
    assert np.ptp(flux) < 1e-4 * flux.mean()
    line = rp[ny // 2]
    slope = np.polyfit(xc, line, 1)
    assert np.abs(np.polyval(slope, xc) - line).max() < 2e-4 * drho  # first-order wall layers
    assert abs(np.polyval(slope, 0.0) - (1 + drho / 2)) < 1e-6
    assert abs(np.polyval(slope, float(nx)) - (1 - drho / 2)) < 1e-6


def test_density_axis_rules(oracle):
    """Thermal grids keep periodic x and plates on y; the ST step has no
    fixed-density boundary."""
    with pytest.raises(ValueError):
        oracle.RefGrid(8, 8, bcx=oracle.DENSITY, thermal=True)
    with pytest.raises(ValueError):
        oracle.RefGrid(8, 8, bcy=oracle.DENSITY, thermal=True)
    r = oracle.RefGrid(8, 8, bcx=oracle.DENSITY).set_params(tau=0.5, dt=1.0)
    r.init_fields()
    with pytest.raises(ValueError):
        r.step_st(1)
    with pytest.raises(ValueError):
        r.set_boundary_density(0.0, 1.0)
