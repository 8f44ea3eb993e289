"""Post-processing of the 3-D Rayleigh-Benard statistics (Sec. IV; no GPU):
the stretched-grid z derivative, the gradient used for the dissipation rates
and the turnover time from the kinetic-energy autocorrelation."""
import numpy as np
import pytest

from paper_1505_03271_gb300 import studies as S


def test_z_derivative_exact_on_quadratics():
    z = np.cumsum(np.linspace(0.5, 1.5, 12))
    f = 3 * z ** 2 - 2 * z + 1
    m, w = S._ddz_weights(z)
    d = w[:, 0] * f[m - 1] + w[:, 1] * f[m] + w[:, 2] * f[m + 1]
    assert np.allclose(d, 6 * z - 2, rtol=0, atol=1e-12)
    assert np.allclose(d, S._ddz(z, f), rtol=0, atol=1e-12)


def test_gradient_of_a_periodic_field():
    nz, ny, nx = 6, 16, 20
    z = np.cumsum(np.linspace(0.8, 1.2, nz))
    m, w = S._ddz_weights(z)
    x = (np.arange(nx) + 0.5) * 0.5
    y = (np.arange(ny) + 0.5) * 0.25
    kx, ky = 2 * np.pi / (nx * 0.5), 2 * np.pi / (ny * 0.25)
    f = (np.sin(kx * x)[None, None, :] * np.cos(ky * y)[None, :, None]) * (1 + 0 * z)[:, None, None] + \
        (z ** 2)[:, None, None]
    gx, gy, gz = S._grad(f, 0.5, 0.25, m, w)
    # central differences: the exact derivative times sin(k h)/(k h)
    ex = kx * np.cos(kx * x)[None, None, :] * np.cos(ky * y)[None, :, None] * np.sinc(kx * 0.5 / np.pi)
    ey = -ky * np.sin(kx * x)[None, None, :] * np.sin(ky * y)[None, :, None] * np.sinc(ky * 0.25 / np.pi)
    assert np.allclose(gx, ex, atol=1e-12) and np.allclose(gy, ey, atol=1e-12)
    assert np.allclose(gz, np.broadcast_to((2 * z)[:, None, None], f.shape), atol=1e-12)


def test_turnover_time_of_a_cosine():
    t = np.arange(400) * 0.5
    assert S._turnover(np.cos(2 * np.pi * t / 40.0), 0.5) == pytest.approx(10.0, rel=0.05)
    assert S._turnover(np.ones(50), 1.0) is None
