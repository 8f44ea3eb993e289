"""Seeded synthetic input generators shared by the oracle and the CUDA tests.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no equilibrium, force, flux or moment formula).
"""
from __future__ import annotations

import numpy as np

# D2Q9 weights in the standard order; used only to place random populations
# near a physically sensible magnitude.
_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def random_populations(nx: int, ny: int, seed: int, amp: float = 0.05, base: float = 1.0):
    """Populations base*w_a*(1 + amp*U(-1,1)), shape [9, ny, nx], FP64."""
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-1.0, 1.0, size=(9, ny, nx))
    return (_W[:, None, None] * base * (1.0 + amp * noise)).astype(np.float64)


def random_fields(nx: int, ny: int, seed: int, u_amp: float = 0.02, rho_amp: float = 0.01,
                  T_amp: float = 0.0, T0: float = 1.0):
    """Random macroscopic fields rho, ux, uy, T, each [ny, nx], FP64."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, (ny, nx))
    ux = u_amp * rng.uniform(-1, 1, (ny, nx))
    uy = u_amp * rng.uniform(-1, 1, (ny, nx))
    T = T0 + T_amp * rng.uniform(-1, 1, (ny, nx))
    return rho, ux, uy, T


# D3Q19 weights in the library's order (rest, 6 axis, 12 edge velocities).
_W3 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def random_populations3(nx: int, ny: int, nz: int, seed: int, amp: float = 0.05, base: float = 1.0):
    """D3Q19 populations base*w_a*(1 + amp*U(-1,1)), shape [19, nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-1.0, 1.0, size=(19, nz, ny, nx))
    return (_W3[:, None, None, None] * base * (1.0 + amp * noise)).astype(np.float64)


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0):
    return np.random.default_rng(seed).uniform(lo, hi, n)
