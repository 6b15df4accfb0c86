"""Closed-form solution pairs for -Δu = f (TEST INFRASTRUCTURE ONLY).

These pin the oracle to the mathematics rather than to itself: for a finite
sum of plane waves the periodic solution is known exactly, and on a grid with
every |k_i| < n_i/2 the discrete solve reproduces it up to rounding.
"""
from __future__ import annotations

import numpy as np


def _phase(k, phi, shape):
    nx, ny, nz = shape
    x = np.arange(nx)[:, None, None] / nx
    y = np.arange(ny)[None, :, None] / ny
    z = np.arange(nz)[None, None, :] / nz
    return 2.0 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + phi


def mode_sum_f(k, a, phi, shape) -> np.ndarray:
    """f = sum_m a_m sin(2π k_m·x + φ_m), evaluated directly with np.sin."""
    f = np.zeros(tuple(shape))
    for km, am, pm in zip(k, a, phi):
        f += am * np.sin(_phase(km, pm, shape))
    return f


def mode_sum_u(k, a, phi, shape) -> np.ndarray:
    """u for f = sum a sin(2π k·x + φ):  -Δ sin(2π k·x + φ) = 4π²|k|² sin(...),
    so u = sum a/(4π²|k|²) sin(2π k·x + φ) (mean zero, as the solve fixes)."""
    u = np.zeros(tuple(shape))
    for km, am, pm in zip(k, a, phi):
        k2 = float(np.dot(km, km))
        u += am / (4.0 * np.pi ** 2 * k2) * np.sin(_phase(km, pm, shape))
    return u


def paper_case1_u(kw: int, shape) -> np.ndarray:
    """Test case 1 of §3: u = sin(2πk x1) sin(2πk x2) sin(2πk x3)."""
    nx, ny, nz = shape
    sx = np.sin(2.0 * np.pi * kw * np.arange(nx) / nx)
    sy = np.sin(2.0 * np.pi * kw * np.arange(ny) / ny)
    sz = np.sin(2.0 * np.pi * kw * np.arange(nz) / nz)
    return sx[:, None, None] * sy[None, :, None] * sz[None, None, :]


def paper_case1_f(kw: int, shape) -> np.ndarray:
    """f = -Δu for test case 1: each factor contributes (2πk)², so f = 12π²k² u."""
    return 12.0 * np.pi ** 2 * kw ** 2 * paper_case1_u(kw, shape)
