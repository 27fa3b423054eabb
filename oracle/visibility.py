"""Visibility oracle, Sec. 6.4, Eqs. (108)-(109).  Test infrastructure only.

V(u, v) = sum_ij I_ij exp[-2 pi i (u X_i + v Y_j)] dX dY on the cell-centred
screen, evaluated directly in FP64 one baseline at a time (no separation of
the exponential, no blocking).  u, v are in cycles per M.
"""
from __future__ import annotations

import numpy as np

from .diagnostics import screen_centres


def visibilities(I, x_min, x_max, y_min, y_max, uv) -> np.ndarray:
    I = np.asarray(I, dtype=np.float64)
    ny, nx = I.shape
    X, Y, dx, dy = screen_centres(nx, ny, x_min, x_max, y_min, y_max)
    XX, YY = np.meshgrid(X, Y)
    uv = np.asarray(uv, dtype=np.float64).reshape(-1, 2)
    out = np.empty(uv.shape[0], dtype=np.complex128)
    for k, (u, v) in enumerate(uv):
        phase = -2.0 * np.pi * (u * XX + v * YY)
        out[k] = np.sum(I * np.exp(1j * phase)) * dx * dy               # Eq. (108)
    return out


def normalised_amplitude(V, V0):
    """Eq. (109): |V(u, v)| / |V(0, 0)|."""
    return np.abs(V) / np.abs(V0)
