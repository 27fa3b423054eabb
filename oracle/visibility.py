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


def amplitude_curves(I, x_min, x_max, y_min, y_max, q, n_phi):
    """Fourier-domain summaries of Sec. 6.4: for each q, the azimuthally
    averaged normalised amplitude (Eq. 109 averaged over the position angle)
    and the horizontal cut |V(q, 0)| / |V(0, 0)|.

    Reading: the average is over the amplitude, not over the complex
    visibility, taken by the midpoint rule at phi_k = (k + 1/2) pi / n_phi,
    k < n_phi (|V(-u, -v)| = |V(u, v)| for a real image, so [0, pi) covers the
    circle).  Returns (V_avg, V_cut)."""
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    V0 = visibilities(I, x_min, x_max, y_min, y_max, [[0.0, 0.0]])[0]
    phi = (np.arange(n_phi) + 0.5) * np.pi / n_phi
    avg = np.empty(q.shape[0])
    cut = np.empty(q.shape[0])
    for j, qj in enumerate(q):
        uv = np.stack([qj * np.cos(phi), qj * np.sin(phi)], 1)
        amp = normalised_amplitude(visibilities(I, x_min, x_max, y_min, y_max, uv), V0)
        avg[j] = np.mean(amp)
        cut[j] = normalised_amplitude(
            visibilities(I, x_min, x_max, y_min, y_max, [[qj, 0.0]])[0], V0)
    return avg, cut
