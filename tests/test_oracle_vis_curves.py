"""Pins for the oracle's visibility-amplitude curves (Sec. 6.4): the
azimuthally averaged normalised amplitude V(q) and the horizontal cut
|V(q, 0)| / |V(0, 0)|.

A shifted elliptical Gaussian, I = exp(-(X-x0)^2/2 sx^2 - (Y-y0)^2/2 sy^2),
sampled finely on a screen much wider than it: its continuous transform has
amplitude exp(-2 pi^2 (sx^2 u^2 + sy^2 v^2)), so
  cut(q) = exp(-2 pi^2 sx^2 q^2),
  avg(q) = (1/pi) int_0^pi exp(-2 pi^2 q^2 (sx^2 cos^2 + sy^2 sin^2)) dphi
         = exp(-pi^2 q^2 (sx^2 + sy^2)) I0(pi^2 q^2 (sx^2 - sy^2)),
with I0 the modified Bessel function.  The shift changes only the phase,
so averaging the complex visibility instead of its amplitude, or taking the
cut along v, fails these; q = 0 gives exactly 1.
"""
import math

import numpy as np
import pytest

from oracle.visibility import amplitude_curves


def _gaussian(n, ext, sx, sy, x0, y0):
    c = -ext + (np.arange(n) + 0.5) * (2 * ext / n)
    XX, YY = np.meshgrid(c, c)
    return np.exp(-0.5 * ((XX - x0) / sx) ** 2 - 0.5 * ((YY - y0) / sy) ** 2)


def test_elliptical_gaussian_closed_forms():
    from scipy.special import i0
    sx, sy = 1.2, 0.7
    I = _gaussian(160, 12.0, sx, sy, 0.8, -0.5)
    q = np.array([0.0, 0.05, 0.1, 0.2, 0.3])
    avg, cut = amplitude_curves(I, -12.0, 12.0, -12.0, 12.0, q, 64)
    a = math.pi ** 2 * q ** 2
    assert np.allclose(cut, np.exp(-2 * a * sx ** 2), rtol=1e-9, atol=1e-13)
    want = np.exp(-a * (sx ** 2 + sy ** 2)) * i0(a * (sx ** 2 - sy ** 2))
    assert np.allclose(avg, want, rtol=1e-9, atol=1e-13)
    assert avg[0] == 1.0 and cut[0] == 1.0


def test_isotropic_image_average_equals_cut():
    I = _gaussian(96, 10.0, 1.0, 1.0, 0.0, 0.0)
    q = np.linspace(0.0, 0.4, 9)
    avg, cut = amplitude_curves(I, -10.0, 10.0, -10.0, 10.0, q, 16)
    assert np.allclose(avg, cut, rtol=1e-10, atol=1e-14)
