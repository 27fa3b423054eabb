"""Pins for the oracle's outer stationary-limit surface R_s(theta), the
largest root of R^2 H(R) + chi^2 cos^2 theta = 0 (Sec. 2.3, Eqs. 38-41).

- Kerr: R_s = 1 + sqrt(1 - chi^2 cos^2 theta) in closed form.
- At the poles Eq. (40) is the horizon condition (Eq. 33): R_s = R_+.
- On the equator Eq. (40) reduces to H(R_s) = 0 (Eq. 41): R_s is the largest
  zero of the lapse, found here by scipy's brentq on a bracket of its own.
- R_+ <= R_s(theta) <= R_s(pi/2) (the ergoregion of Eq. 42 is non-empty off
  the poles and widest on the equator), and g_TT of the metric vanishes at
  R_s (Eq. 38).
"""
import math

import numpy as np
import pytest

SPACES = [(1, dict(lam_E=0.3), 0.5), (1, dict(lam_E=0.1), 0.9),
          (2, dict(eta=0.02, lam_c=10.0), 0.9), (2, dict(eta=0.2, lam_c=10.0), 1.05)]


@pytest.mark.parametrize("chi", [0.0, 0.3, 0.7, 0.95, 0.999])
def test_kerr_closed_form(oracle, chi):
    P = oracle.problem(metric=oracle.KERR, chi=chi)
    for th in np.linspace(0.0, math.pi, 13):
        rs = oracle.ergosurface(P, th)
        assert rs == pytest.approx(1.0 + math.sqrt(1.0 - chi * chi * math.cos(th) ** 2),
                                   rel=1e-14, abs=1e-14)


@pytest.mark.parametrize("metric,halo,chi", SPACES)
def test_poles_equator_and_ordering(oracle, metric, halo, chi):
    from scipy.optimize import brentq
    P = oracle.problem(metric=metric, chi=chi, **halo)
    rp = oracle.horizon(P)
    assert oracle.ergosurface(P, 0.0) == pytest.approx(rp, rel=1e-14)
    assert oracle.ergosurface(P, math.pi) == pytest.approx(rp, rel=1e-14)
    # the largest zero of H: H > 0 beyond it up to R = 50
    grid = np.linspace(50.0, 0.05, 20000)
    h = np.array([oracle.H(P, r) for r in grid])
    k = int(np.argmax(h <= 0.0))
    r_eq = brentq(lambda r: oracle.H(P, r), grid[k], grid[k - 1], xtol=1e-15, rtol=1e-15)
    rs_eq = oracle.ergosurface(P, 0.5 * math.pi)
    assert rs_eq == pytest.approx(r_eq, rel=1e-13)
    prev = rp
    for th in np.linspace(0.0, 0.5 * math.pi, 9)[1:]:
        rs = oracle.ergosurface(P, th)
        assert prev - 1e-14 <= rs <= rs_eq + 1e-14
        prev = rs
        assert abs(oracle.metric(P, rs, th)[0, 0]) < 1e-12   # g_TT = 0 there (Eq. 38)


def test_no_horizon_no_polar_surface(oracle):
    P = oracle.problem(metric=oracle.EINASTO, chi=0.7, lam_E=0.3)   # above chi_e = 0.640
    assert oracle.horizon(P) is None
    assert oracle.ergosurface(P, 0.0) is None
    # the equatorial static limit does not depend on the spin (Eq. 41)
    assert oracle.ergosurface(P, 0.5 * math.pi) == pytest.approx(
        oracle.ergosurface(oracle.problem(metric=oracle.EINASTO, chi=0.0, lam_E=0.3),
                           0.5 * math.pi), rel=1e-15)
