"""Pins for the oracle's shadow-boundary search (Sec. 4.1, Eqs. 78-79):
bisection in the screen impact parameter b along each polar direction psi.

- Schwarzschild: a static observer at R_o sees the capture boundary at the
  angle sin(alpha) = sqrt(27 (1 - 2/R_o)) / R_o from the inward radial
  direction (critical impact parameter L/E = sqrt(27)); the screen of
  Eqs. 70-72 puts it at b = R_o tan(alpha), in every direction.
- Kerr: the textbook radial potential (Bardeen 1973) calls every returned
  bracket's captured end captured and its escaping end escaping, i.e. the
  bracket contains the analytic critical curve, at spin 0.9.
- Fig. 5 (chi = 0.5, i = 60 deg): the cored-NFW boundary lies outside the
  Kerr one in every direction and the Einasto one (lambda_E = 0.3) stays
  closer to Kerr than the cored-NFW one does.
- A bracket whose ends do not straddle the transition is flagged and
  returned unchanged.
"""
import math

import numpy as np
import pytest

from test_oracle_trace import kerr_radial_capture

PSI = np.linspace(0.0, 2.0 * math.pi, 24, endpoint=False)


@pytest.mark.parametrize("incl", [17.0, 60.0, 90.0])
def test_schwarzschild_closed_form(oracle, incl):
    P = oracle.problem(metric=oracle.KERR, chi=0.0, incl=math.radians(incl))
    Ro = P.r_obs
    b_c = Ro * math.tan(math.asin(math.sqrt(27.0 * (1.0 - 2.0 / Ro)) / Ro))
    tol = 1e-9
    r = oracle.shadow_boundary(P, PSI[::3], 2.0, 9.0, tol)
    assert np.all(r["flags"] == 0)
    assert np.all(r["b_out"] - r["b_in"] <= tol)
    # the bracket holds the closed form (up to the integration's own error)
    assert np.all(r["b_in"] <= b_c + 1e-9) and np.all(r["b_out"] >= b_c - 1e-9)


def test_kerr_bracket_contains_analytic_critical_curve(oracle):
    a = 0.9
    P = oracle.problem(metric=oracle.KERR, chi=a, incl=math.radians(60.0))
    geo = oracle.geometry(P)
    r = oracle.shadow_boundary(P, PSI, 1.0, 9.0, 1e-7)
    assert np.all(r["flags"] == 0)
    for key, want in (("b_in", True), ("b_out", False)):
        xy = np.stack([r[key] * np.cos(PSI), r[key] * np.sin(PSI)], 1)
        for ray in oracle.trace_points(P, xy):
            cap, margin = kerr_radial_capture(a, ray["E"], ray["ell"], ray["K0"], geo["r_plus"],
                                              P.r_obs)
            assert abs(margin) > 1e-12
            assert cap == want


def test_fig5_ordering(oracle):
    b = {}
    for name, kw in (("kerr", dict(metric=oracle.KERR)),
                     ("einasto", dict(metric=oracle.EINASTO, lam_E=0.3)),
                     ("cnfw", dict(metric=oracle.CNFW, eta=0.02, lam_c=10.0))):
        P = oracle.problem(chi=0.5, incl=math.radians(60.0), **kw)
        r = oracle.shadow_boundary(P, PSI, 1.0, 9.0, 1e-8)
        assert np.all(r["flags"] == 0)
        b[name] = 0.5 * (r["b_in"] + r["b_out"])
    assert np.all(b["cnfw"] > b["kerr"])
    assert np.max(np.abs(b["einasto"] - b["kerr"])) < np.min(b["cnfw"] - b["kerr"])


def test_unbracketed_transition_is_flagged(oracle):
    P = oracle.problem(metric=oracle.KERR, chi=0.5, incl=math.radians(30.0))
    r = oracle.shadow_boundary(P, PSI[:4], 6.5, 9.0, 1e-6)     # both ends escape
    assert np.all(r["flags"] & 1) and not np.any(r["flags"] & 2)
    assert np.all(r["b_in"] == 6.5) and np.all(r["b_out"] == 9.0)
    r = oracle.shadow_boundary(P, PSI[:4], 1.0, 2.5, 1e-6)     # both ends captured
    assert np.all(r["flags"] & 2) and not np.any(r["flags"] & 1)
    with pytest.raises(ValueError):
        oracle.shadow_boundary(P, PSI[:4], 3.0, 2.0, 1e-6)
