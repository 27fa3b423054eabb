"""Pins for the oracle pieces that the adjoint parity test leans on: the
frozen-step replay (trace_points_record / trace_points_frozen) and the smooth
bright-ring radius (rho_peak_smooth, a differentiable reading of Eq. 105).

- Replaying a ray's recorded accepted steps with the same parameters gives
  the adaptive result bit for bit (the replay is the adaptive algorithm with
  its step decisions held, nothing else; it has no termination test, so only
  its status word differs).
- Emission parameters do not move the geodesic, so the frozen derivative of
  I with respect to them has closed forms in the recorded crossings:
  dI/dj0 = I/j0 (Eq. 83 is linear in j0) and
  dI/dR_s = sum_n I_n (R_em,n - R_in) / R_s^2 (the exp(-(rho-R_in)/R_s) factor).
- A geometric derivative (dR_em/dchi) of the frozen replay at
  rtol 1e-10 agrees with the derivative of the exact flow, approximated by
  central differences of fully adaptive traces at rtol 1e-13 with a step
  large enough that their step-selection noise is negligible.
- rho_peak_smooth returns the exact vertex when the bin means lie on a
  parabola, and the bin centre at the ends of the profile.
"""
import math

import numpy as np
import pytest

from oracle.diagnostics import rho_peak_smooth, screen_centres

RAYS = np.array([[3.1, 4.0], [-5.2, 1.7], [6.4, -2.2], [0.9, 7.3], [-7.5, -4.8],
                 [4.6, 5.9], [-2.4, -6.1], [8.8, 0.4], [-6.9, 6.2], [5.5, -5.1]])


@pytest.mark.parametrize("metric,halo", [(0, {}), (1, dict(lam_E=0.1)),
                                         (2, dict(eta=0.02, lam_c=10.0))])
def test_frozen_replay_is_bitwise_adaptive(oracle, metric, halo):
    P = oracle.problem(metric=metric, chi=0.7, incl=math.radians(50.0), **halo)
    adaptive = oracle.trace_points(P, RAYS)
    rec, hbuf, counts = oracle.trace_points_record(P, RAYS)
    replay = oracle.trace_points_frozen(P, RAYS, hbuf, counts)
    for f in ("status", "ncross", "I_tot", "I_n", "R_em", "phi_em", "g", "n_accept"):
        assert np.array_equal(adaptive[f], rec[f]), f
    # the replay has no termination test (its status stays "undetermined"),
    # but it stops after the same accepted step, at the same radius
    for f in ("ncross", "I_tot", "I_n", "R_em", "phi_em", "g", "n_accept", "R_final"):
        assert np.array_equal(adaptive[f], replay[f]), f
    assert np.all(counts == adaptive["n_accept"])


def test_frozen_emission_derivatives_closed_form(oracle):
    P = oracle.problem(metric=2, chi=0.9, incl=math.radians(60.0), eta=0.02, lam_c=10.0)
    rec, hbuf, counts = oracle.trace_points_record(P, RAYS)
    R_in = oracle.geometry(P)["R_in"]
    keep = (rec["ncross"] >= 1) & (rec["ncross"] <= 3) & (rec["I_tot"] > 0)
    assert keep.sum() >= 4

    def frozen(**kw):
        return oracle.trace_points_frozen(oracle.problem(
            metric=2, chi=0.9, incl=math.radians(60.0), eta=0.02, lam_c=10.0, **kw),
            RAYS, hbuf, counts)

    h = 1e-5
    Ip, Im = frozen(j0=1.0 + h)["I_tot"], frozen(j0=1.0 - h)["I_tot"]
    dj0 = (Ip - Im) / (2 * h)
    assert np.allclose(dj0[keep], rec["I_tot"][keep], rtol=1e-9)

    Rs = 8.0
    Ip, Im = frozen(R_s=Rs + h)["I_tot"], frozen(R_s=Rs - h)["I_tot"]
    dRs = (Ip - Im) / (2 * h)
    closed = np.sum(rec["I_n"] * (rec["R_em"] - R_in), axis=1) / Rs ** 2
    assert np.allclose(dRs[keep], closed[keep], rtol=1e-7, atol=1e-12)


def test_frozen_geometric_derivative_matches_exact_flow(oracle):
    base = dict(metric=0, chi=0.6, incl=math.radians(40.0))
    pts = RAYS[:6]
    P = oracle.problem(**base)
    rec, hbuf, counts = oracle.trace_points_record(P, pts)
    h_f, h_a = 1e-6, 2e-4
    fp = oracle.trace_points_frozen(oracle.problem(**dict(base, chi=0.6 + h_f)), pts, hbuf, counts)
    fm = oracle.trace_points_frozen(oracle.problem(**dict(base, chi=0.6 - h_f)), pts, hbuf, counts)
    d_frozen = (fp["R_em"][:, 0] - fm["R_em"][:, 0]) / (2 * h_f)
    tight = dict(base, rtol=1e-13, atol=1e-15)
    ap = oracle.trace_points(oracle.problem(**dict(tight, chi=0.6 + h_a)), pts)
    am = oracle.trace_points(oracle.problem(**dict(tight, chi=0.6 - h_a)), pts)
    d_exact = (ap["R_em"][:, 0] - am["R_em"][:, 0]) / (2 * h_a)
    ok = (rec["ncross"] >= 1) & (ap["ncross"] == rec["ncross"]) & (am["ncross"] == rec["ncross"])
    assert ok.sum() >= 4
    scale = np.max(np.abs(d_exact[ok]))
    assert np.allclose(d_frozen[ok], d_exact[ok], rtol=1e-5, atol=1e-6 * scale)


def test_rho_peak_smooth_exact_vertex():
    n, ext = 96, 12.0
    X, Y, dx, _ = screen_centres(n, n, -ext, ext, -ext, ext)
    XX, YY = np.meshgrid(X, Y)
    b = np.floor(np.sqrt(XX ** 2 + YY ** 2) / dx)
    for r0 in (5.3, 7.0 * dx + 0.5 * dx, 4.0 * dx + 0.8 * dx):
        I = 50.0 - ((b + 0.5) * dx - r0) ** 2       # bin means lie on a parabola
        assert rho_peak_smooth(I, -ext, ext, -ext, ext) == pytest.approx(r0, rel=1e-12)
    I = np.exp(-np.hypot(XX, YY))                    # peak in the first bin: no neighbour
    assert rho_peak_smooth(I, -ext, ext, -ext, ext) == 0.5 * dx
