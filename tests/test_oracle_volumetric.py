"""Pins for the oracle's volumetric intensity, the paper's I = int g^3 j dlambda
over the finite-thickness emitting layer (Eqs. 83-88), integrated as a
seventh ODE component by the same Dormand-Prince steps.

- Thin-layer limit: with the Gaussian vertical profile exp(-z^2 / 2 H^2) and
  H -> 0, the integral across the layer at each equatorial crossing tends to
  g^3 j(R_em, z = 0) sqrt(2 pi) H(R_em) / |dz/dlambda|, |dz/dlambda| =
  R_em |dtheta/dlambda| on the plane.  The thin-disk mode records g^3 j, R_em
  and dtheta/dlambda per crossing by a separate code path (event root finding
  instead of quadrature), so the sum over crossings checks the quadrature,
  the source term and the layer step cap together.
- Convergence: rtol 1e-10 and 1e-12 give the same integral to 1e-8.
- Linearity in j0 (Eq. 83), to the step-selection noise.
- The volumetric mode does not change the fate, the crossing count or the
  transfer radius of a ray (the geodesic is the same; only the steps differ).
"""
import math

import numpy as np
import pytest

PTS = np.array([[3.1, 4.0], [-5.2, 1.7], [6.4, -2.2], [0.9, 7.3], [-7.5, -4.8],
                [4.6, 5.9], [-2.4, -6.1], [8.8, 0.4]])


def _thin_limit(thin, H0, h):
    out = np.zeros(len(thin))
    for k, r in enumerate(thin):
        for n in range(min(int(r["ncross"]), 3)):
            Hc = H0 + h * r["R_em"][n]                       # Eq. (84) at z = 0
            out[k] += r["I_n"][n] * math.sqrt(2 * math.pi) * Hc / (r["R_em"][n] * abs(r["thdot"][n]))
    return out


@pytest.mark.parametrize("metric,halo", [(0, {}), (2, dict(eta=0.02, lam_c=10.0))])
@pytest.mark.parametrize("H0,h", [(1e-3, 0.0), (1e-4, 0.0), (1e-4, 2e-4)])
def test_thin_layer_limit(oracle, metric, halo, H0, h):
    base = dict(metric=metric, chi=0.7, incl=math.radians(60.0), r_in_mode=1, **halo)
    thin = oracle.trace_points(oracle.problem(**base), PTS)
    vol = oracle.trace_points(oracle.problem(**base, volumetric=1, H0=H0, h=h), PTS)
    keep = (thin["ncross"] >= 1) & (thin["ncross"] <= 3)
    assert keep.sum() >= 5
    pred = _thin_limit(thin, H0, h)
    assert np.allclose(vol["I_tot"][keep], pred[keep], rtol=2e-6, atol=0.0)
    # no event intensity in volumetric mode
    assert np.all(vol["I_n"] == 0.0)


def test_convergence_and_linearity(oracle):
    base = dict(metric=1, lam_E=0.1, chi=0.9, incl=math.radians(30.0), volumetric=1)
    a = oracle.trace_points(oracle.problem(**base), PTS)
    b = oracle.trace_points(oracle.problem(**base, rtol=1e-12, atol=1e-14), PTS)
    assert np.all(a["I_tot"] > 0)
    assert np.allclose(a["I_tot"], b["I_tot"], rtol=1e-8, atol=0.0)
    c = oracle.trace_points(oracle.problem(**base, j0=2.0), PTS)
    assert np.allclose(c["I_tot"], 2.0 * a["I_tot"], rtol=1e-9, atol=0.0)


def test_geodesic_unchanged_by_volumetric_mode(oracle):
    base = dict(metric=0, chi=0.5, incl=math.radians(17.0))
    thin = oracle.trace_points(oracle.problem(**base), PTS)
    vol = oracle.trace_points(oracle.problem(**base, volumetric=1), PTS)
    assert np.array_equal(thin["status"], vol["status"])
    assert np.array_equal(thin["ncross"], vol["ncross"])
    has = thin["ncross"] >= 1
    assert np.allclose(vol["R_em"][has, 0], thin["R_em"][has, 0], rtol=1e-8)
