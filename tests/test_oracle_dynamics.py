"""Pins for the oracle's launch, Hamiltonian right-hand side and integrator.

- ZAMO tetrad orthonormality and launch nullity (Sec. 3.2, statements after
  Eqs. 69 and 73), closed forms of E and ell derived from Eqs. (63)-(74).
- Hamilton's equations (Eqs. 46-47, 57-62) against finite differences of the
  oracle's own Hamiltonian (Eq. 54).
- Dormand-Prince 5(4): textbook ODEs with exact solutions, and agreement of
  one step and of its dense output with scipy's RK45, an independent
  implementation of the same published method.
"""
import math

import numpy as np
import pytest


def test_zamo_tetrad_orthonormal(oracle):
    for metric, kw in [(0, {}), (1, dict(lam_E=0.1)), (2, dict(eta=0.02))]:
        P = oracle.problem(metric=metric, chi=0.9, incl=math.radians(80.0), r_obs=1000.0)
        for Ro in [1000.0, 15.0]:
            P.r_obs = Ro
            g = oracle.metric(P, Ro, P.incl)
            w = -g[0, 3] / g[3, 3]
            N = math.sqrt(-(g[0, 0] + 2 * w * g[0, 3] + w * w * g[3, 3]))
            u = np.array([1 / N, 0, 0, w / N])
            e = [np.array([0, 1 / math.sqrt(g[1, 1]), 0, 0]),
                 np.array([0, 0, 1 / math.sqrt(g[2, 2]), 0]),
                 np.array([0, 0, 0, 1 / math.sqrt(g[3, 3])])]
            assert u @ g @ u == pytest.approx(-1.0, abs=1e-14)
            for a in range(3):
                assert u @ g @ e[a] == pytest.approx(0.0, abs=1e-14)
                for b in range(3):
                    assert e[a] @ g @ e[b] == pytest.approx(float(a == b), abs=1e-14)
            L = oracle.launch(P, 3.0, -2.0)
            assert np.allclose(L["u_o"], u, rtol=1e-15, atol=0)


@pytest.mark.parametrize("metric,kw", [(0, {}), (1, dict(lam_E=0.1)), (2, dict(eta=0.02))])
def test_launch_is_null_and_matches_closed_forms(oracle, metric, kw):
    P = oracle.problem(metric=metric, chi=0.7, incl=math.radians(50.0), **kw)
    Ro, th = P.r_obs, P.incl
    g = oracle.metric(P, Ro, th)
    w = -g[0, 3] / g[3, 3]
    N = math.sqrt(-(g[0, 0] + w * g[0, 3]))
    for X, Y in [(0.3, 0.2), (-7.0, 4.0), (11.0, -11.0)]:
        L = oracle.launch(P, X, Y)
        y0, E, ell = L["y0"], L["E"], L["ell"]
        p = np.array([-E, y0[4], y0[5], ell])
        assert abs(oracle.two_hamiltonian(P, Ro, th, p)) < 1e-13
        d = math.sqrt(Ro * Ro + X * X + Y * Y)
        assert ell == pytest.approx(math.sqrt(g[3, 3]) * (-X / d), rel=1e-13)
        assert E == pytest.approx(N + w * ell, rel=1e-13)
        assert y0[4] == pytest.approx(math.sqrt(g[1, 1]) * (-Ro / d), rel=1e-13)
        assert y0[5] == pytest.approx(math.sqrt(g[2, 2]) * (-Y / d), rel=1e-13)
        # locally measured photon energy is E_loc = 1 (Eq. 73)
        assert -(p[0] * L["u_o"][0] + p[3] * L["u_o"][3]) == pytest.approx(1.0, abs=1e-14)


def test_screen_matches_bardeen_celestial_coordinates(oracle):
    """Far observer: X ~ alpha = -xi / sin(theta_o) to O(1/R_o) (Sec. 3.2)."""
    a = 0.5
    P = oracle.problem(metric=oracle.KERR, chi=a, incl=math.radians(60.0), r_obs=1e6)
    for X, Y in [(4.0, 1.0), (-3.0, -5.0)]:
        L = oracle.launch(P, X, Y)
        xi = L["ell"] / L["E"]
        K = oracle.carter(P, L["E"], L["ell"], P.incl, L["y0"][5]) / L["E"] ** 2
        eta = K - (xi - a) ** 2
        th = P.incl
        alpha = -xi / math.sin(th)
        beta2 = eta + a * a * math.cos(th) ** 2 - xi * xi / math.tan(th) ** 2
        assert alpha == pytest.approx(X, rel=1e-5)
        assert math.sqrt(beta2) == pytest.approx(abs(Y), rel=1e-5)


def _fd(f, x, h):
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


@pytest.mark.parametrize("metric,kw", [(0, {}), (1, dict(lam_E=0.1)), (2, dict(eta=0.02))])
def test_hamilton_equations_against_finite_differences(oracle, metric, kw):
    rng = np.random.default_rng(7)
    P = oracle.problem(metric=metric, chi=0.8, **kw)
    rp = oracle.horizon(P)
    for _ in range(20):
        R = rp * (1.1 + 15 * rng.random())
        th = 0.1 + (math.pi - 0.2) * rng.random()
        E, ell, pR, pth = 1.0, rng.normal() * 3, rng.normal(), rng.normal() * 2
        y = np.array([0.0, R, th, 0.0, pR, pth])
        dy = oracle.rhs(P, E, ell, y)

        def Hm(R_=R, th_=th, pT=-E, pR_=pR, pth_=pth, pph=ell):
            return 0.5 * oracle.two_hamiltonian(P, R_, th_, [pT, pR_, pth_, pph])

        ref = [
            _fd(lambda v: Hm(pT=v), -E, 1e-4),          # dT/dl = dH/dp_T
            _fd(lambda v: Hm(pR_=v), pR, 1e-4),          # dR/dl
            _fd(lambda v: Hm(pth_=v), pth, 1e-4),        # dth/dl
            _fd(lambda v: Hm(pph=v), ell, 1e-4),         # dphi/dl
            -_fd(lambda v: Hm(R_=v), R, 1e-5 * R),       # dp_R/dl = -dH/dR
            -_fd(lambda v: Hm(th_=v), th, 1e-5),         # dp_th/dl = -dH/dth
        ]
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.allclose(dy, ref, rtol=1e-7, atol=1e-8 * scale)


def test_dp5_exponential(oracle):
    y, n = oracle.dp5_solve(0, [1.0], 0.0, 5.0, 1e-10, 1e-12)
    assert n > 0
    assert y[0] == pytest.approx(math.exp(5.0), rel=3e-9)


def test_dp5_oscillator_and_kepler(oracle):
    w = 3.0
    y, n = oracle.dp5_solve(1, [1.0, 0.0], 0.0, 10.0, 1e-10, 1e-12, w=w)
    assert y[0] == pytest.approx(math.cos(w * 10.0), abs=5e-8)
    assert y[1] == pytest.approx(-w * math.sin(w * 10.0), abs=5e-7)
    # Kepler ellipse e = 0.5 (a = 1, period 2 pi): returns to perihelion.
    e = 0.5
    y0 = [1 - e, 0.0, 0.0, math.sqrt((1 + e) / (1 - e))]
    y, n = oracle.dp5_solve(2, y0, 0.0, 2 * math.pi, 1e-11, 1e-13)
    assert np.allclose(y, y0, atol=1e-8)


def test_dp5_local_order(oracle):
    """One step of a 5th-order method: local error O(h^6); the embedded
    estimate O(h^5); the dense output at mid-step O(h^5)."""
    errs, ests, dens = [], [], []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        y1, err, dense = oracle.dp5_step_dense(0, [1.0], h, [0.5])
        errs.append(abs(y1[0] - math.exp(h)))
        ests.append(abs(err[0]))
        dens.append(abs(dense[0, 0] - math.exp(0.5 * h)))
    for arr, order in [(errs, 6), (ests, 5), (dens, 5)]:
        ratio = math.log2(arr[1] / arr[2])
        assert ratio == pytest.approx(order, abs=0.35)


def test_dp5_step_and_dense_output_match_scipy(oracle):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    w = 2.0
    y0 = np.array([0.3, -1.1])
    h = 0.37

    def f(t, y):
        return [y[1], -w * w * y[0]]

    s = scipy_integrate.RK45(f, 0.0, y0, t_bound=10.0, first_step=h, rtol=1e3, atol=1e3)
    s.step()
    assert s.t == pytest.approx(h, rel=1e-15)
    sig = np.array([0.1, 0.25, 0.5, 0.8, 1.0])
    y1, err, dense = oracle.dp5_step_dense(1, y0, h, sig, w=w)
    assert np.allclose(y1, s.y, rtol=1e-14, atol=1e-15)
    interp = s.dense_output()
    for k, sg in enumerate(sig):
        assert np.allclose(dense[k], interp(sg * h), rtol=1e-12, atol=1e-14)
