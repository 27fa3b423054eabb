"""Pins for the oracle's spacetime layer: lapses, metric, inverse metric,
horizon, extremal spin, circular orbits, ISCO and emissivity.

Each check ties the oracle to something other than itself: a closed form
(Kerr horizon, Kerr Omega, Bardeen-Press-Teukolsky ISCO), a limit the paper
states (Kerr and static limits after Eq. 26, eta = 0 cored-NFW), an identity
(g g^-1 = 1), finite differences of the oracle's own functions, or a number
the paper prints (extremal spins of Fig. 2).
"""
import math

import numpy as np
import pytest

from paper_values import load as load_paper

pytestmark = pytest.mark.filterwarnings("ignore")


def fd(f, x, h):
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


@pytest.mark.parametrize("chi", [0.0, 0.3, 0.5, 0.9, 0.98, 0.999])
def test_kerr_horizon_closed_form(oracle, chi):
    P = oracle.problem(metric=oracle.KERR, chi=chi)
    assert oracle.horizon(P) == pytest.approx(1 + math.sqrt(1 - chi * chi), rel=1e-14, abs=1e-14)


def test_kerr_superextremal_has_no_horizon(oracle):
    assert oracle.horizon(oracle.problem(metric=oracle.KERR, chi=1.01)) is None
    # Einasto lam_E = 0.3 is horizonless above chi_e = 0.6396 (Fig. 2).
    assert oracle.horizon(oracle.problem(metric=oracle.EINASTO, lam_E=0.3, chi=0.7)) is None
    assert oracle.horizon(oracle.problem(metric=oracle.EINASTO, lam_E=0.3, chi=0.6)) is not None


@pytest.mark.parametrize("metric,kw", [(1, dict(lam_E=0.1)), (1, dict(lam_E=0.3)),
                                       (2, dict(eta=0.02, lam_c=10.0)),
                                       (2, dict(eta=0.2, lam_c=10.0))])
@pytest.mark.parametrize("chi", [0.0, 0.5])
def test_horizon_is_largest_root(oracle, metric, kw, chi):
    P = oracle.problem(metric=metric, chi=chi, **kw)
    rp = oracle.horizon(P)
    scale = rp * rp
    assert abs(oracle.Delta(P, rp)) < 1e-12 * scale
    for R in np.linspace(rp * (1 + 1e-9), 60.0, 4000):
        assert oracle.Delta(P, R) > 0.0


def test_extremal_spins_printed_in_paper(oracle):
    paper = load_paper()
    ck, _ = oracle.extremal_spin(oracle.problem(metric=oracle.KERR))
    ce, Re = oracle.extremal_spin(oracle.problem(metric=oracle.EINASTO, lam_E=0.3))
    cc, Rc = oracle.extremal_spin(oracle.problem(metric=oracle.CNFW, eta=0.2, lam_c=10.0))
    assert ck == pytest.approx(paper["chi_e_kerr"][0], abs=5e-4)
    assert ce == pytest.approx(paper["chi_e_einasto_lamE0.3"][0], abs=5e-4)
    assert cc == pytest.approx(paper["chi_e_cnfw_eta0.2_lamc10"][0], abs=5e-4)
    # Eq. (36) holds at the extremal radius, and Delta has a double root there (Eq. 34).
    for P, R in [(oracle.problem(metric=1, lam_E=0.3), Re), (oracle.problem(metric=2, eta=0.2), Rc)]:
        assert 2 * oracle.H(P, R) + R * oracle.dH(P, R) == pytest.approx(0.0, abs=1e-7)


def test_extremal_spin_separates_black_holes(oracle):
    for P in [oracle.problem(metric=1, lam_E=0.1), oracle.problem(metric=2, eta=0.02)]:
        ce, _ = oracle.extremal_spin(P)
        P.chi = ce - 1e-4
        assert oracle.horizon(P) is not None
        P.chi = ce + 1e-4
        assert oracle.horizon(P) is None


@pytest.mark.parametrize("metric,kw", [(0, {}), (1, dict(lam_E=0.1)), (1, dict(lam_E=0.7)),
                                       (2, dict(eta=0.02, lam_c=10.0)),
                                       (2, dict(eta=0.3, lam_c=3.0))])
def test_lapse_derivative_matches_finite_difference(oracle, metric, kw):
    P = oracle.problem(metric=metric, **kw)
    for R in [0.3, 1.0, 1.7, 2.5, 4.0, 11.0, 150.0]:
        num = fd(lambda r: oracle.H(P, r), R, 1e-4 * R)
        assert oracle.dH(P, R) == pytest.approx(num, rel=1e-8, abs=1e-11)


def test_lapse_limits(oracle):
    # eta = 0: the cored-NFW lapse (Eq. 13) is exactly Schwarzschild.
    P0 = oracle.problem(metric=oracle.CNFW, eta=0.0, lam_c=10.0)
    K = oracle.problem(metric=oracle.KERR)
    for R in [0.5, 2.0, 7.3, 1000.0]:
        assert oracle.H(P0, R) == oracle.H(K, R)
        assert oracle.dH(P0, R) == oracle.dH(K, R)
    # Einasto: Schwarzschild recovered at large radius (Sec. 2.1) and the
    # mass function vanishes at the regular centre.
    PE = oracle.problem(metric=oracle.EINASTO, lam_E=0.3)
    assert oracle.H(PE, 50.0) == pytest.approx(1 - 2 / 50.0, abs=1e-60)
    assert oracle.mu(PE, 1e-3) < 1e-6
    assert oracle.mu(PE, 40.0) == pytest.approx(1.0, abs=1e-12)
    # Small lam_E: indistinguishable from Kerr outside the horizon.
    PS = oracle.problem(metric=oracle.EINASTO, lam_E=0.05)
    for R in [1.5, 2.0, 3.0]:
        assert abs(oracle.H(PS, R) - (1 - 2 / R)) < 2e-7


@pytest.mark.parametrize("metric,kw", [(0, {}), (1, dict(lam_E=0.1)), (2, dict(eta=0.02))])
def test_metric_times_inverse_is_identity(oracle, metric, kw):
    rng = np.random.default_rng(1)
    P = oracle.problem(metric=metric, chi=0.7, **kw)
    rp = oracle.horizon(P)
    for _ in range(50):
        R = rp * (1.05 + 20 * rng.random())
        th = 0.05 + (math.pi - 0.1) * rng.random()
        g = oracle.metric(P, R, th)
        gi = oracle.metric_inv(P, R, th)
        assert np.allclose(g @ gi, np.eye(4), atol=1e-12, rtol=0)


def test_kerr_metric_is_textbook_boyer_lindquist(oracle):
    """Kerr limit stated after Eq. (26): the Boyer-Lindquist Kerr metric."""
    a = 0.8
    P = oracle.problem(metric=oracle.KERR, chi=a)
    for r, th in [(3.0, 0.4), (7.5, 1.3), (2.1, 2.8)]:
        S = r * r + a * a * math.cos(th) ** 2
        D = r * r - 2 * r + a * a
        s2 = math.sin(th) ** 2
        ref = np.zeros((4, 4))
        ref[0, 0] = -(1 - 2 * r / S)
        ref[0, 3] = ref[3, 0] = -2 * a * r * s2 / S
        ref[1, 1] = S / D
        ref[2, 2] = S
        ref[3, 3] = (r * r + a * a + 2 * a * a * r * s2 / S) * s2
        assert np.allclose(oracle.metric(P, r, th), ref, rtol=1e-14, atol=1e-14)


def test_static_limit_is_seed_metric(oracle):
    """chi -> 0 reduces Eq. (26) to the static seed, Eq. (3)."""
    P = oracle.problem(metric=oracle.CNFW, chi=0.0, eta=0.05, lam_c=5.0)
    for R, th in [(2.5, 0.7), (9.0, 1.9)]:
        H = oracle.H(P, R)
        g = oracle.metric(P, R, th)
        assert g[0, 0] == pytest.approx(-H, rel=1e-14)
        assert g[1, 1] == pytest.approx(1 / H, rel=1e-14)
        assert g[2, 2] == pytest.approx(R * R, rel=1e-14)
        assert g[3, 3] == pytest.approx(R * R * math.sin(th) ** 2, rel=1e-14)
        assert g[0, 3] == 0.0


@pytest.mark.parametrize("metric,kw", [(0, {}), (1, dict(lam_E=0.1)), (2, dict(eta=0.02))])
def test_metric_derivatives_match_finite_differences(oracle, metric, kw):
    P = oracle.problem(metric=metric, chi=0.6, **kw)
    for R, th in [(2.3, 0.5), (4.0, 1.2), (9.0, 1.5707), (30.0, 2.6)]:
        dR, dth = oracle.dmetric_inv(P, R, th)
        nR = fd(lambda r: oracle.metric_inv(P, r, th), R, 1e-4 * R)
        nth = fd(lambda t: oracle.metric_inv(P, R, t), th, 1e-4)
        assert np.allclose(dR, nR, rtol=1e-7, atol=1e-10)
        assert np.allclose(dth, nth, rtol=1e-7, atol=1e-10)
        dg = oracle.dmetric_dR(P, R, th)
        ng = fd(lambda r: oracle.metric(P, r, th), R, 1e-4 * R)
        assert np.allclose(dg, ng, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("chi", [0.0, 0.3, 0.9])
def test_kerr_keplerian_omega_and_ut(oracle, chi):
    """Eq. (91) reduces to 1/(R^{3/2} + chi) for Kerr (Bardeen, Press &
    Teukolsky 1972), with u^T = (R^{3/2}+chi)/sqrt(R^{3/2}(R^{3/2}-3R^{1/2}+2chi))."""
    P = oracle.problem(metric=oracle.KERR, chi=chi)
    for R in [4.0, 6.5, 12.0, 40.0]:
        W, uT = oracle.circular(P, R)
        assert W == pytest.approx(1 / (R ** 1.5 + chi), rel=1e-13)
        ref = (R ** 1.5 + chi) / math.sqrt(R ** 1.5 * (R ** 1.5 - 3 * R ** 0.5 + 2 * chi))
        assert uT == pytest.approx(ref, rel=1e-12)


def _bpt_isco(a):
    z1 = 1 + (1 - a * a) ** (1 / 3) * ((1 + a) ** (1 / 3) + (1 - a) ** (1 / 3))
    z2 = math.sqrt(3 * a * a + z1 * z1)
    return 3 + z2 - math.sqrt((3 - z1) * (3 + z1 + 2 * z2))


@pytest.mark.parametrize("chi", [0.0, 0.5, 0.7, 0.9, 0.94])
def test_kerr_isco_closed_form(oracle, chi):
    P = oracle.problem(metric=oracle.KERR, chi=chi)
    assert oracle.isco(P) == pytest.approx(_bpt_isco(chi), abs=2e-7)


def test_dark_matter_isco_is_energy_minimum(oracle):
    """For the dressed metrics the ISCO has dE/dR = 0 with E minimal."""
    for P in [oracle.problem(metric=1, lam_E=0.1, chi=0.9), oracle.problem(metric=2, chi=0.94)]:
        r = oracle.isco(P)

        def energy(R):
            W, uT = oracle.circular(P, R)
            g = oracle.metric(P, R, math.pi / 2)
            return -uT * (g[0, 0] + W * g[0, 3])

        e0 = energy(r)
        assert energy(r * (1 + 1e-3)) > e0 and energy(r * (1 - 1e-3)) > e0


def test_emissivity_profile(oracle):
    """Eqs. (83)-(86): tapers are 1/2 at their edges; vertical Gaussian."""
    P = oracle.problem(j0=2.0, p=2.0, R_s=8.0, sigma_in=0.2, sigma_out=2.0, R_out=20.0,
                       H0=0.05, h=0.05)
    Rin = 4.0
    j = oracle.emissivity(P, Rin, Rin, math.pi / 2)
    assert j == pytest.approx(2.0 * 0.5 * 0.5 * (1 - math.tanh((Rin - 20.0) / 2.0)), rel=1e-14)
    # sharp-taper limit: nothing inside R_in
    Ps = oracle.problem(sigma_in=1e-6, sigma_out=1e-6)
    assert oracle.emissivity(Ps, Rin, 3.9, math.pi / 2) == 0.0
    R = 10.0
    jr = oracle.emissivity(Ps, Rin, R, math.pi / 2)
    assert jr == pytest.approx((R / Rin) ** -2 * math.exp(-(R - Rin) / 8.0), rel=1e-13)
    # off-plane: rho = R sin th, z = R cos th, H = H0 + h rho
    th = math.pi / 2 - 0.01
    rho, z = R * math.sin(th), R * math.cos(th)
    Hd = 0.05 + 0.05 * rho
    ref = (rho / Rin) ** -2 * math.exp(-(rho - Rin) / 8.0) * math.exp(-z * z / (2 * Hd * Hd))
    assert oracle.emissivity(Ps, Rin, R, th) == pytest.approx(ref, rel=1e-12)
