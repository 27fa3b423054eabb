"""GPU horizon, extremal-spin and stationary-limit scan (Sec. 2.3, Eqs. 33-41)
through the C ABI, against the oracle and the Kerr closed forms.

Bar: R_+ and R_s(theta) within 1e-12 relative of the oracle's away from the
extremal boundary (|chi| < chi_e - 1e-3, where the roots are simple), chi_e
within 1e-12 relative, R_e within 1e-7 (the oracle locates the maximiser by
golden section, to about sqrt(eps)); flags exact.  Kerr: R_+ = 1 +
sqrt(1 - chi^2), chi_e = R_e = 1, R_s = 1 + sqrt(1 - chi^2 cos^2 theta).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


THETA = np.linspace(0.0, math.pi, 7)


def _np(res):
    return {k: v.cpu().numpy() for k, v in res.items()}


def test_kerr_closed_forms(B):
    chis = np.linspace(-0.999, 0.999, 1037)           # ragged count
    res = _np(B.geometry_scan([B.Spacetime(metric=B.KERR, chi=float(c)) for c in chis], THETA))
    assert np.all(res["flags"] == 0)
    assert np.allclose(res["r_plus"], 1.0 + np.sqrt(1.0 - chis ** 2), rtol=1e-13, atol=0)
    assert np.allclose(res["chi_e"], 1.0, rtol=1e-13)
    assert np.allclose(res["R_e"], 1.0, rtol=1e-9)
    want = 1.0 + np.sqrt(1.0 - np.outer(chis ** 2, np.cos(THETA) ** 2))
    assert np.allclose(res["R_s"], want, rtol=1e-13, atol=0)


def test_mixed_families_against_oracle(B, oracle):
    rng = np.random.default_rng(20261203)
    sts, probs = [], []
    for _ in range(160):
        fam = int(rng.integers(0, 3))
        chi = float(rng.uniform(0.0, 1.2))
        if fam == 1:
            lam = float(rng.uniform(0.05, 1.0))
            kw, okw = dict(lambda_E=lam), dict(lam_E=lam)
        elif fam == 2:
            eta, lc = float(rng.uniform(0.0, 0.3)), float(rng.uniform(2.0, 20.0))
            kw, okw = dict(eta=eta, lambda_c=lc), dict(eta=eta, lam_c=lc)
        else:
            kw, okw = {}, {}
        sts.append(B.Spacetime(metric=fam, chi=chi, **kw))
        probs.append(oracle.problem(metric=fam, chi=chi, **okw))
    import torch
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    res = _np(B.geometry_scan(sts, THETA, stats=stats))
    assert np.all(stats.cpu().numpy() > 0)
    checked = 0
    for i, P in enumerate(probs):
        ce, Re = oracle.extremal_spin(P)
        # where -R^2 H never becomes positive chi_e is 0 (the oracle's golden
        # section returns round-off there) and R_e is not defined
        assert res["chi_e"][i] == pytest.approx(ce, rel=1e-12, abs=1e-12)
        if ce > 1e-8:
            assert res["R_e"][i] == pytest.approx(Re, rel=1e-7)
        rp = oracle.horizon(P)
        assert res["flags"][i] == (0 if rp is not None else 1)
        if rp is None or abs(P.chi) > ce - 1e-3:
            continue
        checked += 1
        assert res["r_plus"][i] == pytest.approx(rp, rel=1e-12)
        for k, th in enumerate(THETA):
            rs = oracle.ergosurface(P, th)
            assert res["R_s"][i, k] == pytest.approx(rs, rel=1e-12)
    assert checked >= 60


def test_flags_and_edges(B):
    sts = [B.Spacetime(metric=7, chi=0.5), B.Spacetime(metric=B.EINASTO, chi=0.5, lambda_E=0.0),
           B.Spacetime(metric=B.CNFW, chi=0.5, eta=-0.1, lambda_c=10.0),
           B.Spacetime(metric=B.CNFW, chi=float("nan"), eta=0.02, lambda_c=10.0),
           B.Spacetime(metric=B.EINASTO, chi=0.7, lambda_E=0.3),      # chi_e = 0.640
           B.Spacetime(metric=B.KERR, chi=1.2)]
    res = _np(B.geometry_scan(sts, THETA))
    assert list(res["flags"]) == [2, 2, 2, 2, 1, 1]
    assert np.all(res["r_plus"] == 0.0)
    assert np.all(res["R_s"][:4] == 0.0)
    # above the extremal spin the poles have no stationary-limit root; the
    # equator keeps H(R_s) = 0 (Eq. 41), which does not involve the spin
    assert res["R_s"][4, 0] == 0.0 and res["R_s"][4, 3] > 0.0
    assert res["R_s"][5, 3] == pytest.approx(2.0, rel=1e-14)
    empty = _np(B.geometry_scan([], THETA))
    assert empty["flags"].shape == (0,)
    none = _np(B.geometry_scan(sts[4:], ()))
    assert none["R_s"].shape == (2, 0)
