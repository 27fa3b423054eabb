"""GPU shadow-boundary search (Sec. 4.1, Eqs. 78-79) through the C ABI,
against the oracle's bisection and the closed forms it is pinned to.

Bar: every bracket at most b_tol wide and unflagged; its midpoint within
b_tol + 3e-9 of the oracle's (both hold the transition of the same FP64
integrator at rtol 1e-10; the slack is the integration noise of rays that
graze the critical curve); the Schwarzschild closed form and the Kerr
radial-potential criterion hold on the GPU's own brackets.  The lane-group
width the host picks (bisection to 32-way multisection) is covered by the
direction counts; ragged counts, the empty call and unbracketed ends too.
"""
import math

import numpy as np
import pytest

from test_oracle_trace import kerr_radial_capture

pytestmark = pytest.mark.gpu

HALOS = {0: {}, 1: dict(lam_E=0.3), 2: dict(eta=0.02, lam_c=10.0)}


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


def _flat(metric, chi, incl):
    from paper_2605_05635_gb300 import workloads
    return dict(workloads.kerr_64(), metric=metric, chi=chi, incl=math.radians(incl),
                **HALOS[metric])


def _gpu(B, flat, psi, lo, hi, tol):
    st, cam, _, it = B.from_flat(flat)
    b_in, b_out, fl = B.shadow_boundary(st, cam, it, psi, lo, hi, tol)
    return b_in.cpu().numpy(), b_out.cpu().numpy(), fl.cpu().numpy()


def _oracle(oracle, flat, psi, lo, hi, tol):
    P = oracle.problem(**{k: v for k, v in flat.items() if k in oracle.DEFAULTS})
    return oracle.shadow_boundary(P, psi, lo, hi, tol)


@pytest.mark.parametrize("metric,chi,incl,n", [(0, 0.9, 60.0, 37), (1, 0.5, 60.0, 48),
                                               (2, 0.5, 60.0, 5), (2, 0.9, 17.0, 3001)])
def test_shadow_matches_oracle(B, oracle, metric, chi, incl, n):
    rng = np.random.default_rng(1000 + n)
    psi = rng.uniform(0.0, 2.0 * math.pi, n)
    tol = 1e-9
    b_in, b_out, fl = _gpu(B, _flat(metric, chi, incl), psi, 1.0, 9.0, tol)
    assert np.all(fl == 0)
    assert np.all(b_out - b_in <= tol) and np.all(b_out > b_in)
    sample = np.arange(n) if n <= 48 else rng.choice(n, 24, replace=False)
    ref = _oracle(oracle, _flat(metric, chi, incl), psi[sample], 1.0, 9.0, tol)
    assert np.all(ref["flags"] == 0)
    mid_g = 0.5 * (b_in[sample] + b_out[sample])
    mid_o = 0.5 * (ref["b_in"] + ref["b_out"])
    assert np.max(np.abs(mid_g - mid_o)) <= tol + 3e-9


def test_schwarzschild_closed_form(B):
    psi = np.linspace(0.0, 2.0 * math.pi, 64, endpoint=False)
    flat = _flat(0, 0.0, 30.0)
    Ro = flat["r_obs"]
    b_c = Ro * math.tan(math.asin(math.sqrt(27.0 * (1.0 - 2.0 / Ro)) / Ro))
    b_in, b_out, fl = _gpu(B, flat, psi, 2.0, 9.0, 1e-10)
    assert np.all(fl == 0)
    assert np.all(b_in <= b_c + 1e-9) and np.all(b_out >= b_c - 1e-9)


def test_kerr_brackets_contain_analytic_curve(B, oracle):
    a = 0.9
    flat = _flat(0, a, 60.0)
    psi = np.linspace(0.0, 2.0 * math.pi, 24, endpoint=False)
    b_in, b_out, fl = _gpu(B, flat, psi, 1.0, 9.0, 1e-7)
    assert np.all(fl == 0)
    P = oracle.problem(**{k: v for k, v in flat.items() if k in oracle.DEFAULTS})
    geo = oracle.geometry(P)
    for b, want in ((b_in, True), (b_out, False)):
        xy = np.stack([b * np.cos(psi), b * np.sin(psi)], 1)
        for ray in oracle.trace_points(P, xy):
            cap, margin = kerr_radial_capture(a, ray["E"], ray["ell"], ray["K0"], geo["r_plus"],
                                              P.r_obs)
            assert abs(margin) > 1e-12
            assert cap == want


def test_many_directions_bisection(B, oracle):
    """Enough directions to fill the resident threads one lane each (the
    host then bisects); a sample against the oracle."""
    n = 40000
    psi = np.linspace(0.0, 2.0 * math.pi, n, endpoint=False)
    flat = _flat(2, 0.7, 45.0)
    tol = 1e-6
    b_in, b_out, fl = _gpu(B, flat, psi, 1.0, 9.0, tol)
    assert np.all(fl == 0) and np.all(b_out - b_in <= tol)
    k = np.arange(0, n, 2500)
    ref = _oracle(oracle, flat, psi[k], 1.0, 9.0, tol)
    mid_g = 0.5 * (b_in[k] + b_out[k])
    assert np.max(np.abs(mid_g - 0.5 * (ref["b_in"] + ref["b_out"]))) <= tol + 3e-9


def test_edges(B):
    flat = _flat(0, 0.5, 30.0)
    psi = np.array([0.0, 1.0, 2.0, 4.0])
    b_in, b_out, fl = _gpu(B, flat, psi, 6.5, 9.0, 1e-6)      # both ends escape
    assert np.all(fl & 1) and not np.any(fl & 2)
    assert np.all(b_in == 6.5) and np.all(b_out == 9.0)
    b_in, b_out, fl = _gpu(B, flat, psi, 1.0, 2.5, 1e-6)      # both ends captured
    assert np.all(fl & 2) and not np.any(fl & 1)
    b_in, b_out, fl = _gpu(B, flat, np.zeros(0), 1.0, 9.0, 1e-6)
    assert b_in.shape == (0,) and fl.shape == (0,)
    st, cam, _, it = B.from_flat(dict(flat, precision=1))
    with pytest.raises(B.BHRTError):
        B.shadow_boundary(st, cam, it, psi, 1.0, 9.0, 1e-6)


def test_lane_widths_agree(B):
    """Bisection (1 lane), 4-lane and 32-lane multisection bracket the same
    transition: each bracket holds the others' midpoints to within b_tol
    plus the integration slack."""
    flat = _flat(0, 0.9, 60.0)
    psi = np.linspace(0.1, 6.2, 19)
    st, cam, _, it = B.from_flat(flat)
    tol = 1e-9
    mids = []
    for lanes in (1, 4, 32):
        b_in, b_out, fl = B.shadow_boundary(st, cam, it, psi, 1.0, 9.0, tol, lanes=lanes)
        assert np.all(fl.cpu().numpy() == 0)
        w = (b_out - b_in).cpu().numpy()
        assert np.all((w > 0) & (w <= tol))
        mids.append(0.5 * (b_in + b_out).cpu().numpy())
    for m in mids[1:]:
        assert np.max(np.abs(m - mids[0])) <= tol + 3e-9


def test_time_budget_reports_timeout(B):
    """A device time budget far below the work ends the call early with the
    workspace status BH_ERR_TIMEOUT (no fault, no hang)."""
    flat = dict(_flat(2, 0.9, 17.0), time_budget_s=1e-5)
    st, cam, _, it = B.from_flat(flat)
    psi = np.linspace(0.0, 2.0 * math.pi, 2048, endpoint=False)
    with pytest.raises(B.BHRTError) as e:
        B.shadow_boundary(st, cam, it, psi, 1.0, 9.0, 1e-12)
    assert e.value.code == 6
