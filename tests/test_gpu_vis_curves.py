"""GPU visibility-amplitude curves (Sec. 6.4: the azimuthally averaged
normalised amplitude V(q) and the horizontal cut |V(q, 0)| / |V(0, 0)|)
through the C ABI, against the oracle and the elliptical Gaussian's closed
forms.

Bar: the FP64 mode within 1e-11 of the oracle's curves (normalised amplitudes
of a traced image and of a ragged ring image); the split tensor-core modes
within 4e-4 (the visibility path's bar, |V - V_ref| <= 2e-4 |V(0,0)|, enters
both the amplitude and its normaliser |V(0,0)|); the Gaussian's closed forms
within the float32 rounding of its samples.
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


def _traced(oracle):
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), nx=48, ny=40, x_min=-12, x_max=12, y_min=-10, y_max=10,
                chi=0.95, incl=math.radians(70.0))
    ref = oracle.trace_image(oracle.problem(**{k: v for k, v in flat.items()
                                               if k in oracle.DEFAULTS}))
    return ref["I"].astype(np.float32), flat


def _ring(nx, ny, ext_x, ext_y):
    cx = -ext_x + (np.arange(nx) + 0.5) * (2 * ext_x / nx)
    cy = -ext_y + (np.arange(ny) + 0.5) * (2 * ext_y / ny)
    XX, YY = np.meshgrid(cx, cy)
    r = np.hypot(XX - 0.7, YY + 0.3)
    I = np.exp(-0.5 * ((r - 5.0) / 0.8) ** 2) * (1.0 + 0.4 * XX / (1.0 + r))
    return I.astype(np.float32), dict(nx=nx, ny=ny, x_min=-ext_x, x_max=ext_x, y_min=-ext_y,
                                      y_max=ext_y)


def _cam(B, g):
    return B.Camera(nx=g["nx"], ny=g["ny"], x_min=g["x_min"], x_max=g["x_max"],
                    y_min=g["y_min"], y_max=g["y_max"])


@pytest.mark.parametrize("mode,tol", [(0, 1e-11), (1, 4e-4), (2, 4e-4)])
def test_curves_match_oracle(B, oracle, mode, tol):
    import torch
    from oracle.visibility import amplitude_curves
    q = np.concatenate([[0.0], np.linspace(0.005, 0.5, 37)])
    for I, g in (_traced(oracle), _ring(201, 157, 10.0, 7.8)):
        avg, cut = B.visibility_curves(torch.from_numpy(I).cuda(), _cam(B, g), q, n_phi=45,
                                       mode=mode)
        ra, rc = amplitude_curves(I.astype(np.float64), g["x_min"], g["x_max"], g["y_min"],
                                  g["y_max"], q, 45)
        assert np.max(np.abs(avg.cpu().numpy() - ra)) <= tol
        assert np.max(np.abs(cut.cpu().numpy() - rc)) <= tol
        assert avg[0].item() == pytest.approx(1.0, abs=1e-14)
        assert cut[0].item() == pytest.approx(1.0, abs=1e-14)


def test_gaussian_closed_forms(B):
    import torch
    from scipy.special import i0
    sx, sy, n, ext = 1.2, 0.7, 256, 12.0
    c = -ext + (np.arange(n) + 0.5) * (2 * ext / n)
    XX, YY = np.meshgrid(c, c)
    I = np.exp(-0.5 * ((XX - 0.8) / sx) ** 2 - 0.5 * ((YY + 0.5) / sy) ** 2).astype(np.float32)
    g = dict(nx=n, ny=n, x_min=-ext, x_max=ext, y_min=-ext, y_max=ext)
    q = np.linspace(0.0, 0.3, 61)
    avg, cut = B.visibility_curves(torch.from_numpy(I).cuda(), _cam(B, g), q, n_phi=128, mode=0)
    a = math.pi ** 2 * q ** 2
    assert np.allclose(cut.cpu().numpy(), np.exp(-2 * a * sx ** 2), rtol=0, atol=2e-7)
    want = np.exp(-a * (sx ** 2 + sy ** 2)) * i0(a * (sx ** 2 - sy ** 2))
    assert np.allclose(avg.cpu().numpy(), want, rtol=0, atol=2e-7)


def test_edges(B):
    import torch
    I, g = _ring(64, 48, 10.0, 7.5)
    It = torch.from_numpy(I).cuda()
    avg, cut = B.visibility_curves(It, _cam(B, g), np.zeros(0), n_phi=8, mode=1)
    assert avg.shape == (0,)
    for kw in (dict(n_phi=0), dict(mode=3), dict(image_max=-1.0)):
        with pytest.raises(B.BHRTError):
            B.visibility_curves(It, _cam(B, g), [0.1], **{"n_phi": 8, **kw})
    # a single angle is the direction phi = pi/2: the cut along v
    avg, cut = B.visibility_curves(It, _cam(B, g), [0.1, 0.2], n_phi=1, mode=0)
    from oracle.visibility import normalised_amplitude, visibilities
    V = visibilities(I.astype(np.float64), -10.0, 10.0, -7.5, 7.5,
                     [[0.0, 0.0], [0.0, 0.1], [0.0, 0.2]])
    assert np.allclose(avg.cpu().numpy(), normalised_amplitude(V[1:], V[0]), rtol=1e-11)
