"""GPU parity of the image products against the oracle: diagnostics
(Sec. 6.2-6.3) and FP64 visibilities (Sec. 6.4), on analytic images and on an
oracle-traced image (the same float32 image is given to both sides)."""
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


def _ring(n, ext, r0=5.0, w=0.4, x0=0.7, y0=-0.3):
    d = 2 * ext / n
    c = -ext + (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(c, c)
    I = np.exp(-(np.hypot(X - x0, Y - y0) - r0) ** 2 / (2 * w * w)) * (1 + 0.5 * np.tanh(X))
    return I.astype(np.float32)


def _images(oracle):
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), nx=48, ny=40, x_min=-12, x_max=12, y_min=-10, y_max=10,
                chi=0.9, incl=math.radians(70.0))
    ref = oracle.trace_image(oracle.problem(**{k: v for k, v in flat.items()
                                               if k in oracle.DEFAULTS}))
    yield "traced", ref["I"].astype(np.float32), flat
    yield "ring", _ring(256, 12.0), dict(nx=256, ny=256, x_min=-12.0, x_max=12.0, y_min=-12.0,
                                         y_max=12.0)
    odd = _ring(201, 10.0)[:, :201]
    yield "ring_odd", np.ascontiguousarray(odd[:157]), dict(nx=201, ny=157, x_min=-10.0,
                                                             x_max=10.0, y_min=-7.8,
                                                             y_max=7.8)


def test_diagnostics_match_oracle(B, oracle):
    import torch
    from oracle.diagnostics import NAMES, diagnostics
    for name, I, g in _images(oracle):
        cam = B.Camera(nx=g["nx"], ny=g["ny"], x_min=g["x_min"], x_max=g["x_max"],
                       y_min=g["y_min"], y_max=g["y_max"])
        out = B.diagnostics(torch.from_numpy(I).cuda(), cam, theta_g=3.8).cpu().numpy()
        ref = diagnostics(I.astype(np.float64), g["x_min"], g["x_max"], g["y_min"], g["y_max"],
                          theta_g=3.8)
        for k, nm in enumerate(NAMES):
            assert out[k] == pytest.approx(ref[nm], rel=1e-11, abs=1e-12), (name, nm)


def test_diagnostics_all_zero_and_single_pixel(B, oracle):
    import torch
    from oracle.diagnostics import NAMES, diagnostics
    I = np.zeros((9, 7), np.float32)
    I[4, 5] = 2.0
    cam = B.Camera(nx=7, ny=9, x_min=-3.5, x_max=3.5, y_min=-4.5, y_max=4.5)
    out = B.diagnostics(torch.from_numpy(I).cuda(), cam).cpu().numpy()
    ref = diagnostics(I.astype(np.float64), -3.5, 3.5, -4.5, 4.5)
    for k, nm in enumerate(NAMES):
        if nm == "A_LR":
            # F_R = F_L = 0 when the only pixel sits on the centroid column
            assert math.isnan(ref[nm]) and math.isnan(out[k])
            continue
        assert out[k] == pytest.approx(ref[nm], rel=1e-12, abs=1e-12), nm


def test_visibilities_fp64_match_oracle(B, oracle):
    import torch
    from oracle.visibility import visibilities
    from paper_2605_05635_gb300 import workloads
    uv = workloads.uv_points(40, seed=20260515)
    uv = np.concatenate([[[0.0, 0.0]], uv])
    for name, I, g in _images(oracle):
        cam = B.Camera(nx=g["nx"], ny=g["ny"], x_min=g["x_min"], x_max=g["x_max"],
                       y_min=g["y_min"], y_max=g["y_max"])
        V = B.visibilities_fp64(torch.from_numpy(I).cuda(), cam, torch.from_numpy(uv)).cpu().numpy()
        ref = visibilities(I.astype(np.float64), g["x_min"], g["x_max"], g["y_min"], g["y_max"], uv)
        scale = abs(ref[0])
        assert np.max(np.abs(V - ref)) <= 1e-12 * scale, name


@pytest.mark.parametrize("mode,tol", [(1, 2e-4), (2, 2e-4)])
def test_visibilities_tensor_core_split(B, oracle, mode, tol):
    """Split BF16 / FP16 tensor-core contraction vs the oracle's FP64 direct
    sum: |V - V_ref| <= tol |V(0,0)| (the split keeps ~16 significant bits of
    each operand, so the error sits near 2^-16 of the zero-baseline flux)."""
    import torch
    from oracle.visibility import visibilities
    from paper_2605_05635_gb300 import workloads
    uv = np.concatenate([[[0.0, 0.0]], workloads.uv_points(150, seed=20260515)])
    for name, I, g in _images(oracle):
        cam = B.Camera(nx=g["nx"], ny=g["ny"], x_min=g["x_min"], x_max=g["x_max"],
                       y_min=g["y_min"], y_max=g["y_max"])
        It = torch.from_numpy(I).cuda()
        V = B.visibilities(It, cam, torch.from_numpy(uv), mode=mode).cpu().numpy()
        ref = visibilities(I.astype(np.float64), g["x_min"], g["x_max"], g["y_min"], g["y_max"], uv)
        err = np.max(np.abs(V - ref)) / abs(ref[0])
        assert err <= tol, (name, err)


def test_visibilities_large_image_vs_gpu_fp64(B):
    """1024^2 (two 512-row passes, 16 reduction chunks per third): tensor path
    against the FP64 direct mode on sampled baselines."""
    import torch
    from paper_2605_05635_gb300 import workloads
    n = 1024
    I = _ring(n, 12.0, r0=4.5, w=0.3)
    cam = B.Camera(nx=n, ny=n, x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0)
    uv = torch.from_numpy(np.concatenate([[[0.0, 0.0]], workloads.uv_points(511, seed=5)]))
    It = torch.from_numpy(I).cuda()
    Vt = B.visibilities(It, cam, uv, mode=1).cpu().numpy()
    Vd = B.visibilities_fp64(It, cam, uv).cpu().numpy()
    assert np.max(np.abs(Vt - Vd)) / abs(Vd[0]) <= 2e-4


def test_visibilities_widest_screen_and_ragged_baselines(B):
    """nx = 4096, the widest screen the tensor-core path takes (its per-CTA
    phase table), a short screen (40 rows of one 256-row pass) and 70
    baselines (a ragged last CTA), against the FP64 direct mode; nx = 4097
    is refused before any work."""
    import torch
    from paper_2605_05635_gb300 import workloads
    nx, ny = 4096, 40
    rng = np.random.default_rng(11)
    I = rng.random((ny, nx)).astype(np.float32)
    cam = B.Camera(nx=nx, ny=ny, x_min=-12.0, x_max=12.0, y_min=-1.0, y_max=1.0)
    uv = torch.from_numpy(np.concatenate([[[0.0, 0.0]], workloads.uv_points(69, seed=7)]))
    It = torch.from_numpy(I).cuda()
    Vt = B.visibilities(It, cam, uv, mode=1).cpu().numpy()
    Vd = B.visibilities_fp64(It, cam, uv).cpu().numpy()
    assert Vt.shape == (70,)
    assert np.max(np.abs(Vt - Vd)) / abs(Vd[0]) <= 2e-4
    wide = B.Camera(nx=nx + 1, ny=ny, x_min=-12.0, x_max=12.0, y_min=-1.0, y_max=1.0)
    with pytest.raises(B.BHRTError):
        B.visibilities(torch.zeros(ny, nx + 1, device="cuda"), wide, uv, mode=1)


@pytest.mark.parametrize("mode,tol", [(0, 1e-12), (1, 2e-4), (2, 2e-4)])
def test_normalised_amplitudes_match_oracle(B, oracle, mode, tol):
    """Eq. (109): the normalised amplitude |V|/|V(0,0)| returned beside V,
    against the oracle's FP64 direct sum divided by its zero-baseline value
    (the flux, Eq. 92): within 1e-12 for the FP64 mode and within the split
    modes' bound on |V - V_ref| / |V(0,0)|; 1 at the zero baseline."""
    import torch
    from oracle.visibility import visibilities
    from paper_2605_05635_gb300 import workloads
    uv = np.concatenate([[[0.0, 0.0]], workloads.uv_points(99, seed=20260514)])
    for name, I, g in _images(oracle):
        cam = B.Camera(nx=g["nx"], ny=g["ny"], x_min=g["x_min"], x_max=g["x_max"],
                       y_min=g["y_min"], y_max=g["y_max"])
        V, Vn = B.visibilities(torch.from_numpy(I).cuda(), cam, torch.from_numpy(uv), mode=mode,
                               normalised=True)
        ref = visibilities(I.astype(np.float64), g["x_min"], g["x_max"], g["y_min"], g["y_max"], uv)
        want = np.abs(ref) / abs(ref[0])
        got = Vn.cpu().numpy()
        assert got.shape == (100,)
        assert np.max(np.abs(got - want)) <= tol, (name, mode)
        assert abs(got[0] - 1.0) <= tol


def test_visibilities_time_budget_stops_cleanly(B):
    """A device time budget already spent when the contraction starts: every
    CTA stops at its first chunk, before issuing any copy or product, and the
    workspace status reads BH_ERR_TIMEOUT (no fault, no hang).  The same
    workspace then serves an unbudgeted call whose visibilities match the
    FP64 direct mode, so the context is still usable."""
    import torch
    from paper_2605_05635_gb300 import workloads
    n = 1024
    I = torch.from_numpy(_ring(n, 12.0, r0=4.5, w=0.3)).cuda()
    cam = B.Camera(nx=n, ny=n, x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0)
    uv = torch.from_numpy(np.concatenate([[[0.0, 0.0]], workloads.uv_points(4095, seed=9)]))
    ws = B.visibilities_workspace(cam, I.device)
    with pytest.raises(B.BHRTError) as err:
        B.visibilities(I, cam, uv, mode=1, workspace=ws, time_budget_s=1e-9)
    assert err.value.code == 6  # BH_ERR_TIMEOUT
    torch.cuda.synchronize()
    Vt = B.visibilities(I, cam, uv, mode=1, workspace=ws).cpu().numpy()
    Vd = B.visibilities_fp64(I, cam, uv).cpu().numpy()
    assert np.max(np.abs(Vt - Vd)) / abs(Vd[0]) <= 2e-4
    with pytest.raises(B.BHRTError):
        B.visibilities(I, cam, uv, mode=1, workspace=ws, time_budget_s=-1.0)
