"""Parity at the benchmark's full size and launch configuration: the six
512^2 images of the sweep ({Einasto, cored-NFW, Kerr} x i in {17, 80} deg,
a = 0.9, three refinement levels) traced in one batched plan with the default
persistent grids, exactly as bench.py times them, in both precisions.

The oracle cannot trace whole images this size in a test, so sampled base
pixels (most of them refined, where the method does its work) are computed
one by one with their refinement subtrees and compared: the pixel value
within 1e-6 (FP64 path) or 1e-4 (mixed path) of the image maximum, the base
ray's class exactly, except where the oracle shows the class to be
undetermined at the path's precision (the exemption rules of parity.py); a
pixel whose refinement depth differs holds such a ray in its subtree and is
counted, not compared.
"""
import numpy as np
import pytest

from parity import class_sensitive, oracle_class_is_undetermined, oracle_flat, pixel_centre

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (0, 1e-6)])
def test_fullsize_sweep_sampled_pixels(B, oracle, precision, tol):
    from paper_2605_05635_gb300 import workloads
    flats = workloads.sweep_512(precision=precision)
    plan = B.Plan([B.from_flat(d) for d in flats])
    plan.launch()
    plan.check()
    outs = [{k: v.cpu().numpy() for k, v in o.items()} for o in plan.outputs]
    plan.close()
    rng = np.random.default_rng(512 + precision)
    compared, skipped_depth = 0, 0
    for img, d in enumerate(flats):
        g = outs[img]
        refined = np.argwhere(g["refine_level"] > 0)          # (j, i)
        picks = [tuple(refined[k]) for k in rng.choice(len(refined), 5, replace=False)]
        picks += [tuple(x) for x in rng.integers(0, 512, (2, 2))]
        ij = np.array([[i, j] for j, i in picks], dtype=np.int32)
        P = oracle.problem(**{**oracle_flat(d, oracle), "rtol": 1e-10, "atol": 1e-12})
        ref = oracle.trace_pixels(P, ij)
        base = oracle.trace_points(P, [pixel_centre(d, i, j) for i, j in ij])
        scale = float(np.abs(g["I"]).max())
        exempt = class_sensitive if precision == 1 else oracle_class_is_undetermined
        for k, (i, j) in enumerate(ij):
            X, Y = pixel_centre(d, i, j)
            if (g["status"][j, i], g["ncross"][j, i]) != (base[k]["status"], base[k]["ncross"]):
                assert exempt(oracle, d, X, Y), (img, i, j)
                continue
            if g["refine_level"][j, i] != ref["level"][k]:
                skipped_depth += 1
                continue
            assert abs(float(g["I"][j, i]) - ref["val"][k, 0]) <= tol * scale, \
                (img, i, j, float(g["I"][j, i]), ref["val"][k, 0])
            compared += 1
    assert compared >= 30 and skipped_depth <= 6


def test_fullsize_shadow_fig5(B, oracle):
    """The shadow workload as bench.py times it (three spacetimes x 4096
    directions to 1e-10, the library's lane choice): no flags, brackets at
    most 1e-10 wide, sampled directions within 1e-10 + 3e-9 of the oracle's
    bisection."""
    from paper_2605_05635_gb300 import workloads
    flats, psi, lo, hi, tol = workloads.shadow_fig5()
    psi = np.asarray(psi)
    rng = np.random.default_rng(31)
    for d in flats:
        st, cam, _, it = B.from_flat(d)
        b_in, b_out, fl = (t.cpu().numpy() for t in B.shadow_boundary(st, cam, it, psi, lo, hi,
                                                                      tol))
        assert np.all(fl == 0) and np.all((b_out - b_in <= tol) & (b_out > b_in))
        k = rng.choice(len(psi), 6, replace=False)
        ref = oracle.shadow_boundary(oracle.problem(**oracle_flat(d, oracle)), psi[k], lo, hi,
                                     tol)
        mid = 0.5 * (b_in[k] + b_out[k])
        assert np.max(np.abs(mid - 0.5 * (ref["b_in"] + ref["b_out"]))) <= tol + 3e-9


def test_fullsize_geometry_scan(B, oracle):
    """The scan workload (2 x 1024^2 spacetimes, 16 angles) in one call:
    sampled spacetimes against the oracle's horizon, extremal spin and
    stationary-limit radius."""
    import math

    import torch
    from paper_2605_05635_gb300 import workloads
    metric, chi, lam_E, eta, lam_c, theta = workloads.geometry_grid()
    n = metric.shape[0]
    rec = np.zeros(n, dtype=np.dtype([("metric", "<i4"), ("reserved", "<i4"), ("chi", "<f8"),
                                      ("lambda_E", "<f8"), ("eta", "<f8"), ("lambda_c", "<f8")]))
    rec["metric"], rec["chi"], rec["lambda_E"], rec["eta"], rec["lambda_c"] = (
        metric, chi, lam_E, eta, lam_c)
    st_d = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
    res = {k: v.cpu().numpy() for k, v in B.geometry_scan(st_d, theta).items()}
    rng = np.random.default_rng(32)
    checked = 0
    for i in rng.choice(n, 40, replace=False):
        P = oracle.problem(metric=int(metric[i]), chi=float(chi[i]), lam_E=float(lam_E[i]),
                           eta=float(eta[i]), lam_c=float(lam_c[i]))
        ce, _ = oracle.extremal_spin(P)
        assert res["chi_e"][i] == pytest.approx(ce, rel=1e-12, abs=1e-12)
        rp = oracle.horizon(P)
        assert res["flags"][i] == (0 if rp is not None else 1)
        if rp is None or abs(chi[i]) > ce - 1e-3:
            continue
        checked += 1
        assert res["r_plus"][i] == pytest.approx(rp, rel=1e-12)
        k = int(rng.integers(0, len(theta)))
        assert res["R_s"][i, k] == pytest.approx(oracle.ergosurface(P, float(theta[k])),
                                                 rel=1e-12)
    assert checked >= 10


def test_fullsize_amplitude_curves(B):
    """The amplitude-curve workload (Fig. 12 images at 1024^2, 256 radii x 256
    angles) on the split BF16 path against the FP64 direct mode of the same
    call (itself held to the oracle in test_gpu_vis_curves.py), and a few
    radii of one image against the oracle's direct sums."""
    from oracle.visibility import amplitude_curves
    from paper_2605_05635_gb300 import workloads
    flats = workloads.fig12_images()
    items = [B.from_flat(d) for d in flats]
    imgs = [o["I"] for o in B.trace_batch(items)]
    q = np.linspace(0.5 / 256, 0.5, 256)
    for I, (_, cam, _, _) in zip(imgs, items):
        a1, c1 = B.visibility_curves(I, cam, q, n_phi=256, mode=B.VIS_BF16)
        a0, c0 = B.visibility_curves(I, cam, q, n_phi=256, mode=B.VIS_FP64)
        assert float((a1 - a0).abs().max()) <= 4e-4
        assert float((c1 - c0).abs().max()) <= 4e-4
    d = flats[0]
    qs = q[[10, 120]]
    a, c = B.visibility_curves(imgs[0], items[0][1], qs, n_phi=8, mode=B.VIS_FP64)
    ra, rc = amplitude_curves(imgs[0].double().cpu().numpy(), d["x_min"], d["x_max"], d["y_min"],
                              d["y_max"], qs, 8)
    assert np.allclose(a.cpu().numpy(), ra, atol=1e-10) and np.allclose(c.cpu().numpy(), rc,
                                                                      atol=1e-10)
