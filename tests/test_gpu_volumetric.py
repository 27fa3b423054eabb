"""GPU parity of the volumetric intensity (Eq. 88: I = int g^3 j dlambda over
the finite-thickness layer of Eqs. 83-87, integrated as a seventh ODE
component) against the CPU oracle, through the C ABI.

Bar: the FP64 path within 1e-6 of the image maximum, the mixed path within
1e-4 (the thin-disk bars); integer planes exact outside the numerically
undetermined set; the per-order planes I_n stay zero; the geodesic outputs
(class, refinement pattern, transfer radius) are those of the thin-disk mode.
The argument checks (H0 > 0, h >= 0, flag in {0, 1}) and the adjoint's
refusal of the volumetric mode are checked too.
"""
import math

import numpy as np
import pytest

from parity import class_sensitive, oracle_class_is_undetermined, oracle_flat, pixel_centre

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-6
TOL_MIXED = 1e-4

HALOS = {0: {}, 1: dict(lam_E=0.1), 2: dict(eta=0.02, lam_c=10.0)}


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


def _flat(workloads, metric, incl, **kw):
    # 24 x 20 with one refinement level: several 16 x 16 tiles of work and a
    # ragged tail in both directions
    return dict(workloads.kerr_64(), metric=metric, chi=0.9, incl=math.radians(incl), nx=24,
                ny=20, x_min=-10.0, x_max=10.0, y_min=-9.0, y_max=9.0, levels=1,
                volumetric=1, **HALOS[metric], **kw)


def _gpu_image(B, flat):
    st, cam, em, it = B.from_flat(flat)
    return {k: v.cpu().numpy() for k, v in B.trace_image(st, cam, em, it).items()}


@pytest.mark.parametrize("metric,incl", [(0, 17.0), (1, 80.0), (2, 60.0)])
def test_volumetric_fp64_image(B, oracle, metric, incl):
    from paper_2605_05635_gb300 import workloads
    flat = _flat(workloads, metric, incl)
    gpu = _gpu_image(B, flat)
    ref = oracle.trace_image(oracle.problem(**oracle_flat(flat, oracle)))
    ok = np.ones(gpu["status"].shape, bool)
    for j, i in np.argwhere((gpu["status"] != ref["status"]) | (gpu["ncross"] != ref["ncross"])):
        assert oracle_class_is_undetermined(oracle, flat, *pixel_centre(flat, i, j)), (i, j)
        ok[j, i] = False
    assert (~ok).sum() <= 2
    scale = np.abs(ref["I"]).max()
    assert scale > 0
    assert np.max(np.abs(gpu["I"][ok] - ref["I"][ok])) <= TOL_FP64 * scale
    assert np.all(gpu["I_n"] == 0.0)
    assert np.array_equal(gpu["refine_level"], ref["level"])
    # the geodesic is the thin-disk mode's: same classes and transfer radii
    # (to the transfer-map bar: the step sequences differ)
    thin = _gpu_image(B, dict(flat, volumetric=0))
    assert np.array_equal(thin["status"], gpu["status"])
    assert np.array_equal(thin["ncross"], gpu["ncross"])
    has = gpu["ncross"] > 0
    assert np.allclose(thin["R_em"][0][has], gpu["R_em"][0][has], rtol=TOL_FP64)


@pytest.mark.parametrize("metric,incl", [(0, 80.0), (2, 17.0)])
def test_volumetric_mixed_image(B, oracle, metric, incl):
    from paper_2605_05635_gb300 import workloads
    flat = dict(_flat(workloads, metric, incl), **workloads.MIXED_INTEG)
    gpu = _gpu_image(B, flat)
    ref = oracle.trace_image(oracle.problem(**{**oracle_flat(flat, oracle), "rtol": 1e-10,
                                               "atol": 1e-12}))
    ok = np.ones(gpu["status"].shape, bool)
    for j, i in np.argwhere((gpu["status"] != ref["status"]) | (gpu["ncross"] != ref["ncross"])):
        assert class_sensitive(oracle, flat, *pixel_centre(flat, i, j)), (i, j)
        ok[j, i] = False
    assert (~ok).sum() <= 3
    scale = np.abs(ref["I"]).max()
    err = np.max(np.abs(gpu["I"][ok] - ref["I"][ok])) / scale
    assert err <= TOL_MIXED, err
    assert np.all(gpu["I_n"] == 0.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_volumetric_points_thin_layer(B, oracle, precision):
    """Points mode, thin layer (H0 = 1e-3): the GPU integral against the
    oracle's and against the thin-layer limit sum_n g^3 j sqrt(2 pi) H /
    (R |dtheta/dlambda|) built from the oracle's thin-disk records (event
    root finding, not quadrature)."""
    from paper_2605_05635_gb300 import workloads
    rng = np.random.default_rng(20261203)
    xy = rng.uniform(-8.0, 8.0, size=(96, 2))
    base = dict(workloads.kerr_64(), metric=2, chi=0.7, incl=math.radians(60.0), r_in_mode=1,
                **HALOS[2])
    if precision:
        base.update(workloads.MIXED_INTEG)
    vol = dict(base, volumetric=1, H0=1e-3, h=0.0)
    g_vol = B.trace_points(*B.from_flat(vol), xy)
    tight = {"rtol": 1e-10, "atol": 1e-12}
    r_vol = oracle.trace_points(oracle.problem(**{**oracle_flat(vol, oracle), **tight}), xy)
    r_thin = oracle.trace_points(oracle.problem(**{**oracle_flat(base, oracle), **tight}), xy)
    keep = (r_thin["ncross"] >= 1) & (r_thin["ncross"] <= 3)
    keep &= (g_vol["status"] == r_vol["status"]) & (g_vol["ncross"] == r_vol["ncross"])
    assert keep.sum() >= 40
    assert np.all(g_vol["I_n"] == 0.0)
    tol = TOL_MIXED if precision else TOL_FP64
    scale = np.abs(r_vol["I_tot"][keep]).max()
    assert np.max(np.abs(g_vol["I_tot"][keep] - r_vol["I_tot"][keep])) <= tol * scale
    pred = np.zeros(len(xy))
    for k, r in enumerate(r_thin):
        for n in range(min(int(r["ncross"]), 3)):
            pred[k] += r["I_n"][n] * math.sqrt(2 * math.pi) * 1e-3 / (
                r["R_em"][n] * abs(r["thdot"][n]))
    # the limit is exact only as H -> 0: where a ray grazes the layer or
    # crosses it at a taper the oracle itself departs from it, so each point
    # may depart by twice the oracle's own departure plus the bar
    lim_tol = 2e-4 if precision else 1e-5
    own = np.abs(r_vol["I_tot"] - pred)
    assert np.all(np.abs(g_vol["I_tot"] - pred)[keep] <= (lim_tol * np.abs(pred) + 2 * own)[keep])
    assert np.count_nonzero(own[keep] <= 1e-5 * np.abs(pred[keep])) >= 0.9 * keep.sum()


def test_volumetric_argument_checks(B):
    from paper_2605_05635_gb300 import workloads
    import torch
    flat = dict(workloads.kerr_64(), nx=8, ny=8, volumetric=1)
    for bad in (dict(H0=0.0), dict(H0=-1.0), dict(h=-0.1), dict(h=float("nan")),
                dict(volumetric=2), dict(volumetric=-1)):
        st, cam, em, it = B.from_flat(dict(flat, **bad))
        with pytest.raises(B.BHRTError):
            B.trace_image(st, cam, em, it)
    # the discrete adjoint differentiates the thin-disk intensity only
    st, cam, em, it = B.from_flat(flat)
    with pytest.raises(B.BHRTError):
        B.trace_backward(st, cam, em, it, dL_dI=torch.ones(8, 8))
