"""GPU parity of the tracing path (C ABI through the Python binding) against
the CPU oracle, on the same seeded synthetic screens.

Bar: integer planes (status, N_cross, refinement pattern) bit-exact outside
the numerically undetermined set (see tests/parity.py); FP64 intensity,
transfer maps and redshift within 1e-6 relative (intensity relative to the
image maximum, maps per pixel).
"""
import math

import numpy as np
import pytest

from parity import oracle_class_is_undetermined, oracle_flat, pixel_centre, rel_max_err

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-6


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


def _gpu_image(B, flat, keys_cap=0):
    st, cam, em, it = B.from_flat(flat)
    out = B.trace_image(st, cam, em, it, keys_cap=keys_cap)
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check_integer_planes(oracle, flat, gpu, ref, max_exempt_frac=2e-3):
    bad = np.argwhere((gpu["status"] != ref["status"]) | (gpu["ncross"] != ref["ncross"]))
    exempt = 0
    for j, i in bad:
        X, Y = pixel_centre(flat, i, j)
        assert oracle_class_is_undetermined(oracle, flat, X, Y), (
            f"class mismatch at pixel ({i},{j}) X={X} Y={Y}: gpu "
            f"({gpu['status'][j, i]},{gpu['ncross'][j, i]}) oracle "
            f"({ref['status'][j, i]},{ref['ncross'][j, i]})")
        exempt += 1
    assert exempt <= max_exempt_frac * gpu["status"].size + 1
    return bad


def test_kerr_64_parity(B, oracle):
    from paper_2605_05635_gb300 import workloads
    flat = workloads.kerr_64()
    gpu = _gpu_image(B, flat)
    ref = oracle.trace_image(oracle.problem(**oracle_flat(flat, oracle)))
    bad = _check_integer_planes(oracle, flat, gpu, ref)
    ok = np.ones_like(gpu["status"], dtype=bool)
    for j, i in bad:
        ok[j, i] = False
    scale = np.abs(ref["I"]).max()
    assert scale > 0
    assert np.max(np.abs(gpu["I"][ok] - ref["I"][ok])) <= TOL_FP64 * scale
    for n in range(3):
        assert np.max(np.abs(gpu["I_n"][n][ok] - ref["I_n"][n][ok])) <= TOL_FP64 * scale
        has = ok & (ref["ncross"] > n)
        if has.any():
            for k in ("R_em", "g"):
                r = ref[k][n][has]
                gk = gpu[k][n][has]
                nz = r != 0.0  # g = 0 where no timelike circular emitter exists
                assert np.all(gk[~nz] == 0.0), k
                assert np.max(np.abs(gk[nz] - r[nz]) / np.abs(r[nz])) <= TOL_FP64, k
            # phi wraps at 2 pi; T is compared relative to its magnitude
            dphi = np.angle(np.exp(1j * (gpu["phi_em"][n][has] - ref["phi_em"][n][has])))
            assert np.max(np.abs(dphi)) <= 1e-5
            assert rel_max_err(gpu["T_em"][n][has], ref["T_em"][n][has]) <= TOL_FP64
        none = ok & (ref["ncross"] <= n)
        assert np.all(gpu["R_em"][n][none] == 0.0)
    assert np.all(gpu["refine_level"] == 0)
    assert np.max(gpu["h_drift"]) < 1e-8
    # qualitative structure (Fig. 6): captured centre with N_cross = 0
    assert gpu["status"][32, 32] == 1 and gpu["ncross"][32, 32] == 0


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_points_parity(B, oracle, metric):
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), metric=metric, chi=0.9, incl=math.radians(80.0),
                **workloads.HALO[metric])
    rng = np.random.default_rng(100 + metric)
    xy = np.concatenate([rng.uniform(-12, 12, (48, 2)),
                         np.stack([5.2 * np.cos(np.linspace(0, 6.2, 16)),
                                   5.2 * np.sin(np.linspace(0, 6.2, 16))], 1)])
    st, cam, em, it = B.from_flat(flat)
    g = B.trace_points(st, cam, em, it, xy)
    r = oracle.trace_points(oracle.problem(**oracle_flat(flat, oracle)), xy)
    for k in range(len(xy)):
        same = g[k]["status"] == r[k]["status"] and g[k]["ncross"] == r[k]["ncross"]
        if not same:
            assert oracle_class_is_undetermined(oracle, flat, *xy[k])
            continue
        assert g[k]["E"] == pytest.approx(r[k]["E"], rel=1e-14)
        assert g[k]["ell"] == pytest.approx(r[k]["ell"], rel=1e-13, abs=1e-15)
        assert g[k]["I_tot"] == pytest.approx(r[k]["I_tot"], rel=TOL_FP64, abs=1e-12)
        for n in range(min(r[k]["ncross"], 3)):
            assert g[k]["R_em"][n] == pytest.approx(r[k]["R_em"][n], rel=TOL_FP64)
            assert g[k]["g"][n] == pytest.approx(r[k]["g"][n], rel=TOL_FP64, abs=1e-300)
            assert g[k]["T_em"][n] == pytest.approx(r[k]["T_em"][n], rel=TOL_FP64)
        # step counts of the same adaptive scheme stay close
        assert abs(int(g[k]["n_accept"]) - int(r[k]["n_accept"])) <= 0.02 * r[k]["n_accept"] + 3


@pytest.mark.parametrize("metric,incl", [(0, 80.0), (1, 17.0), (2, 50.0)])
def test_refined_parity(B, oracle, metric, incl):
    """Ragged screen (odd, non-square), 2 refinement levels: integer planes,
    refinement pattern and leaf-mean intensity."""
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), metric=metric, chi=0.9, incl=math.radians(incl), nx=21,
                ny=17, x_min=-12.0, x_max=12.0, y_min=-10.0, y_max=10.0, levels=2,
                **workloads.HALO[metric])
    gpu = _gpu_image(B, flat, keys_cap=1 << 20)
    ref = oracle.trace_image(oracle.problem(**oracle_flat(flat, oracle)))
    bad = _check_integer_planes(oracle, flat, gpu, ref, max_exempt_frac=0.01)
    gk = np.sort(gpu["refine_keys"].astype(np.uint64))
    rk = ref["keys"]
    base_of = lambda k: (k >> np.uint64(16)).astype(np.int64)
    diff_pix = set(base_of(np.setxor1d(gk, rk)).tolist())
    diff_pix |= {int(j * flat["nx"] + i) for j, i in bad}
    assert len(diff_pix) <= 0.02 * gpu["status"].size + 1
    # a pixel whose refinement subtree differs must be numerically
    # undetermined: the oracle's own subtree changes when its tolerance is
    # tightened to 1e-12
    Pw = oracle.problem(**oracle_flat(flat, oracle))
    Pt = oracle.problem(**{**oracle_flat(flat, oracle), "rtol": 1e-12, "atol": 1e-14})
    for q in diff_pix:
        j, i = divmod(q, flat["nx"])
        a, b = oracle.trace_pixel(Pw, i, j), oracle.trace_pixel(Pt, i, j)
        undetermined = (not np.array_equal(a["keys"], b["keys"]) or a["status"] != b["status"]
                        or a["ncross"] != b["ncross"])
        assert undetermined, f"refinement differs at pixel ({i},{j}) without an undetermined ray"
    ok = np.ones(gpu["status"].shape, bool)
    for q in diff_pix:
        ok[divmod(q, flat["nx"])] = False
    scale = np.abs(ref["I"]).max()
    assert np.max(np.abs(gpu["I"][ok] - ref["I"][ok])) <= TOL_FP64 * scale
    assert np.array_equal(gpu["refine_level"][ok], ref["level"][ok])
    assert (gpu["refine_level"] > 0).sum() > 0


def test_single_pixel_and_determinism(B, oracle):
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), nx=1, ny=1, x_min=4.0, x_max=6.0, y_min=-1.0, y_max=1.0)
    a = _gpu_image(B, flat)
    b = _gpu_image(B, flat)
    ref = oracle.trace_image(oracle.problem(**oracle_flat(flat, oracle)))
    assert a["status"][0, 0] == ref["status"][0, 0] and a["ncross"][0, 0] == ref["ncross"][0, 0]
    assert a["I"][0, 0] == pytest.approx(ref["I"][0, 0], rel=TOL_FP64)
    for k in a:
        assert np.array_equal(a[k], b[k])


def test_argument_errors(B):
    from paper_2605_05635_gb300 import workloads
    flat = workloads.kerr_64()
    st, cam, em, it = B.from_flat(flat)
    with pytest.raises(B.BHRTError) as e:
        B.trace_image(B.Spacetime(metric=0, chi=1.05), cam, em, it)
    assert e.value.code == 2
    with pytest.raises(B.BHRTError) as e:
        B.trace_image(st, B.Camera(r_obs=15.0), em, it)
    assert e.value.code == 3
    with pytest.raises(B.BHRTError) as e:
        B.trace_image(st, cam, em, B.Integrator(rtol=-1.0))
    assert e.value.code == 1


def test_time_budget_returns_status(B):
    """A device time budget that runs out makes the kernel return
    BH_ERR_TIMEOUT; the context stays usable."""
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), time_budget_s=1e-6)
    st, cam, em, it = B.from_flat(flat)
    with pytest.raises(B.BHRTError) as e:
        B.trace_image(st, cam, em, it)
    assert e.value.code == 6
    it.time_budget_s = 0.0
    out = B.trace_image(st, cam, em, it)
    assert int(out["status"][32, 32]) == 1


def test_queue_overflow_returns_status(B):
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), levels=2, refine_capacity=32)
    st, cam, em, it = B.from_flat(flat)
    with pytest.raises(B.BHRTError) as e:
        B.trace_image(st, cam, em, it)
    assert e.value.code == 7


def test_step_and_promotion_planes(B):
    """Per-pixel step counters equal those of the same rays traced as points
    (the same step sequence); the FP64 path promotes nothing; on the mixed
    path every captured base ray took FP64 steps (promotion within 0.1 M of
    the horizon comes before capture at 1.01 R_+)."""
    from paper_2605_05635_gb300 import workloads
    flat = workloads.kerr_64()
    g = _gpu_image(B, flat)
    st, cam, em, it = B.from_flat(flat)
    xy = [pixel_centre(flat, i, j) for j in range(0, 64, 7) for i in range(0, 64, 5)]
    rec = B.trace_points(st, cam, em, it, xy)
    k = 0
    for j in range(0, 64, 7):
        for i in range(0, 64, 5):
            assert g["steps"][0, j, i] == rec[k]["n_accept"]
            assert g["steps"][1, j, i] == rec[k]["n_reject"]
            k += 1
    assert not g["promoted"].any() and (g["steps"][0] > 0).all()
    mixed = _gpu_image(B, dict(flat, **workloads.MIXED_INTEG, chi=0.9))
    captured = mixed["status"] == 1
    assert captured.any() and (mixed["promoted"][captured] == 1).all()
    assert (mixed["steps"][0] > 0).all()
