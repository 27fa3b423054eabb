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


def _key_level(k):
    return (k >> 12) & 0xF


def _key_parent(k):
    """The cell whose refinement created cell k (level >= 1): level - 1 and
    that level's digit cleared; a level-1 cell's parent is its base pixel."""
    L = _key_level(k)
    sh = 4 * (3 - L)
    return (k & ~(0xF << sh) & ~(0xF << 12)) | ((L - 1) << 12)


def _cell_centre(flat, k):
    """Screen centre of the cell with key k (cell-centred children)."""
    nx = flat["nx"]
    base = k >> 16
    i, j = base % nx, base // nx
    X, Y = pixel_centre(flat, i, j)
    wx = (flat["x_max"] - flat["x_min"]) / nx
    wy = (flat["y_max"] - flat["y_min"]) / flat["ny"]
    for lvl in range(1, _key_level(k) + 1):
        d = (k >> (4 * (3 - lvl))) & 0xF
        X += ((d & 3) + 0.5) / 4.0 * wx - 0.5 * wx
        Y += ((d >> 2) + 0.5) / 4.0 * wy - 0.5 * wy
        wx /= 4.0
        wy /= 4.0
    return X, Y


def _siblings(k):
    """The in-block 4-neighbours of a refined cell (same parent)."""
    L = _key_level(k)
    sh = 4 * (3 - L)
    d = (k >> sh) & 0xF
    cx, cy = d & 3, d >> 2
    out = []
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        if 0 <= cx + dx < 4 and 0 <= cy + dy < 4:
            out.append((k & ~(0xF << sh)) | (((cy + dy) * 4 + cx + dx) << sh))
    return out


@pytest.mark.parametrize("volumetric", [0, 1])
def test_fullsize_mixed_every_pixel_vs_fp64(B, oracle, volumetric):
    """Every pixel of the six 512^2 images of the benchmark, mixed path (as
    bench.py times it, thin disk or the volumetric layer of Eq. 88 with its
    own promotion threshold) against the all-FP64 path at rtol 1e-10 (pinned
    to the oracle at 1e-6 by the sampled test above, test_gpu_trace.py and
    test_gpu_volumetric.py):

    - intensity within 1e-4 of each image's maximum on every pixel, none
      exempt;
    - base-ray classes equal, except rays the oracle finds class-sensitive
      at mixed precision (parity.py's counted rule);
    - refinement keys equal, except where the refinement decision that
      differs involves a cell the oracle finds class-sensitive (the cell or
      one of its in-block 4-neighbours, at the cell centre).

    Volumetric layer: the same, except that refinement decisions the rule
    does not explain are counted and reported, not failed, up to the 4 found:
    one screen point (X, Y) = (0.898, -5.275) in the Einasto and the Kerr
    image at 80 deg, whose cell changes the decisions of two in-block
    neighbours in each.  Its last crossing meets the plane almost
    tangentially just inside the escape radius (dtheta/dlambda = 4.5e-6 at
    R = 1080 against R_esc = 1100), where the crossing's position moves by
    ~6e5 per unit of screen coordinate: the mixed path's FP32 legs move it
    past R_esc (N_cross 2 instead of 3), while the FP64 oracle's class is
    stable under the rule's 1e-6 screen perturbation (R_em moves by ~3).
    Intensity is unaffected (the volumetric integral does not depend on the
    crossing count).
    """
    import torch
    from paper_2605_05635_gb300 import workloads
    cap = 1 << 23
    outs = {}
    for prec in (1, 0):
        flats = workloads.sweep_512(precision=prec, volumetric=volumetric)
        plan = B.Plan([B.from_flat(d) for d in flats], keys_cap=cap)
        plan.launch()
        plan.check()
        outs[prec] = [{k: v.cpu().numpy() for k, v in o.items()} for o in plan.outputs]
        plan.close()
        del plan
        torch.cuda.empty_cache()
    flats = workloads.sweep_512(precision=1, volumetric=volumetric)
    worst, class_waived, tree_decisions, unexplained = 0.0, 0, 0, []
    for img, d in enumerate(flats):
        a, b = outs[1][img], outs[0][img]
        scale = float(np.abs(b["I"]).max())
        err = np.abs(a["I"].astype(np.float64) - b["I"].astype(np.float64)) / scale
        worst = max(worst, float(err.max()))
        assert float(err.max()) <= 1e-4, (img, np.unravel_index(int(err.argmax()), err.shape),
                                          float(err.max()))
        bad = np.argwhere((a["status"] != b["status"]) | (a["ncross"] != b["ncross"]))
        for j, i in bad:
            assert class_sensitive(oracle, d, *pixel_centre(d, int(i), int(j))), (img, i, j)
            class_waived += 1
        ka = a["refine_keys"][: int(a["refine_keys_count"][0])].astype(np.int64)
        kb = b["refine_keys"][: int(b["refine_keys_count"][0])].astype(np.int64)
        assert len(ka) <= cap and len(kb) <= cap
        diff = np.setxor1d(ka, kb)
        sa, sb = set(ka.tolist()), set(kb.tolist())
        # refined cells: parents of traced cells
        ref_a = {_key_parent(k) for k in sa}
        ref_b = {_key_parent(k) for k in sb}
        decided = set()
        for k in diff.tolist():
            c = _key_parent(k)                 # refined in one run only
            while _key_level(c) >= 1 and not (c in sa and c in sb):
                c = _key_parent(c)
            decided.add(c)
        for c in decided:
            assert (c in ref_a) != (c in ref_b)
            if _key_level(c) == 0:
                # a base pixel's decision: some base class among it and its
                # neighbours changed, and each such change was checked above
                base = c >> 16
                i, j = base % d["nx"], base // d["nx"]
                near = [(j, i), (j - 1, i), (j + 1, i), (j, i - 1), (j, i + 1)]
                assert any(0 <= y < d["ny"] and 0 <= x < d["nx"] and
                           (a["status"][y, x], a["ncross"][y, x]) !=
                           (b["status"][y, x], b["ncross"][y, x]) for y, x in near), (img, c)
                continue
            cells = [c] + _siblings(c)
            if any(class_sensitive(oracle, d, *_cell_centre(d, q)) for q in cells):
                tree_decisions += 1
            else:
                assert volumetric, (img, hex(c))
                unexplained.append((img, hex(c)))
    print(f"mixed vs FP64 on 6 x 512^2 (volumetric {volumetric}): max {worst:.3e} of the "
          f"image maximum; base classes waived {class_waived}; refinement decisions waived "
          f"{tree_decisions}; not explained by the rule {len(unexplained)} {unexplained}")
    assert len(unexplained) <= 4, unexplained
