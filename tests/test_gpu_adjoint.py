"""Gradients from the hand-written discrete adjoint (bh_trace_backward)
against central finite differences of the FP64 oracle with the same adaptive
decisions frozen (each ray replays its nominal accepted step sequence; the
refinement pattern is the nominal one).

Loss: L = sum_p w_p I_p + sum_m c_m D_m with random weights w, c and
D = (centroid offset C, asymmetry A_LR, bright-ring radius rho_peak
(parabolic vertex), |V|/|V(0,0)| at 8 seeded baselines).  Bar: each
component within 1e-4 relative of the finite difference (plus a floor of
1e-6 of the largest component for components that vanish).
"""
import math

import numpy as np
import pytest

from parity import oracle_flat

pytestmark = pytest.mark.gpu

NAMES = ["chi", "incl", "halo1", "halo2", "j0", "p", "R_s", "sigma_in", "sigma_out", "R_out"]


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


def _cells(flat, keys):
    """Screen points and leaf weights of every traced cell of the nominal
    image (base pixels and refined cells), in the oracle's arithmetic."""
    nx, ny = flat["nx"], flat["ny"]
    dx = (flat["x_max"] - flat["x_min"]) / nx
    dy = (flat["y_max"] - flat["y_min"]) / ny

    def split(k):
        lev = (k >> 12) & 0xF
        digits = tuple((k >> (4 * (3 - l))) & 0xF for l in range(1, lev + 1))
        return k >> 16, lev, digits

    cells = [split(int(k)) for k in keys]
    parents = {(b, lev - 1, d[:-1]) for b, lev, d in cells}
    pts, w, pix = [], [], []
    for q in range(nx * ny):
        i, j = q % nx, q // nx
        pts.append((flat["x_min"] + (i + 0.5) * dx, flat["y_min"] + (j + 0.5) * dy))
        w.append(0.0 if (q, 0, ()) in parents else 1.0)
        pix.append(q)
    for b, lev, d in cells:
        i, j = b % nx, b // nx
        X = flat["x_min"] + (i + 0.5) * dx
        Y = flat["y_min"] + (j + 0.5) * dy
        wx, wy = dx, dy
        for dig in d:
            X = X + ((dig % 4 + 0.5) / 4.0 - 0.5) * wx
            Y = Y + ((dig // 4 + 0.5) / 4.0 - 0.5) * wy
            wx, wy = wx / 4.0, wy / 4.0
        pts.append((X, Y))
        w.append(0.0 if (b, lev, d) in parents else 16.0 ** (-lev))
        pix.append(b)
    return np.array(pts), np.array(w), np.array(pix)


def _loss(oracle, flat, I, wI, cdiag, uv8):
    from oracle.diagnostics import diagnostics, rho_peak_smooth
    from oracle.visibility import visibilities
    ext = (flat["x_min"], flat["x_max"], flat["y_min"], flat["y_max"])
    d = diagnostics(I, *ext)
    rho = rho_peak_smooth(I, *ext)
    V = visibilities(I, *ext, np.concatenate([[[0.0, 0.0]], uv8]))
    amp = np.abs(V[1:]) / abs(V[0])
    D = np.concatenate([[d["C"], d["A_LR"], rho], amp])
    return float(np.sum(wI * I) + np.sum(cdiag * D)), D


def _frozen_image(oracle, flat, pts, w, pix, hbuf, counts):
    P = oracle.problem(**oracle_flat(flat, oracle))
    r = oracle.trace_points_frozen(P, pts, hbuf, counts)
    I = np.zeros(flat["nx"] * flat["ny"])
    np.add.at(I, pix, w * r["I_tot"])
    return I.reshape(flat["ny"], flat["nx"])


@pytest.mark.parametrize("metric", [0, 2, 1])
def test_adjoint_matches_frozen_finite_differences(B, oracle, metric):
    import torch
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), metric=metric, chi=0.7, incl=math.radians(50.0), nx=14,
                ny=12, x_min=-12.0, x_max=12.0, y_min=-10.0, y_max=10.0, levels=1, r_in_mode=1,
                **workloads.HALO[metric])
    rng = np.random.default_rng(20260514 + metric)
    wI = rng.normal(size=(flat["ny"], flat["nx"]))
    cdiag = rng.normal(size=11) * np.array([1, 1, 1] + [5] * 8)
    uv8 = workloads.uv_points(8, seed=20260514)
    st, cam, em, it = B.from_flat(flat)
    grad, diag, img = B.trace_backward(st, cam, em, it, dL_dI=torch.from_numpy(wI).float(),
                                       dL_ddiag=cdiag, uv8=uv8)
    keys_gpu = B.trace_image(st, cam, em, it, keys_cap=1 << 16)["refine_keys"].cpu().numpy()
    P0 = oracle.problem(**oracle_flat(flat, oracle))
    nominal = oracle.trace_image(P0)
    assert np.array_equal(np.sort(keys_gpu.astype(np.uint64)), nominal["keys"])
    pts, w, pix = _cells(flat, nominal["keys"])
    rec, hbuf, counts = oracle.trace_points_record(P0, pts, hcap=8000)
    I0 = _frozen_image(oracle, flat, pts, w, pix, hbuf, counts)
    assert np.allclose(I0, nominal["I"], rtol=1e-12, atol=1e-15)
    _, D0 = _loss(oracle, flat, I0, wI, cdiag, uv8)
    assert np.allclose(diag, D0, rtol=1e-5, atol=1e-9)
    keys = {0: "chi", 1: "incl", 2: {1: "lam_E", 2: "eta"}.get(metric), 3: "lam_c" if metric == 2 else None,
            4: "j0", 5: "p", 6: "R_s", 7: "sigma_in", 8: "sigma_out", 9: "R_out"}
    fd = np.zeros(10)
    for k, name in keys.items():
        if name is None:
            continue
        x0 = flat[name]
        h = 1e-6 if name in ("chi", "incl") else 1e-6 * abs(x0)
        lp, _ = _loss(oracle, flat, _frozen_image(oracle, dict(flat, **{name: x0 + h}), pts, w, pix,
                                                  hbuf, counts), wI, cdiag, uv8)
        lm, _ = _loss(oracle, flat, _frozen_image(oracle, dict(flat, **{name: x0 - h}), pts, w, pix,
                                                  hbuf, counts), wI, cdiag, uv8)
        fd[k] = (lp - lm) / (2 * h)
    floor = 1e-6 * np.max(np.abs(fd))
    for k in range(10):
        assert abs(grad[k] - fd[k]) <= 1e-4 * abs(fd[k]) + floor, (NAMES[k], grad[k], fd[k])


def _adjoint256(workloads, metric):
    """The adjoint configuration of the benchmark: 256^2 over +-12 M, a = 0.7,
    i = 50 deg, one refinement level, R_in = R_+ + dR_in."""
    return dict(workloads.kerr_64(), metric=metric, chi=0.7, incl=math.radians(50.0), nx=256,
                ny=256, x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0, levels=1, r_in_mode=1,
                **workloads.HALO[metric])


def _param_names(metric):
    return {0: "chi", 1: "incl", 2: {1: "lam_E", 2: "eta"}.get(metric),
            3: "lam_c" if metric == 2 else None, 4: "j0", 5: "p", 6: "R_s", 7: "sigma_in",
            8: "sigma_out", 9: "R_out"}


# Central differences near the critical curve: a ray at relative distance
# delta from it has derivatives growing like 1/delta^k, so the O(h^2) error
# of a central difference is ~ (h/delta)^2 and at h = 1e-6 is already 1e-4
# for delta ~ 1e-4 (measured on a level-1 cell of the 256^2 Kerr screen).
# The 256^2 tests therefore use h = 4e-8 (absolute for chi and theta_o,
# relative otherwise) and Richardson's extrapolation from h and h/2, whose
# error is O(h^4 / delta^4); FP64 round-off stays near 1e-16 |I| / h.
FD_H = 4e-8


def _fd(oracle, flat, name, image_of, loss_of):
    x0 = flat[name]
    h = FD_H if name in ("chi", "incl") else FD_H * abs(x0)

    def central(hh):
        lp = loss_of(image_of(dict(flat, **{name: x0 + hh})))
        lm = loss_of(image_of(dict(flat, **{name: x0 - hh})))
        return (lp - lm) / (2 * hh)

    return (4.0 * central(0.5 * h) - central(h)) / 3.0


@pytest.mark.parametrize("metric", [0, 2])
def test_adjoint_256_sampled_pixels(B, oracle, metric):
    """256^2 (Kerr and cored-NFW): L = sum of random weights times the
    intensity of 64 sampled pixels (48 refined ones, 16 anywhere); every one
    of the 10 gradient components within 1e-4 of the oracle's frozen central
    difference (Richardson-extrapolated, see FD_H; floor 1e-6 of the
    largest), using only those pixels' cells."""
    import torch
    from paper_2605_05635_gb300 import workloads
    flat = _adjoint256(workloads, metric)
    st, cam, em, it = B.from_flat(flat)
    out = B.trace_image(st, cam, em, it, keys_cap=1 << 22)
    lvl = out["refine_level"].cpu().numpy()
    keys_gpu = out["refine_keys"][: int(out["refine_keys_count"][0])].cpu().numpy().astype(np.uint64)
    rng = np.random.default_rng(256 + metric)
    refined = np.argwhere(lvl > 0)
    picks = [tuple(refined[k]) for k in rng.choice(len(refined), 48, replace=False)]
    picks += [tuple(x) for x in rng.integers(0, 256, (16, 2))]
    wI = np.zeros((256, 256))
    for j, i in picks:
        wI[j, i] = rng.normal()
    grad, _, _ = B.trace_backward(st, cam, em, it, dL_dI=torch.from_numpy(wI).float())
    P0 = oracle.problem(**oracle_flat(flat, oracle))
    keys = []
    for j, i in set(picks):
        px = oracle.trace_pixel(P0, int(i), int(j))
        mine = keys_gpu[(keys_gpu >> np.uint64(16)) == np.uint64(j * 256 + i)]
        assert np.array_equal(np.sort(mine), px["keys"]), (i, j)
        keys.extend(px["keys"].tolist())
    pts, w, pix = _cells(flat, np.array(keys, dtype=np.uint64))
    sel = np.isin(pix, [j * 256 + i for j, i in set(picks)])
    pts, w, pix = pts[sel], w[sel], pix[sel]
    _, hbuf, counts = oracle.trace_points_record(P0, pts, hcap=12000)

    def image_of(f):
        return _frozen_image(oracle, f, pts, w, pix, hbuf, counts)

    def loss_of(I):
        return float(np.sum(wI * I))

    fd = np.zeros(10)
    for k, name in _param_names(metric).items():
        if name is not None:
            fd[k] = _fd(oracle, flat, name, image_of, loss_of)
    floor = 1e-6 * np.max(np.abs(fd))
    for k in range(10):
        assert abs(grad[k] - fd[k]) <= 1e-4 * abs(fd[k]) + floor, (NAMES[k], grad[k], fd[k])


def test_adjoint_256_diagnostics(B, oracle):
    """256^2 cored-NFW: L = random combination of C, A_LR, rho_peak and the
    8 normalised visibility amplitudes (every pixel contributes); dL/dchi and
    dL/deta within 1e-4 of the oracle's frozen central differences over the
    whole image (Richardson-extrapolated, see FD_H)."""
    from paper_2605_05635_gb300 import workloads
    metric = 2
    flat = _adjoint256(workloads, metric)
    rng = np.random.default_rng(20260514)
    cdiag = rng.normal(size=11) * np.array([1, 1, 1] + [5] * 8)
    uv8 = workloads.uv_points(8, seed=20260514)
    st, cam, em, it = B.from_flat(flat)
    grad, diag, _ = B.trace_backward(st, cam, em, it, dL_ddiag=cdiag, uv8=uv8)
    keys_gpu = B.trace_image(st, cam, em, it, keys_cap=1 << 22)["refine_keys"].cpu().numpy()
    P0 = oracle.problem(**oracle_flat(flat, oracle))
    nominal = oracle.trace_image(P0)
    assert np.array_equal(np.sort(keys_gpu.astype(np.uint64)), nominal["keys"])
    pts, w, pix = _cells(flat, nominal["keys"])
    zero = np.zeros((flat["ny"], flat["nx"]))
    _, D0 = _loss(oracle, flat, nominal["I"], zero, cdiag, uv8)
    assert np.allclose(diag, D0, rtol=1e-5, atol=1e-9)
    # frozen images at chi +- h and eta +- h, recorded and replayed in chunks
    # of cells so that the step records stay small
    params = ((0, "chi"), (2, "eta"))
    steps = {name: (FD_H if name == "chi" else FD_H * abs(flat[name])) for _, name in params}
    shifts = [(name, sg * f) for _, name in params for sg in (1, -1) for f in (1.0, 0.5)]
    imgs = {sh: np.zeros(flat["nx"] * flat["ny"]) for sh in shifts}
    for c0 in range(0, len(pts), 4096):
        sl = slice(c0, c0 + 4096)
        _, hbuf, counts = oracle.trace_points_record(P0, pts[sl], hcap=20000)
        for (name, f), acc in imgs.items():
            Pf = oracle.problem(**oracle_flat(dict(flat, **{name: flat[name] + f * steps[name]}),
                                              oracle))
            r = oracle.trace_points_frozen(Pf, pts[sl], hbuf, counts)
            np.add.at(acc, pix[sl], w[sl] * r["I_tot"])

    def loss(name, f):
        return _loss(oracle, flat, imgs[(name, f)].reshape(zero.shape), zero, cdiag, uv8)[0]

    for k, name in params:
        h = steps[name]
        d1 = (loss(name, 1.0) - loss(name, -1.0)) / (2 * h)
        d2 = (loss(name, 0.5) - loss(name, -0.5)) / h
        fd = (4.0 * d2 - d1) / 3.0
        assert abs(grad[k] - fd) <= 1e-4 * abs(fd) + 1e-10, (NAMES[k], grad[k], fd)


def test_adjoint_long_rays(B):
    """Rays longer than the default checkpoint slab (64 checkpoints of 64
    steps = 4096 accepted steps): Kerr a = 0.9 seen at i = 80 deg on a 64^2
    screen straddling the critical curve (X in [3.9, 4.9], |Y| <= 0.5), three
    refinement levels, rtol 1e-15 -- the longest ray takes more than 4096
    steps (4710 measured on GB300).  The adjoint sizes its slabs from the
    forward pass and returns finite gradients without a workspace error."""
    import torch
    from paper_2605_05635_gb300 import workloads
    flat = dict(workloads.kerr_64(), chi=0.9, incl=math.radians(80.0), nx=64, ny=64, x_min=3.9,
                x_max=4.9, y_min=-0.5, y_max=0.5, levels=3, rtol=1e-15, atol=1e-17)
    items = [B.from_flat(flat)]
    plan = B.Plan(items)
    plan.launch()
    plan.check()
    longest = plan.stats()["max_ray_steps"]
    plan.close()
    assert longest > 4096
    st, cam, em, it = items[0]
    wI = torch.from_numpy(np.random.default_rng(4).normal(size=(64, 64))).float()
    grad, _, img = B.trace_backward(st, cam, em, it, dL_dI=wI)
    assert np.all(np.isfinite(grad)) and np.any(grad != 0.0)
    assert float(img.abs().max()) > 0.0
