"""Seeded synthetic workloads shaped like the paper's images.

Holds parameters and seeded random draws only (no arithmetic of the method),
as flat dicts in the oracle's naming; ``bhrt.from_flat`` turns a dict into the
library's structs and ``oracle.problem(**d)`` into the oracle's.

Halo readings: Einasto lambda_E = 0.1 (the paper's lambda_E = 0.3 is
horizonless above chi = 0.64, Fig. 2), cored-NFW eta = 0.02, lambda_c = 10
(Fig. 5 caption).  Emissivity constants are readings (the paper prints none).
"""
from __future__ import annotations

import math

import numpy as np

KERR, EINASTO, CNFW = 0, 1, 2

HALO = {KERR: {}, EINASTO: dict(lam_E=0.1), CNFW: dict(eta=0.02, lam_c=10.0)}

EMISSION = dict(r_in_mode=0, j0=1.0, p=2.0, R_s=8.0, sigma_in=0.2, sigma_out=2.0, R_out=20.0,
                dR_in=0.5, H0=0.05, h=0.05)

FP64_INTEG = dict(precision=0, rtol=1e-10, atol=1e-12, max_steps=1_000_000, cap_factor=1.01,
                  esc_factor=1.1, thetadot_min=1e-8, dlambda_min=1e-6, promote_dr=0.1)

# Mixed path: FP32 bulk with FP64 promotion; its step tolerances sit above
# the FP32 round-off floor of the error estimate (an absolute tolerance
# below about 1e-8 only adds rejected steps where a component passes
# through zero, without changing the images); rays within 3e-3 of a double
# root of their radial potential take FP64 steps (promote_turning).
MIXED_INTEG = dict(FP64_INTEG, precision=1, rtol=1e-8, atol=1e-8, promote_turning=3e-3)
# The volumetric layer (Eq. 88) integrates the source along the whole path, so
# near-critical rays need their FP64 steps from further out: kappa = 3e-2.
VOLUMETRIC_TURNING = 3e-2


def kerr_64():
    """Kerr a = 0.5, i = 17 deg, 64 x 64 over [-10, 10]^2, R_o = 1000,
    no refinement, FP64, rtol 1e-10: the small case the oracle finishes in
    seconds."""
    return dict(metric=KERR, chi=0.5, incl=math.radians(17.0), r_obs=1000.0, nx=64, ny=64,
                x_min=-10.0, x_max=10.0, y_min=-10.0, y_max=10.0, levels=0, **EMISSION,
                **FP64_INTEG)


def sweep_512(precision=0, volumetric=0):
    """Six 512^2 images: {Einasto, cored-NFW, Kerr} x i in {17, 80} deg at
    a = 0.9, +-12 M, 4x4 refinement to 3 levels; thin disk, or with
    ``volumetric`` the layer of Eqs. 83-88 (H0 = h = 0.05) integrated along
    the ray."""
    out = []
    for metric in (EINASTO, CNFW, KERR):
        for inc in (17.0, 80.0):
            d = dict(metric=metric, chi=0.9, incl=math.radians(inc), r_obs=1000.0, nx=512,
                     ny=512, x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0, levels=3,
                     **HALO[metric], **EMISSION, volumetric=int(volumetric),
                     **(MIXED_INTEG if precision == 1 else FP64_INTEG))
            if precision == 1 and volumetric:
                d["promote_turning"] = VOLUMETRIC_TURNING
            out.append(d)
    return out


def shadow_fig5(n_psi=4096):
    """Shadow boundaries of Fig. 5: Kerr, Einasto (lambda_E = 0.3) and
    cored-NFW (eta = 0.02, lambda_c = 10) at a = 0.5, i = 60 deg, R_o = 1000,
    n_psi directions uniform in [0, 2 pi), b bracketed in [1, 9] to 1e-10,
    FP64 at rtol 1e-10.  Returns (flats, psi, b_lo, b_hi, b_tol)."""
    flats = [dict(metric=m, chi=0.5, incl=math.radians(60.0), r_obs=1000.0, nx=1, ny=1,
                  x_min=-1.0, x_max=1.0, y_min=-1.0, y_max=1.0, levels=0, **EMISSION,
                  **FP64_INTEG, **h)
             for m, h in ((KERR, {}), (EINASTO, dict(lam_E=0.3)),
                          (CNFW, dict(eta=0.02, lam_c=10.0)))]
    psi = [2.0 * math.pi * k / n_psi for k in range(n_psi)]
    return flats, psi, 1.0, 9.0, 1e-10


def geometry_grid(n=1024, n_theta=16):
    """Parameter grids of Figs. 3-4: Einasto (chi, lambda_E) over [0, 1.2] x
    [0.05, 1] and cored-NFW (chi, eta) over [0, 1.2] x [0, 0.3] at
    lambda_c = 10, n x n each (chi slowest), and n_theta polar angles in
    [0, pi/2] for the stationary-limit surface.  Returns numpy arrays
    (metric, chi, lambda_E, eta, lambda_c) of length 2 n^2 and theta."""
    import numpy as np
    chi = np.repeat(np.linspace(0.0, 1.2, n), n)
    u = np.tile(np.linspace(0.0, 1.0, n), n)
    metric = np.concatenate([np.full(n * n, EINASTO), np.full(n * n, CNFW)]).astype(np.int32)
    lam_E = np.concatenate([0.05 + 0.95 * u, np.full(n * n, 0.1)])
    eta = np.concatenate([np.full(n * n, 0.02), 0.3 * u])
    lam_c = np.full(2 * n * n, 10.0)
    theta = np.linspace(0.0, 0.5 * math.pi, n_theta)
    return metric, np.concatenate([chi, chi]), lam_E, eta, lam_c, theta


def sweep_96(seed=20260513, n=256):
    """96 images: 3 metrics x 8 spins x 4 inclinations, n^2 over +-12 M with
    refinement; halo parameters jittered x U(0.8, 1.2) in image order
    (metric-major, then spin, then inclination)."""
    rng = np.random.default_rng(seed)
    spins = [0.0, 0.3, 0.5, 0.7, 0.8, 0.9, 0.94, 0.98]
    incs = [17.0, 30.0, 50.0, 80.0]
    out = []
    for metric in (KERR, EINASTO, CNFW):
        for chi in spins:
            for inc in incs:
                halo = {k: v * rng.uniform(0.8, 1.2) for k, v in HALO[metric].items()}
                d = dict(metric=metric, chi=chi, incl=math.radians(inc), r_obs=1000.0, nx=n,
                         ny=n, x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0, levels=3,
                         **halo, **EMISSION, **FP64_INTEG)
                out.append(d)
    return out


def vis_1024(precision=1):
    """One 1024^2 cored-NFW image (a = 0.94, i = 17 deg, +-12 M, 4x4
    refinement to 3 levels): the input of the visibility benchmark."""
    return dict(metric=CNFW, chi=0.94, incl=math.radians(17.0), r_obs=1000.0, nx=1024, ny=1024,
                x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0, levels=3, **HALO[CNFW],
                **EMISSION, **(MIXED_INTEG if precision == 1 else FP64_INTEG))


def fig12_images(precision=1, n=1024):
    """The Fig. 12 images: Kerr, Einasto (lambda_E = 0.1) and cored-NFW at
    a = 0.95, i = 70 deg, n x n over +-12 M, 4x4 refinement to 3 levels."""
    return [dict(metric=m, chi=0.95, incl=math.radians(70.0), r_obs=1000.0, nx=n, ny=n,
                 x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0, levels=3, **HALO[m],
                 **EMISSION, **(MIXED_INTEG if precision == 1 else FP64_INTEG))
            for m in (KERR, EINASTO, CNFW)]


def uv_points(k, seed, theta_g_muas=3.8, b_max_glambda=15.0):
    """k baselines with |b| ~ U(0, b_max) G-lambda and position angle
    ~ U(0, pi), returned as (u, v) in cycles per M: u = b theta_g."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(0.0, b_max_glambda, k) * 1e9
    pa = rng.uniform(0.0, math.pi, k)
    theta_g = theta_g_muas * 1e-6 / 3600.0 * math.pi / 180.0
    return np.stack([b * np.cos(pa) * theta_g, b * np.sin(pa) * theta_g], 1)
