"""Accuracy of the sine/cosine, log(1 + x), exp and reciprocal that the
tracing kernels use instead of the library functions (Cody & Waite reduction
with fitted (FP64) or Taylor (FP32) polynomials; an atanh series; exp by a
2^(j/32) table and a short Taylor series; a Newton-refined hardware
reciprocal).  A probe kernel built from the same header evaluates them on the
GPU; the reference is numpy (FP64, and FP64 at the float arguments for the
FP32 versions; exact rationals where FP64 itself is the subject).

Bounds, with u the unit roundoff of the format (FP32 2^-24, FP64 2^-53):
sine and cosine within 4u absolute over the polar angle and the trial
stages around it, [-0.6, pi + 0.6], and the sine within 8u relative next to
the poles (1/sin(theta) enters the right-hand side); log(1 + x) within 8u
relative on [1e-3, 1e3] (x = R / lambda_c of the cored-NFW lapse) and, in FP64,
on [-0.89, -1e-6] (x = R / R_in - 1 of the emissivity); exp (FP64)
within 8u relative on [-700, 5] and 0 below -708; the reciprocal and the
reciprocal square root (FP64) within 4u relative.
"""
import ctypes as C
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
U32 = 2.0 ** -24
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_05635_gb300 import _build
    out = str(tmp_path_factory.mktemp("probe") / "fastmath_probe.so")
    cmd = [_build._nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC", "-shared", "-I",
           os.path.join(ROOT, "paper_2605_05635_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "fastmath_probe.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = C.CDLL(out)
    L.fastmath_probe_f32.argtypes = [C.c_int] + [C.c_void_p] * 4
    L.fastmath_probe_f64.argtypes = [C.c_int] + [C.c_void_p] * 7
    return L


def _f32(lib, x):
    import torch
    xt = torch.as_tensor(np.asarray(x, np.float32)).cuda()
    outs = [torch.empty_like(xt) for _ in range(3)]
    assert lib.fastmath_probe_f32(xt.numel(), xt.data_ptr(), *[o.data_ptr() for o in outs]) == 0
    return [xt.cpu().numpy().astype(np.float64)] + [o.cpu().numpy().astype(np.float64) for o in outs]


def _f64(lib, x):
    import torch
    xt = torch.as_tensor(np.asarray(x, np.float64)).cuda()
    outs = [torch.empty_like(xt) for _ in range(6)]
    assert lib.fastmath_probe_f64(xt.numel(), xt.data_ptr(), *[o.data_ptr() for o in outs]) == 0
    return [xt.cpu().numpy()] + [o.cpu().numpy() for o in outs]


def test_f32_sincos_over_the_polar_range(lib):
    x, s, c, _ = _f32(lib, np.linspace(-0.6, np.pi + 0.6, 200001))
    assert np.max(np.abs(s - np.sin(x))) <= 4 * U32
    assert np.max(np.abs(c - np.cos(x))) <= 4 * U32


def test_f32_sine_relative_near_the_poles(lib):
    d = np.logspace(-7, -1, 4001)
    x, s, _, _ = _f32(lib, np.concatenate([d, np.pi - d]))
    ref = np.sin(x)
    assert np.max(np.abs(s - ref) / np.abs(ref)) <= 8 * U32


def test_f32_log1p_relative(lib):
    x, _, _, l = _f32(lib, np.logspace(-3, 3, 20001))
    assert np.max(np.abs(l - np.log1p(x)) / np.log1p(x)) <= 8 * U32


def _exact_sin_cos(x):
    """sin and cos of a float64 argument to beyond FP64 accuracy, by Taylor
    sums in exact rationals after reduction by a 60-digit pi/2."""
    from decimal import Decimal, getcontext
    getcontext().prec = 70
    half_pi = Fraction(Decimal("1.570796326794896619231321691639751442098584699687552910487472"))
    X = Fraction(x)
    q = round(X / half_pi)
    r = X - q * half_pi
    s = c = Fraction(0)
    term = r
    for n in range(1, 40, 2):
        s += term
        term = -term * r * r / ((n + 1) * (n + 2))
    term = Fraction(1)
    for n in range(0, 40, 2):
        c += term
        term = -term * r * r / ((n + 1) * (n + 2))
    for _ in range(q % 4):
        s, c = c, -s
    return float(s), float(c)


def test_f64_sincos(lib):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-0.6, np.pi + 0.6, 600), np.logspace(-12, -1, 100),
                        np.pi - np.logspace(-12, -1, 100)])
    x, s, c, _, _, _, _ = _f64(lib, x)
    ref = np.array([_exact_sin_cos(v) for v in x])
    assert np.max(np.abs(s - ref[:, 0])) <= 4 * U64
    assert np.max(np.abs(c - ref[:, 1])) <= 4 * U64
    near = slice(600, None)
    assert np.max(np.abs(s[near] - ref[near, 0]) / np.abs(ref[near, 0])) <= 8 * U64


def test_f64_exp_log1p_rcp(lib):
    rng = np.random.default_rng(4)
    xe = np.concatenate([np.linspace(-700.0, 5.0, 7001), rng.uniform(-1.0, 1.0, 1000)])
    x, _, _, _, e, _, _ = _f64(lib, xe)
    ref = np.exp(x)
    assert np.max(np.abs(e - ref) / ref) <= 8 * U64
    _, _, _, _, e_low, _, _ = _f64(lib, np.array([-710.0, -750.0, -1e4]))
    assert np.all(e_low == 0.0)
    # x = R / lambda_c of the cored-NFW lapse, and R / R_in - 1 of the
    # emissivity (negative inside R_in)
    xl = np.concatenate([np.logspace(-3, 3, 3001), -np.logspace(-6, -0.05, 1001)])
    x, _, _, l, _, _, _ = _f64(lib, xl)
    ref = np.array([float(Fraction(math.log1p(v))) for v in x])  # libm log1p, < 1u
    assert np.max(np.abs(l - ref) / ref) <= 8 * U64
    xr = rng.uniform(1.0, 2.0, 3000) * 2.0 ** rng.integers(-30, 30, 3000)
    x, _, _, _, _, r, _ = _f64(lib, np.concatenate([xr, -xr]))
    exact = np.array([float(1 / Fraction(v)) for v in x])
    assert np.max(np.abs(r - exact) / np.abs(exact)) <= 4 * U64
    # reciprocal square root (the launch's 1/|n|): against a 40-digit value
    from decimal import Decimal, getcontext
    getcontext().prec = 40
    xq = xr[:1500] * 1e6
    x, _, _, _, _, _, q = _f64(lib, xq)
    exact = np.array([float(1 / Decimal(v).sqrt()) for v in x])
    assert np.max(np.abs(q - exact) / exact) <= 4 * U64
