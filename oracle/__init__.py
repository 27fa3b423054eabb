"""Plain FP64 CPU oracle for the ray-tracing path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never calls it, and it imports nothing from the CUDA package.

The numerics live in ``bh_oracle.c`` (one ray at a time, IEEE double, FMA
contraction off); this module only marshals arguments through ctypes.
``diagnostics.py`` and ``visibility.py`` hold the image-product oracles in
numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bh_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_bh_oracle.so")
_lock = threading.Lock()
_lib = None

KERR, EINASTO, CNFW = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``bh_oracle.c`` into ``_bh_oracle.so`` with gcc (OpenMP, -O2,
    no FMA contraction so that results do not depend on the host ISA)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(C.Structure):
    _fields_ = [
        ("metric", C.c_int32), ("r_in_mode", C.c_int32), ("levels", C.c_int32),
        ("max_steps", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("volumetric", C.c_int32), ("pad1", C.c_int32),
        ("chi", C.c_double), ("lam_E", C.c_double), ("eta", C.c_double), ("lam_c", C.c_double),
        ("r_obs", C.c_double), ("incl", C.c_double),
        ("x_min", C.c_double), ("x_max", C.c_double), ("y_min", C.c_double), ("y_max", C.c_double),
        ("j0", C.c_double), ("p", C.c_double), ("R_s", C.c_double), ("sigma_in", C.c_double),
        ("sigma_out", C.c_double), ("R_out", C.c_double), ("dR_in", C.c_double),
        ("H0", C.c_double), ("h", C.c_double),
        ("rtol", C.c_double), ("atol", C.c_double), ("cap_factor", C.c_double),
        ("esc_factor", C.c_double), ("thetadot_min", C.c_double), ("dlambda_min", C.c_double),
    ]


class Ray(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("ncross", C.c_int32), ("n_accept", C.c_int32),
        ("n_reject", C.c_int32),
        ("I_tot", C.c_double), ("I_n", C.c_double * 3),
        ("R_em", C.c_double * 3), ("phi_em", C.c_double * 3), ("T_em", C.c_double * 3),
        ("g", C.c_double * 3), ("thdot", C.c_double * 3), ("lam_cross", C.c_double * 3),
        ("R_min", C.c_double), ("R_final", C.c_double), ("lam_final", C.c_double),
        ("h_drift", C.c_double), ("E", C.c_double), ("ell", C.c_double),
        ("K0", C.c_double), ("K_final", C.c_double),
        ("near_thdot", C.c_double), ("near_dlam", C.c_double),
    ]


class _Image(C.Structure):
    _fields_ = [
        ("I", C.POINTER(C.c_double)), ("I_n", C.POINTER(C.c_double)),
        ("ncross", C.POINTER(C.c_int32)), ("status", C.POINTER(C.c_int32)),
        ("level", C.POINTER(C.c_int32)),
        ("R_em", C.POINTER(C.c_double)), ("phi_em", C.POINTER(C.c_double)),
        ("T_em", C.POINTER(C.c_double)), ("g", C.POINTER(C.c_double)),
        ("h_drift", C.POINTER(C.c_double)),
        ("keys", C.POINTER(C.c_uint64)), ("keys_cap", C.c_int64), ("keys_count", C.c_int64),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB_PATH)
        P = C.POINTER(Problem)
        D = C.POINTER(C.c_double)
        lib.orc_H.argtypes = [P, C.c_double]; lib.orc_H.restype = C.c_double
        lib.orc_dH.argtypes = [P, C.c_double]; lib.orc_dH.restype = C.c_double
        lib.orc_mu.argtypes = [P, C.c_double]; lib.orc_mu.restype = C.c_double
        lib.orc_Delta.argtypes = [P, C.c_double]; lib.orc_Delta.restype = C.c_double
        for fn in ("orc_metric", "orc_dmetric_dR", "orc_metric_inv"):
            getattr(lib, fn).argtypes = [P, C.c_double, C.c_double, D]
            getattr(lib, fn).restype = None
        lib.orc_dmetric_inv.argtypes = [P, C.c_double, C.c_double, D, D]
        lib.orc_two_hamiltonian.argtypes = [P, C.c_double, C.c_double, D]
        lib.orc_two_hamiltonian.restype = C.c_double
        lib.orc_rhs.argtypes = [P, C.c_double, C.c_double, D, D]
        lib.orc_carter.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double]
        lib.orc_carter.restype = C.c_double
        lib.orc_horizon.argtypes = [P, D]; lib.orc_horizon.restype = C.c_int
        lib.orc_extremal_spin.argtypes = [P, D]; lib.orc_extremal_spin.restype = C.c_double
        lib.orc_circular.argtypes = [P, C.c_double, D, D]; lib.orc_circular.restype = C.c_int
        lib.orc_isco.argtypes = [P, D]; lib.orc_isco.restype = C.c_int
        lib.orc_ergosurface.argtypes = [P, C.c_double, D]
        lib.orc_ergosurface.restype = C.c_int
        lib.orc_emissivity.argtypes = [P, C.c_double, C.c_double, C.c_double]
        lib.orc_emissivity.restype = C.c_double
        lib.orc_launch.argtypes = [P, C.c_double, C.c_double, D, D, D, D, D]
        lib.orc_dp5_solve.argtypes = [C.c_int, C.c_double, C.c_int, D, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_int]
        lib.orc_dp5_solve.restype = C.c_int
        lib.orc_dp5_step_dense.argtypes = [C.c_int, C.c_double, C.c_int, D, C.c_double, D, D,
                                           C.c_int, D, D]
        lib.orc_dp5_step_dense.restype = C.c_int
        lib.orc_trace_points.argtypes = [P, C.c_int64, D, C.POINTER(Ray)]
        lib.orc_trace_points.restype = C.c_int
        lib.orc_trace_image.argtypes = [P, C.POINTER(_Image)]
        lib.orc_trace_image.restype = C.c_int
        lib.orc_trace_pixel.argtypes = [P, C.c_int, C.c_int, C.POINTER(Ray), D,
                                        C.POINTER(C.c_int32), C.POINTER(C.c_uint64), C.c_int64,
                                        C.POINTER(C.c_int64)]
        lib.orc_trace_pixel.restype = C.c_int
        lib.orc_geometry.argtypes = [P, D]; lib.orc_geometry.restype = C.c_int
        lib.orc_trace_pixels.argtypes = [P, C.c_int64, C.POINTER(C.c_int32), D,
                                         C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
        lib.orc_trace_pixels.restype = C.c_int
        lib.orc_shadow_boundary.argtypes = [P, C.c_int64, D, C.c_double, C.c_double, C.c_double,
                                            D, D, C.POINTER(C.c_int32)]
        lib.orc_shadow_boundary.restype = C.c_int
        lib.orc_trace_points_record.argtypes = [P, C.c_int64, D, C.POINTER(Ray), D, C.c_int,
                                                C.POINTER(C.c_int32)]
        lib.orc_trace_points_record.restype = C.c_int
        lib.orc_trace_points_frozen.argtypes = [P, C.c_int64, D, D, C.c_int,
                                                C.POINTER(C.c_int32), C.POINTER(Ray)]
        lib.orc_trace_points_frozen.restype = C.c_int
        _lib = lib
        return lib


# Defaults for the readings the paper leaves open (integrator, emissivity
# constants, thresholds).  Every one is a parameter.
DEFAULTS = dict(
    metric=KERR, r_in_mode=0, levels=0, max_steps=1_000_000, nx=64, ny=64, volumetric=0,
    chi=0.5, lam_E=0.1, eta=0.02, lam_c=10.0, r_obs=1000.0, incl=np.deg2rad(17.0),
    x_min=-10.0, x_max=10.0, y_min=-10.0, y_max=10.0,
    j0=1.0, p=2.0, R_s=8.0, sigma_in=0.2, sigma_out=2.0, R_out=20.0, dR_in=0.5, H0=0.05, h=0.05,
    rtol=1e-10, atol=1e-12, cap_factor=1.01, esc_factor=1.1, thetadot_min=1e-8,
    dlambda_min=1e-6,
)


def problem(**kw) -> Problem:
    """Build a ``Problem`` from the defaults overridden by ``kw``."""
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown oracle parameters: {sorted(unknown)}")
    d.update(kw)
    p = Problem()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def H(P: Problem, R: float) -> float:
    return _load().orc_H(C.byref(P), R)


def dH(P: Problem, R: float) -> float:
    return _load().orc_dH(C.byref(P), R)


def mu(P: Problem, R: float) -> float:
    return _load().orc_mu(C.byref(P), R)


def Delta(P: Problem, R: float) -> float:
    return _load().orc_Delta(C.byref(P), R)


def metric(P: Problem, R: float, th: float) -> np.ndarray:
    g = np.zeros(16)
    _load().orc_metric(C.byref(P), R, th, _dp(g))
    return g.reshape(4, 4)


def dmetric_dR(P: Problem, R: float, th: float) -> np.ndarray:
    g = np.zeros(16)
    _load().orc_dmetric_dR(C.byref(P), R, th, _dp(g))
    return g.reshape(4, 4)


def metric_inv(P: Problem, R: float, th: float) -> np.ndarray:
    g = np.zeros(16)
    _load().orc_metric_inv(C.byref(P), R, th, _dp(g))
    return g.reshape(4, 4)


def dmetric_inv(P: Problem, R: float, th: float):
    a, b = np.zeros(16), np.zeros(16)
    _load().orc_dmetric_inv(C.byref(P), R, th, _dp(a), _dp(b))
    return a.reshape(4, 4), b.reshape(4, 4)


def two_hamiltonian(P: Problem, R: float, th: float, p) -> float:
    p = np.ascontiguousarray(p, dtype=np.float64)
    return _load().orc_two_hamiltonian(C.byref(P), R, th, _dp(p))


def rhs(P: Problem, E: float, ell: float, y) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64)
    dy = np.zeros(6)
    _load().orc_rhs(C.byref(P), E, ell, _dp(y), _dp(dy))
    return dy


def carter(P: Problem, E: float, ell: float, th: float, pth: float) -> float:
    return _load().orc_carter(C.byref(P), E, ell, th, pth)


def horizon(P: Problem):
    r = C.c_double(0.0)
    rc = _load().orc_horizon(C.byref(P), C.byref(r))
    return None if rc else r.value


def extremal_spin(P: Problem):
    Re = C.c_double(0.0)
    chi_e = _load().orc_extremal_spin(C.byref(P), C.byref(Re))
    return chi_e, Re.value


def ergosurface(P: Problem, th: float):
    """Outer stationary-limit radius R_s(theta) (Eq. 40), or None."""
    r = C.c_double(0.0)
    rc = _load().orc_ergosurface(C.byref(P), th, C.byref(r))
    return None if rc else r.value


def circular(P: Problem, R: float):
    W, uT = C.c_double(0.0), C.c_double(0.0)
    rc = _load().orc_circular(C.byref(P), R, C.byref(W), C.byref(uT))
    return None if rc else (W.value, uT.value)


def isco(P: Problem):
    r = C.c_double(0.0)
    rc = _load().orc_isco(C.byref(P), C.byref(r))
    return None if rc else r.value


def emissivity(P: Problem, R_in: float, R: float, th: float) -> float:
    return _load().orc_emissivity(C.byref(P), R_in, R, th)


def launch(P: Problem, X: float, Y: float):
    y0, u, pu = np.zeros(6), np.zeros(4), np.zeros(4)
    E, ell = C.c_double(0.0), C.c_double(0.0)
    _load().orc_launch(C.byref(P), X, Y, _dp(y0), C.byref(E), C.byref(ell), _dp(u), _dp(pu))
    return dict(y0=y0, E=E.value, ell=ell.value, u_o=u, p_up=pu)


def geometry(P: Problem):
    out = np.zeros(4)
    rc = _load().orc_geometry(C.byref(P), _dp(out))
    if rc:
        raise ValueError(f"oracle geometry setup failed (code {rc})")
    return dict(r_plus=out[0], R_in=out[1], R_cap=out[2], R_esc=out[3])


def dp5_solve(kind: int, y0, x0: float, x1: float, rtol: float, atol: float, w: float = 1.0,
              max_steps: int = 1_000_000):
    y = np.array(y0, dtype=np.float64)
    n = _load().orc_dp5_solve(kind, w, len(y), _dp(y), x0, x1, rtol, atol, max_steps)
    return y, n


def dp5_step_dense(kind: int, y0, h: float, sigmas, w: float = 1.0):
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    n = len(y0)
    y1, err = np.zeros(n), np.zeros(n)
    sig = np.ascontiguousarray(sigmas, dtype=np.float64)
    dense = np.zeros((len(sig), n))
    _load().orc_dp5_step_dense(kind, w, n, _dp(y0), h, _dp(y1), _dp(err), len(sig), _dp(sig),
                               _dp(dense))
    return y1, err, dense


RAY_FIELDS = [f for f, _ in Ray._fields_]


def trace_points(P: Problem, xy) -> np.ndarray:
    """Trace rays from explicit screen points; returns a structured array."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    n = xy.shape[0]
    rays = (Ray * max(n, 1))()
    rc = _load().orc_trace_points(C.byref(P), n, _dp(xy), rays)
    if rc:
        raise ValueError(f"oracle geometry setup failed (code {rc})")
    dt = np.dtype([(f, np.int32) if t is C.c_int32 else
                   ((f, np.float64, (3,)) if hasattr(t, "_length_") else (f, np.float64))
                   for f, t in Ray._fields_])
    arr = np.frombuffer(bytes(rays), dtype=dt, count=n).copy()
    return arr


def trace_image(P: Problem, keys_cap: int = 1 << 22) -> dict:
    """Trace a whole image (with refinement if ``P.levels > 0``)."""
    ny, nx = P.ny, P.nx
    npx = nx * ny
    out = dict(I=np.zeros(npx), I_n=np.zeros(3 * npx), ncross=np.zeros(npx, np.int32),
               status=np.zeros(npx, np.int32), level=np.zeros(npx, np.int32),
               R_em=np.zeros(3 * npx), phi_em=np.zeros(3 * npx), T_em=np.zeros(3 * npx),
               g=np.zeros(3 * npx), h_drift=np.zeros(npx), keys=np.zeros(keys_cap, np.uint64))
    img = _Image()
    for k in ("I", "I_n", "R_em", "phi_em", "T_em", "g", "h_drift"):
        setattr(img, k, _dp(out[k]))
    for k in ("ncross", "status", "level"):
        setattr(img, k, out[k].ctypes.data_as(C.POINTER(C.c_int32)))
    img.keys = out["keys"].ctypes.data_as(C.POINTER(C.c_uint64))
    img.keys_cap = keys_cap
    rc = _load().orc_trace_image(C.byref(P), C.byref(img))
    if rc:
        raise ValueError(f"oracle trace_image failed (code {rc})")
    if img.keys_count > keys_cap:
        raise ValueError("oracle key buffer too small")
    res = {k: v.reshape(ny, nx) for k, v in out.items()
           if k in ("I", "ncross", "status", "level", "h_drift")}
    for k in ("I_n", "R_em", "phi_em", "T_em", "g"):
        res[k] = out[k].reshape(3, ny, nx)
    res["keys"] = np.sort(out["keys"][: img.keys_count])
    return res


def trace_pixel(P: Problem, i: int, j: int, keys_cap: int = 1 << 16) -> dict:
    """One base pixel with its refinement subtree, computed on its own."""
    ray = Ray()
    val = np.zeros(4)
    lev = C.c_int32(0)
    keys = np.zeros(keys_cap, np.uint64)
    cnt = C.c_int64(0)
    rc = _load().orc_trace_pixel(C.byref(P), i, j, C.byref(ray), _dp(val), C.byref(lev),
                                 keys.ctypes.data_as(C.POINTER(C.c_uint64)), keys_cap,
                                 C.byref(cnt))
    if rc:
        raise ValueError(f"oracle trace_pixel failed (code {rc})")
    return dict(I=val[0], I_n=val[1:].copy(), level=lev.value, status=ray.status,
                ncross=ray.ncross, R_em=np.array(ray.R_em), g=np.array(ray.g),
                keys=np.sort(keys[: cnt.value]), ray=ray)


def trace_pixels(P: Problem, ij) -> dict:
    """Many base pixels with their refinement subtrees (parallel over pixels).
    Returns per-pixel values, deepest levels and the rays each one cost."""
    ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
    n = ij.shape[0]
    val = np.zeros((max(n, 1), 4))
    lev = np.zeros(max(n, 1), np.int32)
    nr = np.zeros(max(n, 1), np.int64)
    rc = _load().orc_trace_pixels(C.byref(P), n, ij.ctypes.data_as(C.POINTER(C.c_int32)),
                                  _dp(val), lev.ctypes.data_as(C.POINTER(C.c_int32)),
                                  nr.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc:
        raise ValueError(f"oracle trace_pixels failed (code {rc})")
    return dict(val=val[:n], level=lev[:n], rays=nr[:n])


def shadow_boundary(P: Problem, psi, b_lo: float, b_hi: float, tol: float) -> dict:
    """Shadow boundary along screen directions psi (Sec. 4.1, Eqs. 78-79) by
    bisection in b; returns the final brackets b_in (captured side), b_out
    (escaping side) and per-direction flags (1: b_lo not captured, 2: b_hi
    captured, 4: an undetermined ray was met)."""
    psi = np.ascontiguousarray(np.asarray(psi, dtype=np.float64).reshape(-1))
    n = psi.shape[0]
    b_in, b_out = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    flags = np.zeros(max(n, 1), np.int32)
    rc = _load().orc_shadow_boundary(C.byref(P), n, _dp(psi), b_lo, b_hi, tol, _dp(b_in),
                                     _dp(b_out), flags.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc:
        raise ValueError(f"oracle shadow_boundary failed (code {rc})")
    return dict(b_in=b_in[:n], b_out=b_out[:n], flags=flags[:n])


def _rays_to_numpy(rays, n):
    dt = np.dtype([(f, np.int32) if t is C.c_int32 else
                   ((f, np.float64, (3,)) if hasattr(t, "_length_") else (f, np.float64))
                   for f, t in Ray._fields_])
    return np.frombuffer(bytes(rays), dtype=dt, count=n).copy()


def trace_points_record(P: Problem, xy, hcap: int = 20000):
    """Trace points and record each ray's accepted step sizes; returns
    (records, hbuf [n, hcap], counts [n])."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    n = xy.shape[0]
    rays = (Ray * max(n, 1))()
    hbuf = np.zeros((max(n, 1), hcap))
    counts = np.zeros(max(n, 1), np.int32)
    rc = _load().orc_trace_points_record(C.byref(P), n, _dp(xy), rays, _dp(hbuf), hcap,
                                         counts.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc:
        raise ValueError(f"oracle geometry setup failed (code {rc})")
    if np.any(counts[:n] > hcap):
        raise ValueError("step record buffer too small")
    return _rays_to_numpy(rays, n), hbuf[:n], counts[:n]


def trace_points_frozen(P: Problem, xy, hbuf, counts):
    """Replay rays along recorded step sequences (no error control)."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    n = xy.shape[0]
    hbuf = np.ascontiguousarray(hbuf, dtype=np.float64)
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    rays = (Ray * max(n, 1))()
    rc = _load().orc_trace_points_frozen(C.byref(P), n, _dp(xy), _dp(hbuf), hbuf.shape[1],
                                         counts.ctypes.data_as(C.POINTER(C.c_int32)), rays)
    if rc:
        raise ValueError(f"oracle geometry setup failed (code {rc})")
    return _rays_to_numpy(rays, n)
