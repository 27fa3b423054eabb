"""Thin ctypes binding of ``libbhrt.so`` (C ABI declared in include/bhrt.h).

The binding only marshals arguments: it allocates outputs and the workspace
as torch CUDA tensors and passes raw device pointers and the current CUDA
stream to the library.  Every step of the computation runs in the library's
kernels; there is no CPU or PyTorch fallback, and a missing or unloadable
library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import threading
from typing import Dict, List, Optional, Sequence

import torch

from . import _build

KERR, EINASTO, CNFW = 0, 1, 2
FP64, MIXED = 0, 1

_lock = threading.Lock()
_lib = None


class BHRTError(RuntimeError):
    """A bh_status other than BH_OK."""

    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (bh_status {code})")


# --------------------------------------------------------------- ABI structs
class _Spacetime(C.Structure):
    _fields_ = [("metric", C.c_int32), ("reserved", C.c_int32), ("chi", C.c_double),
                ("lambda_E", C.c_double), ("eta", C.c_double), ("lambda_c", C.c_double)]


class _Camera(C.Structure):
    _fields_ = [("r_obs", C.c_double), ("incl", C.c_double), ("x_min", C.c_double),
                ("x_max", C.c_double), ("y_min", C.c_double), ("y_max", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32), ("refine_levels", C.c_int32),
                ("reserved", C.c_int32), ("refine_capacity", C.c_int64)]


class _Emission(C.Structure):
    _fields_ = [("r_in_mode", C.c_int32), ("volumetric", C.c_int32), ("j0", C.c_double),
                ("p", C.c_double), ("R_s", C.c_double), ("sigma_in", C.c_double),
                ("sigma_out", C.c_double), ("R_out", C.c_double), ("dR_in", C.c_double),
                ("H0", C.c_double), ("h", C.c_double)]


class _Integrator(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_steps", C.c_int32), ("rtol", C.c_double),
                ("atol", C.c_double), ("cap_factor", C.c_double), ("esc_factor", C.c_double),
                ("thetadot_min", C.c_double), ("dlambda_min", C.c_double),
                ("promote_dr", C.c_double), ("time_budget_s", C.c_double),
                ("promote_order", C.c_int32), ("reserved", C.c_int32),
                ("promote_turning", C.c_double)]


class _ImageOut(C.Structure):
    _fields_ = [("I", C.c_void_p), ("I_n", C.c_void_p), ("ncross", C.c_void_p),
                ("status", C.c_void_p), ("refine_level", C.c_void_p), ("R_em", C.c_void_p),
                ("phi_em", C.c_void_p), ("T_em", C.c_void_p), ("g", C.c_void_p),
                ("h_drift", C.c_void_p), ("refine_keys", C.c_void_p),
                ("refine_keys_cap", C.c_int64), ("refine_keys_count", C.c_void_p),
                ("steps", C.c_void_p), ("promoted", C.c_void_p)]


class RayRecord(C.Structure):
    _fields_ = [("status", C.c_int32), ("ncross", C.c_int32), ("n_accept", C.c_int32),
                ("n_reject", C.c_int32), ("I_tot", C.c_double), ("I_n", C.c_double * 3),
                ("R_em", C.c_double * 3), ("phi_em", C.c_double * 3),
                ("T_em", C.c_double * 3), ("g", C.c_double * 3), ("E", C.c_double),
                ("ell", C.c_double), ("h_drift", C.c_double), ("lambda_end", C.c_double)]


class RunStats(C.Structure):
    _fields_ = [("cells", C.c_int64 * 4), ("rays", C.c_int64 * 4),
                ("accepted_fp64", C.c_int64), ("rejected_fp64", C.c_int64),
                ("accepted_fp32", C.c_int64), ("rejected_fp32", C.c_int64),
                ("promoted_rays", C.c_int64), ("spill_full", C.c_int64),
                ("max_ray_steps", C.c_int64),
                ("trace_ms", C.c_double * 4), ("fp32_ms", C.c_double), ("fp64_ms", C.c_double),
                ("kernel_launches", C.c_int32), ("status", C.c_int32),
                ("trace_blocks", C.c_int32), ("trace_threads", C.c_int32),
                ("bulk_ms", (C.c_double * 4) * 3), ("tail_ms", (C.c_double * 4) * 3),
                ("lane_util_fp32", C.c_double), ("lane_util_fp64", C.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        for k in ("cells", "rays", "trace_ms"):
            d[k] = list(d[k])
        for k in ("bulk_ms", "tail_ms"):
            d[k] = [list(r) for r in d[k]]
        return d


class TuneReport(C.Structure):
    _fields_ = [("candidates", C.c_int32), ("blocks", C.c_int32 * 2),
                ("threads", C.c_int32 * 2), ("best_ms", C.c_double * 2),
                ("variant", C.c_int32 * 2)]


# ----------------------------------------------------------- user parameters
@dataclasses.dataclass
class Spacetime:
    metric: int = KERR
    chi: float = 0.5
    lambda_E: float = 0.1
    eta: float = 0.02
    lambda_c: float = 10.0

    def _c(self):
        return _Spacetime(self.metric, 0, self.chi, self.lambda_E, self.eta, self.lambda_c)


@dataclasses.dataclass
class Camera:
    r_obs: float = 1000.0
    incl: float = math.radians(17.0)
    x_min: float = -10.0
    x_max: float = 10.0
    y_min: float = -10.0
    y_max: float = 10.0
    nx: int = 64
    ny: int = 64
    refine_levels: int = 0
    refine_capacity: int = 0

    def _c(self):
        return _Camera(self.r_obs, self.incl, self.x_min, self.x_max, self.y_min, self.y_max,
                       self.nx, self.ny, self.refine_levels, 0, self.refine_capacity)


@dataclasses.dataclass
class Emission:
    r_in_mode: int = 0
    j0: float = 1.0
    p: float = 2.0
    R_s: float = 8.0
    sigma_in: float = 0.2
    sigma_out: float = 2.0
    R_out: float = 20.0
    dR_in: float = 0.5
    H0: float = 0.05
    h: float = 0.05
    volumetric: int = 0

    def _c(self):
        return _Emission(self.r_in_mode, self.volumetric, self.j0, self.p, self.R_s,
                         self.sigma_in, self.sigma_out, self.R_out, self.dR_in, self.H0, self.h)


@dataclasses.dataclass
class Integrator:
    precision: int = FP64
    max_steps: int = 1_000_000
    rtol: float = 1e-10
    atol: float = 1e-12
    cap_factor: float = 1.01
    esc_factor: float = 1.1
    thetadot_min: float = 1e-8
    dlambda_min: float = 1e-6
    promote_dr: float = 0.1
    time_budget_s: float = 0.0
    promote_order: int = 2
    promote_turning: float = 3e-3

    def _c(self):
        return _Integrator(self.precision, self.max_steps, self.rtol, self.atol,
                           self.cap_factor, self.esc_factor, self.thetadot_min,
                           self.dlambda_min, self.promote_dr, self.time_budget_s,
                           self.promote_order, 0, self.promote_turning)


def from_flat(d: dict):
    """Split a flat parameter dict (oracle naming) into the four structs."""
    st = Spacetime(metric=d.get("metric", KERR), chi=d.get("chi", 0.5),
                   lambda_E=d.get("lam_E", 0.1), eta=d.get("eta", 0.02),
                   lambda_c=d.get("lam_c", 10.0))
    cam = Camera(r_obs=d.get("r_obs", 1000.0), incl=d.get("incl", math.radians(17.0)),
                 x_min=d.get("x_min", -10.0), x_max=d.get("x_max", 10.0),
                 y_min=d.get("y_min", -10.0), y_max=d.get("y_max", 10.0),
                 nx=d.get("nx", 64), ny=d.get("ny", 64), refine_levels=d.get("levels", 0),
                 refine_capacity=d.get("refine_capacity", 0))
    em = Emission(r_in_mode=d.get("r_in_mode", 0), j0=d.get("j0", 1.0), p=d.get("p", 2.0),
                  R_s=d.get("R_s", 8.0), sigma_in=d.get("sigma_in", 0.2),
                  sigma_out=d.get("sigma_out", 2.0), R_out=d.get("R_out", 20.0),
                  dR_in=d.get("dR_in", 0.5), H0=d.get("H0", 0.05), h=d.get("h", 0.05),
                  volumetric=d.get("volumetric", 0))
    it = Integrator(precision=d.get("precision", FP64), max_steps=d.get("max_steps", 1_000_000),
                    rtol=d.get("rtol", 1e-10), atol=d.get("atol", 1e-12),
                    cap_factor=d.get("cap_factor", 1.01), esc_factor=d.get("esc_factor", 1.1),
                    thetadot_min=d.get("thetadot_min", 1e-8),
                    dlambda_min=d.get("dlambda_min", 1e-6),
                    promote_dr=d.get("promote_dr", 0.1),
                    time_budget_s=d.get("time_budget_s", 0.0),
                    promote_order=d.get("promote_order", 2),
                    promote_turning=d.get("promote_turning", 3e-3))
    return st, cam, em, it


# ------------------------------------------------------------------ library
def lib():
    """Load (building first if needed) the CUDA library; raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not _build.up_to_date():
            _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.bh_status_string.argtypes = [C.c_int]
        L.bh_status_string.restype = C.c_char_p
        L.bh_host_geometry.argtypes = [P(_Spacetime), P(C.c_double), P(C.c_double), P(C.c_double)]
        L.bh_workspace_size.argtypes = [C.c_int32, P(_Camera), P(_Integrator), P(C.c_size_t)]
        L.bh_trace_image.argtypes = [P(_Spacetime), P(_Camera), P(_Emission), P(_Integrator),
                                     P(_ImageOut), C.c_void_p, C.c_size_t, C.c_void_p]
        L.bh_trace_batch.argtypes = [C.c_int32, P(_Spacetime), P(_Camera), P(_Emission),
                                     P(_Integrator), P(_ImageOut), C.c_void_p, C.c_size_t,
                                     C.c_void_p]
        L.bh_points_workspace_size.argtypes = [C.c_int64, P(C.c_size_t)]
        L.bh_trace_points.argtypes = [P(_Spacetime), P(_Camera), P(_Emission), P(_Integrator),
                                      C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                      C.c_void_p]
        L.bh_workspace_status.argtypes = [C.c_void_p, C.c_void_p]
        L.bh_geometry_scan.argtypes = [C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
        L.bh_shadow_workspace_size.argtypes = [C.c_int64, P(C.c_size_t)]
        L.bh_shadow_boundary.argtypes = [P(_Spacetime), P(_Camera), P(_Integrator), C.c_int64,
                                         C.c_void_p, C.c_double, C.c_double, C.c_double,
                                         C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.bh_plan_create.argtypes = [C.c_int32, P(_Spacetime), P(_Camera), P(_Emission),
                                     P(_Integrator), P(_ImageOut), C.c_void_p, C.c_size_t,
                                     C.c_void_p, P(C.c_void_p)]
        L.bh_plan_launch.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.bh_plan_set_timing.argtypes = [C.c_void_p, C.c_int32]
        L.bh_plan_set_launch.argtypes = [C.c_void_p] + [C.c_int32] * 4
        L.bh_plan_stats.argtypes = [C.c_void_p, C.c_void_p, P(RunStats)]
        L.bh_plan_destroy.argtypes = [C.c_void_p]
        L.bh_plan_autotune.argtypes = [C.c_void_p, C.c_void_p, P(TuneReport)]
        L.bh_plan_autotune.restype = C.c_int
        L.bh_diagnostics_workspace_size.argtypes = [P(_Camera), P(C.c_size_t)]
        L.bh_diagnostics.argtypes = [C.c_void_p, P(_Camera), C.c_double, C.c_void_p, C.c_void_p,
                                     C.c_size_t, C.c_void_p]
        L.bh_visibilities_fp64.argtypes = [C.c_void_p, P(_Camera), C.c_void_p, C.c_int64,
                                           C.c_void_p, C.c_void_p]
        L.bh_visibilities_workspace_size.argtypes = [P(_Camera), P(C.c_size_t)]
        L.bh_visibilities.argtypes = [C.c_void_p, P(_Camera), C.c_void_p, C.c_int64, C.c_int32,
                                      C.c_double, C.c_void_p, C.c_void_p, C.c_double,
                                      C.c_void_p, C.c_size_t, C.c_void_p]
        L.bh_visibility_curves_workspace_size.argtypes = [P(_Camera), C.c_int32, C.c_int32,
                                                          P(C.c_size_t)]
        L.bh_visibility_curves.argtypes = [C.c_void_p, P(_Camera), C.c_int32, C.c_void_p,
                                           C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.bh_backward_workspace_size.argtypes = [P(_Camera), P(C.c_size_t)]
        L.bh_trace_backward.argtypes = [P(_Spacetime), P(_Camera), P(_Emission), P(_Integrator),
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                        C.c_void_p]
        L.bh_backward_workspace_size.restype = C.c_int
        L.bh_trace_backward.restype = C.c_int
        for fn in ("bh_diagnostics_workspace_size", "bh_diagnostics", "bh_visibilities_fp64",
                   "bh_visibilities_workspace_size", "bh_visibilities",
                   "bh_visibility_curves_workspace_size", "bh_visibility_curves"):
            getattr(L, fn).restype = C.c_int
        for fn in ("bh_host_geometry", "bh_workspace_size", "bh_trace_image", "bh_trace_batch",
                   "bh_points_workspace_size", "bh_trace_points", "bh_workspace_status",
                   "bh_shadow_workspace_size", "bh_shadow_boundary", "bh_geometry_scan",
                   "bh_plan_create", "bh_plan_launch", "bh_plan_set_timing", "bh_plan_set_launch",
                   "bh_plan_stats",
                   "bh_plan_destroy"):
            getattr(L, fn).restype = C.c_int
        _lib = L
        return L


def status_string(code: int) -> str:
    return lib().bh_status_string(code).decode()


def _check(code: int, where: str):
    if code != 0:
        raise BHRTError(code, where)


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _need_cuda(device):
    if not torch.cuda.is_available():
        raise RuntimeError("bhrt needs a CUDA device; there is no CPU fallback")
    return torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())


def host_geometry(st: Spacetime):
    """(r_plus, chi_e, r_isco) from the library's host geometry."""
    rp, ce, ri = C.c_double(0), C.c_double(0), C.c_double(0)
    code = lib().bh_host_geometry(C.byref(st._c()), C.byref(rp), C.byref(ce), C.byref(ri))
    _check(code, "bh_host_geometry")
    return rp.value, ce.value, ri.value


def _aligned_workspace(nbytes: int, device) -> torch.Tensor:
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + nbytes]


def workspace_bytes(cams: Sequence[Camera], integ: Optional[Integrator] = None) -> int:
    arr = (_Camera * len(cams))(*[c._c() for c in cams])
    n = C.c_size_t(0)
    it = C.byref(integ._c()) if integ is not None else None
    _check(lib().bh_workspace_size(len(cams), arr, it, C.byref(n)), "bh_workspace_size")
    return n.value


def alloc_outputs(cam: Camera, device, keys_cap: int = 0) -> Dict[str, torch.Tensor]:
    ny, nx = cam.ny, cam.nx
    f = dict(dtype=torch.float32, device=device)
    u8 = dict(dtype=torch.uint8, device=device)
    out = dict(I=torch.empty(ny, nx, **f), I_n=torch.empty(3, ny, nx, **f),
               ncross=torch.empty(ny, nx, **u8), status=torch.empty(ny, nx, **u8),
               refine_level=torch.empty(ny, nx, **u8), R_em=torch.empty(3, ny, nx, **f),
               phi_em=torch.empty(3, ny, nx, **f), T_em=torch.empty(3, ny, nx, **f),
               g=torch.empty(3, ny, nx, **f), h_drift=torch.empty(ny, nx, **f),
               steps=torch.empty(2, ny, nx, dtype=torch.int32, device=device),
               promoted=torch.empty(ny, nx, **u8))
    if keys_cap:
        out["refine_keys"] = torch.empty(keys_cap, dtype=torch.int64, device=device)
        out["refine_keys_count"] = torch.zeros(1, dtype=torch.int64, device=device)
    return out


def _image_out(o: Dict[str, torch.Tensor]) -> _ImageOut:
    def ptr(k):
        t = o.get(k)
        return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)

    keys = o.get("refine_keys")
    return _ImageOut(ptr("I"), ptr("I_n"), ptr("ncross"), ptr("status"), ptr("refine_level"),
                     ptr("R_em"), ptr("phi_em"), ptr("T_em"), ptr("g"), ptr("h_drift"),
                     ptr("refine_keys"), keys.numel() if keys is not None else 0,
                     ptr("refine_keys_count"), ptr("steps"), ptr("promoted"))


def trace_batch(items: Sequence[tuple], device=None, stream=None, keys_cap: int = 0,
                outputs: Optional[List[Dict[str, torch.Tensor]]] = None,
                workspace: Optional[torch.Tensor] = None, check: bool = True):
    """Trace several images in one call.  ``items`` is a sequence of
    (Spacetime, Camera, Emission, Integrator) tuples.  Returns the list of
    output dicts (torch tensors on the device)."""
    device = _need_cuda(device)
    n = len(items)
    sts = (_Spacetime * n)(*[it[0]._c() for it in items])
    cams = (_Camera * n)(*[it[1]._c() for it in items])
    ems = (_Emission * n)(*[it[2]._c() for it in items])
    ints = (_Integrator * n)(*[it[3]._c() for it in items])
    if outputs is None:
        outputs = [alloc_outputs(it[1], device, keys_cap) for it in items]
    outs = (_ImageOut * n)(*[_image_out(o) for o in outputs])
    nbytes = workspace_bytes([it[1] for it in items], items[0][3])
    if workspace is None or workspace.numel() < nbytes:
        workspace = _aligned_workspace(nbytes, device)
    sp = _stream_ptr(stream)
    code = lib().bh_trace_batch(n, sts, cams, ems, ints, outs, C.c_void_p(workspace.data_ptr()),
                                workspace.numel(), sp)
    _check(code, "bh_trace_batch")
    if check:
        _check(lib().bh_workspace_status(C.c_void_p(workspace.data_ptr()), sp), "device status")
        for o in outputs:
            if "refine_keys_count" in o:
                cnt = int(o["refine_keys_count"].item())
                o["refine_keys"] = o["refine_keys"][:min(cnt, o["refine_keys"].numel())]
    return outputs


def trace_image(st: Spacetime, cam: Camera, em: Emission, integ: Integrator, device=None,
                stream=None, keys_cap: int = 0, check: bool = True):
    return trace_batch([(st, cam, em, integ)], device=device, stream=stream, keys_cap=keys_cap,
                       check=check)[0]


def trace_points(st: Spacetime, cam: Camera, em: Emission, integ: Integrator, xy, device=None,
                 stream=None):
    """Trace rays from explicit screen points ``xy`` (N x 2); returns a numpy
    structured array of ray records."""
    import numpy as np

    device = _need_cuda(device)
    xy_t = torch.as_tensor(xy, dtype=torch.float64).reshape(-1, 2).contiguous().to(device)
    n = xy_t.shape[0]
    rec = torch.empty(max(n, 1) * C.sizeof(RayRecord), dtype=torch.uint8, device=device)
    nb = C.c_size_t(0)
    _check(lib().bh_points_workspace_size(n, C.byref(nb)), "bh_points_workspace_size")
    ws = _aligned_workspace(nb.value, device)
    sp = _stream_ptr(stream)
    code = lib().bh_trace_points(C.byref(st._c()), C.byref(cam._c()), C.byref(em._c()),
                                 C.byref(integ._c()), n, C.c_void_p(xy_t.data_ptr()),
                                 C.c_void_p(rec.data_ptr()), C.c_void_p(ws.data_ptr()),
                                 ws.numel(), sp)
    _check(code, "bh_trace_points")
    _check(lib().bh_workspace_status(C.c_void_p(ws.data_ptr()), sp), "device status")
    raw = rec[: n * C.sizeof(RayRecord)].cpu().numpy().tobytes()
    dt = np.dtype([(f, np.int32) if t is C.c_int32 else
                   ((f, np.float64, (3,)) if hasattr(t, "_length_") else (f, np.float64))
                   for f, t in RayRecord._fields_])
    return np.frombuffer(raw, dtype=dt, count=n).copy()


def spacetime_array(spacetimes: Sequence[Spacetime], device=None) -> torch.Tensor:
    """The bh_spacetime structs of ``spacetimes`` as one device byte tensor
    (the layout bh_geometry_scan reads)."""
    import numpy as np

    device = _need_cuda(device)
    arr = (_Spacetime * max(len(spacetimes), 1))(*[s._c() for s in spacetimes])
    raw = np.frombuffer(bytes(arr), dtype=np.uint8)[: len(spacetimes) * C.sizeof(_Spacetime)]
    return torch.from_numpy(raw.copy()).to(device)


def geometry_scan(spacetimes, theta=(), device=None, stream=None, stats=None):
    """Horizon, extremal spin and stationary-limit radii of many spacetimes
    (Sec. 2.3, Eqs. 33-41).  ``spacetimes`` is a sequence of Spacetime or a
    device tensor from spacetime_array.  Returns device tensors r_plus,
    chi_e, R_e [n], R_s [n, len(theta)] and flags [n] (0 black hole, 1 no
    horizon, 2 invalid parameters).  ``stats``, an optional int64 device
    tensor of 2, receives the lapse evaluations of the two searches."""
    device = _need_cuda(device)
    if isinstance(spacetimes, torch.Tensor):
        st_d = spacetimes
        if (st_d.dtype != torch.uint8 or not st_d.is_cuda or not st_d.is_contiguous()
                or st_d.numel() % C.sizeof(_Spacetime)):
            raise ValueError("spacetimes must be a contiguous CUDA uint8 tensor of whole "
                             "bh_spacetime structs (see spacetime_array)")
        n = st_d.numel() // C.sizeof(_Spacetime)
    else:
        n = len(spacetimes)
        st_d = spacetime_array(spacetimes, device)
    if stats is not None and (stats.dtype != torch.int64 or not stats.is_cuda
                              or stats.numel() < 2):
        raise ValueError("stats must be an int64 CUDA tensor of at least 2 elements")
    th = torch.as_tensor(theta, dtype=torch.float64).reshape(-1).contiguous().to(device)
    k = th.shape[0]
    out = {name: torch.empty(max(n, 1), dtype=torch.float64, device=device)
           for name in ("r_plus", "chi_e", "R_e")}
    R_s = torch.empty((max(n, 1), max(k, 1)), dtype=torch.float64, device=device)
    flags = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    code = lib().bh_geometry_scan(n, C.c_void_p(st_d.data_ptr() if n else 0), k,
                                  C.c_void_p(th.data_ptr() if k else 0),
                                  C.c_void_p(out["r_plus"].data_ptr()),
                                  C.c_void_p(out["chi_e"].data_ptr()),
                                  C.c_void_p(out["R_e"].data_ptr()),
                                  C.c_void_p(R_s.data_ptr() if k else 0),
                                  C.c_void_p(flags.data_ptr()),
                                  C.c_void_p(stats.data_ptr() if stats is not None else 0),
                                  _stream_ptr(stream))
    _check(code, "bh_geometry_scan")
    res = {name: v[:n] for name, v in out.items()}
    res["R_s"] = R_s[:n, :k]
    res["flags"] = flags[:n]
    return res


def shadow_boundary(st: Spacetime, cam: Camera, integ: Integrator, psi, b_lo: float,
                    b_hi: float, b_tol: float, device=None, stream=None, stats=None,
                    lanes: int = 0):
    """Shadow boundary along screen directions ``psi`` (Sec. 4.1, Eqs. 78-79):
    returns device tensors (b_in, b_out, flags) per direction, the final
    bracket of the capture / escape transition in the impact parameter and
    its flags (1 b_lo not captured, 2 b_hi captured, 4 an undetermined ray,
    8 time budget).  ``stats``, an optional int64 device tensor of 3,
    receives the rays traced and their accepted and rejected steps;
    ``lanes`` (power of two up to 32, 0 = the library's choice) is the rays
    traced per direction and round."""
    device = _need_cuda(device)
    if stats is not None and (stats.dtype != torch.int64 or not stats.is_cuda
                              or stats.numel() < 3):
        raise ValueError("stats must be an int64 CUDA tensor of at least 3 elements")
    psi_t = torch.as_tensor(psi, dtype=torch.float64).reshape(-1).contiguous().to(device)
    n = psi_t.shape[0]
    b_in = torch.empty(max(n, 1), dtype=torch.float64, device=device)
    b_out = torch.empty_like(b_in)
    flags = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    nb = C.c_size_t(0)
    _check(lib().bh_shadow_workspace_size(n, C.byref(nb)), "bh_shadow_workspace_size")
    ws = _aligned_workspace(nb.value, device)
    sp = _stream_ptr(stream)
    code = lib().bh_shadow_boundary(C.byref(st._c()), C.byref(cam._c()), C.byref(integ._c()), n,
                                    C.c_void_p(psi_t.data_ptr()), b_lo, b_hi, b_tol, lanes,
                                    C.c_void_p(b_in.data_ptr()), C.c_void_p(b_out.data_ptr()),
                                    C.c_void_p(flags.data_ptr()),
                                    C.c_void_p(stats.data_ptr() if stats is not None else 0),
                                    C.c_void_p(ws.data_ptr()), ws.numel(), sp)
    _check(code, "bh_shadow_boundary")
    _check(lib().bh_workspace_status(C.c_void_p(ws.data_ptr()), sp), "device status")
    return b_in[:n], b_out[:n], flags[:n]


class Plan:
    """A batch whose constants are uploaded once and that is launched many
    times (optionally as a CUDA graph replay).  Outputs and workspace are
    torch tensors owned by the plan object."""

    def __init__(self, items: Sequence[tuple], device=None, stream=None, keys_cap: int = 0):
        self.device = _need_cuda(device)
        self.items = list(items)
        n = len(self.items)
        self.outputs = [alloc_outputs(it[1], self.device, keys_cap) for it in self.items]
        sts = (_Spacetime * n)(*[it[0]._c() for it in self.items])
        cams = (_Camera * n)(*[it[1]._c() for it in self.items])
        ems = (_Emission * n)(*[it[2]._c() for it in self.items])
        ints = (_Integrator * n)(*[it[3]._c() for it in self.items])
        outs = (_ImageOut * n)(*[_image_out(o) for o in self.outputs])
        nbytes = workspace_bytes([it[1] for it in self.items], self.items[0][3])
        self.workspace = _aligned_workspace(nbytes, self.device)
        self._h = C.c_void_p(0)
        code = lib().bh_plan_create(n, sts, cams, ems, ints, outs,
                                    C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(),
                                    _stream_ptr(stream), C.byref(self._h))
        _check(code, "bh_plan_create")

    def launch(self, use_graph: bool = False, stream=None):
        _check(lib().bh_plan_launch(self._h, int(use_graph), _stream_ptr(stream)),
               "bh_plan_launch")

    def autotune(self, stream=None) -> dict:
        rep = TuneReport()
        _check(lib().bh_plan_autotune(self._h, _stream_ptr(stream), C.byref(rep)),
               "bh_plan_autotune")
        return dict(candidates=rep.candidates, blocks=list(rep.blocks),
                    threads=list(rep.threads), best_ms=list(rep.best_ms),
                    variant=list(rep.variant))

    def set_timing(self, enable: bool):
        _check(lib().bh_plan_set_timing(self._h, int(enable)), "bh_plan_set_timing")

    def set_launch(self, which: int, blocks: int, threads: int = 128, variant: int = 0):
        """Fix the persistent grid of the main (0) or FP64-pass (1) trace kernel."""
        _check(lib().bh_plan_set_launch(self._h, which, blocks, threads, variant),
               "bh_plan_set_launch")

    def stats(self, stream=None) -> dict:
        st = RunStats()
        _check(lib().bh_plan_stats(self._h, _stream_ptr(stream), C.byref(st)), "bh_plan_stats")
        return st.as_dict()

    def check(self, stream=None):
        _check(lib().bh_workspace_status(C.c_void_p(self.workspace.data_ptr()),
                                         _stream_ptr(stream)), "device status")

    def close(self):
        if self._h:
            lib().bh_plan_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


DIAG_NAMES = ["F", "X_c", "Y_c", "C", "rho_bar", "d_img", "w_img", "A_LR", "P", "rho_peak",
              "d_peak", "theta_peak"]


def diagnostics(I: torch.Tensor, cam: Camera, theta_g: float = 1.0, stream=None,
                out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None):
    """Sec. 6.2-6.3 diagnostics of a device intensity plane; returns a device
    tensor of 12 doubles (see DIAG_NAMES)."""
    if I.dtype != torch.float32 or not I.is_cuda or not I.is_contiguous():
        raise ValueError("I must be a contiguous float32 CUDA tensor")
    nb = C.c_size_t(0)
    _check(lib().bh_diagnostics_workspace_size(C.byref(cam._c()), C.byref(nb)),
           "bh_diagnostics_workspace_size")
    if workspace is None or workspace.numel() < nb.value:
        workspace = _aligned_workspace(nb.value, I.device)
    if out is None:
        out = torch.empty(12, dtype=torch.float64, device=I.device)
    _check(lib().bh_diagnostics(C.c_void_p(I.data_ptr()), C.byref(cam._c()), theta_g,
                                C.c_void_p(out.data_ptr()), C.c_void_p(workspace.data_ptr()),
                                workspace.numel(), _stream_ptr(stream)), "bh_diagnostics")
    return out


def visibilities_fp64(I: torch.Tensor, cam: Camera, uv: torch.Tensor, stream=None,
                      out: Optional[torch.Tensor] = None):
    """Eq. (108) by the FP64 direct sum; returns a complex128 device tensor."""
    uv = uv.to(device=I.device, dtype=torch.float64).contiguous()
    K = uv.shape[0]
    if out is None:
        out = torch.empty(K, 2, dtype=torch.float64, device=I.device)
    _check(lib().bh_visibilities_fp64(C.c_void_p(I.data_ptr()), C.byref(cam._c()),
                                      C.c_void_p(uv.data_ptr()), K, C.c_void_p(out.data_ptr()),
                                      _stream_ptr(stream)), "bh_visibilities_fp64")
    return torch.view_as_complex(out)


VIS_FP64, VIS_BF16, VIS_FP16 = 0, 1, 2


def visibilities_workspace(cam: Camera, device=None) -> torch.Tensor:
    """A device workspace for bh_visibilities on this screen."""
    nb = C.c_size_t(0)
    _check(lib().bh_visibilities_workspace_size(C.byref(cam._c()), C.byref(nb)),
           "bh_visibilities_workspace_size")
    return _aligned_workspace(nb.value, _need_cuda(device))


def visibilities(I: torch.Tensor, cam: Camera, uv: torch.Tensor, mode: int = VIS_BF16,
                 image_max: Optional[float] = None, stream=None, out=None, workspace=None,
                 check: bool = True, normalised: bool = False, time_budget_s: float = 0.0):
    """Eq. (108) on the tensor cores (split BF16 / FP16) or by the FP64 direct
    sum (mode 0); returns a complex128 device tensor, or with ``normalised``
    the pair (V, |V|/|V(0,0)|) of Eqs. (108)-(109)."""
    uv = uv.to(device=I.device, dtype=torch.float64).contiguous()
    K = uv.shape[0]
    if image_max is None:
        image_max = float(I.abs().max().item()) or 1.0
    if out is None:
        out = torch.empty(K, 2, dtype=torch.float64, device=I.device)
    nb = C.c_size_t(0)
    _check(lib().bh_visibilities_workspace_size(C.byref(cam._c()), C.byref(nb)),
           "bh_visibilities_workspace_size")
    if workspace is None or workspace.numel() < nb.value:
        workspace = _aligned_workspace(nb.value, I.device)
    vn = torch.empty(K, dtype=torch.float64, device=I.device) if normalised else None
    sp = _stream_ptr(stream)
    _check(lib().bh_visibilities(C.c_void_p(I.data_ptr()), C.byref(cam._c()),
                                 C.c_void_p(uv.data_ptr()), K, mode, image_max,
                                 C.c_void_p(out.data_ptr()),
                                 C.c_void_p(vn.data_ptr() if vn is not None else 0),
                                 float(time_budget_s), C.c_void_p(workspace.data_ptr()),
                                 workspace.numel(), sp),
           "bh_visibilities")
    if check and mode != VIS_FP64:
        _check(lib().bh_workspace_status(C.c_void_p(workspace.data_ptr()), sp), "device status")
    V = torch.view_as_complex(out)
    return (V, vn) if normalised else V


def visibility_curves(I: torch.Tensor, cam: Camera, q, n_phi: int = 256, mode: int = VIS_BF16,
                      image_max: Optional[float] = None, stream=None, check: bool = True):
    """Sec. 6.4's azimuthally averaged normalised amplitude V(q) and horizontal
    cut |V(q, 0)| / |V(0, 0)| at the radii ``q`` (cycles per M); returns two
    float64 device tensors."""
    if I.dtype != torch.float32 or not I.is_cuda or not I.is_contiguous():
        raise ValueError("I must be a contiguous float32 CUDA tensor")
    q_t = torch.as_tensor(q, dtype=torch.float64).reshape(-1).contiguous().to(I.device)
    n_q = q_t.shape[0]
    if image_max is None:
        image_max = float(I.abs().max().item()) or 1.0
    avg = torch.empty(max(n_q, 1), dtype=torch.float64, device=I.device)
    cut = torch.empty_like(avg)
    nb = C.c_size_t(0)
    _check(lib().bh_visibility_curves_workspace_size(C.byref(cam._c()), n_q, n_phi,
                                                     C.byref(nb)),
           "bh_visibility_curves_workspace_size")
    ws = _aligned_workspace(nb.value, I.device)
    sp = _stream_ptr(stream)
    _check(lib().bh_visibility_curves(C.c_void_p(I.data_ptr()), C.byref(cam._c()), n_q,
                                      C.c_void_p(q_t.data_ptr()), n_phi, mode, image_max,
                                      C.c_void_p(avg.data_ptr()), C.c_void_p(cut.data_ptr()),
                                      C.c_void_p(ws.data_ptr()), ws.numel(), sp),
           "bh_visibility_curves")
    if check:
        _check(lib().bh_workspace_status(C.c_void_p(ws.data_ptr()), sp), "device status")
    return avg[:n_q], cut[:n_q]


GRAD_NAMES = ["chi", "incl", "halo1", "halo2", "j0", "p", "R_s", "sigma_in", "sigma_out", "R_out"]
LOSS_DIAG_NAMES = ["C", "A_LR", "rho_peak"] + [f"vis{k}" for k in range(8)]


def trace_backward(st: Spacetime, cam: Camera, em: Emission, integ: Integrator,
                   dL_dI: Optional[torch.Tensor] = None, dL_ddiag=None, uv8=None, device=None,
                   stream=None):
    """Gradient of L = sum dL_dI * I + sum dL_ddiag * D by the discrete adjoint.
    Returns (grad [10] numpy, diag [11] numpy, forward image tensor)."""
    import numpy as np

    device = _need_cuda(device)
    nb = C.c_size_t(0)
    _check(lib().bh_backward_workspace_size(C.byref(cam._c()), C.byref(nb)),
           "bh_backward_workspace_size")
    ws = _aligned_workspace(nb.value, device)
    grad = np.zeros(10)
    diag = np.zeros(11)
    img = torch.empty(cam.ny, cam.nx, dtype=torch.float32, device=device)
    dd = None if dL_ddiag is None else np.ascontiguousarray(dL_ddiag, dtype=np.float64)
    uv = None if uv8 is None else np.ascontiguousarray(np.asarray(uv8).reshape(8, 2),
                                                        dtype=np.float64)
    dli = None
    if dL_dI is not None:
        dli = dL_dI.to(device=device, dtype=torch.float32).contiguous()
    ptr = lambda a: C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)
    code = lib().bh_trace_backward(
        C.byref(st._c()), C.byref(cam._c()), C.byref(em._c()), C.byref(integ._c()),
        C.c_void_p(dli.data_ptr()) if dli is not None else C.c_void_p(0), ptr(dd), ptr(uv),
        ptr(grad), ptr(diag), C.c_void_p(img.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
        _stream_ptr(stream))
    _check(code, "bh_trace_backward")
    return grad, diag, img


class BHRender(torch.autograd.Function):
    """Differentiable render: forward = FP64 image of the given parameters,
    backward = the library's discrete adjoint.  params is a float64 tensor
    (chi, incl, halo1, halo2, j0, p, R_s, sigma_in, sigma_out, R_out); the
    remaining settings come from the template structs."""

    @staticmethod
    def forward(ctx, params, st: Spacetime, cam: Camera, em: Emission, integ: Integrator):
        st2, em2 = _apply_params(params, st, em)
        cam2 = dataclasses.replace(cam, incl=float(params[1]))
        out = trace_image(st2, cam2, em2, dataclasses.replace(integ, precision=FP64))
        ctx.save_for_backward(params)
        ctx.cfg = (st, cam, em, integ)
        return out["I"]

    @staticmethod
    def backward(ctx, gI):
        (params,) = ctx.saved_tensors
        st, cam, em, integ = ctx.cfg
        st2, em2 = _apply_params(params, st, em)
        cam2 = dataclasses.replace(cam, incl=float(params[1]))
        grad, _, _ = trace_backward(st2, cam2, em2, integ, dL_dI=gI)
        return torch.as_tensor(grad, dtype=params.dtype, device=params.device), None, None, \
            None, None


def _apply_params(params, st: Spacetime, em: Emission):
    p = [float(x) for x in params]
    kw = dict(chi=p[0])
    if st.metric == EINASTO:
        kw["lambda_E"] = p[2]
    elif st.metric == CNFW:
        kw["eta"] = p[2]
        kw["lambda_c"] = p[3]
    st2 = dataclasses.replace(st, **kw)
    em2 = dataclasses.replace(em, j0=p[4], p=p[5], R_s=p[6], sigma_in=p[7], sigma_out=p[8],
                              R_out=p[9])
    return st2, em2
