"""The C ABI library loads without a GPU, exports every function that
include/bhrt.h declares, and its host-side parts (geometry, argument checks
that return before any device work) behave; no device compute is called."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bhrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(bh_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def B():
    from paper_2605_05635_gb300 import bhrt
    bhrt.lib()
    return bhrt


def test_library_exports_every_declared_function(B):
    lib = B.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_host_geometry_matches_oracle(B, oracle):
    for metric, kw, okw in [(0, {}, {}), (1, dict(lambda_E=0.1), dict(lam_E=0.1)),
                            (2, dict(eta=0.02, lambda_c=10.0), dict(eta=0.02, lam_c=10.0))]:
        for chi in (0.0, 0.5, 0.9, 0.98):
            rp, ce, ri = B.host_geometry(B.Spacetime(metric=metric, chi=chi, **kw))
            P = oracle.problem(metric=metric, chi=chi, **okw)
            assert rp == pytest.approx(oracle.horizon(P), rel=1e-13)
            assert ce == pytest.approx(oracle.extremal_spin(P)[0], rel=1e-8)
            assert ri == pytest.approx(oracle.isco(P), rel=2e-7)


def test_host_geometry_errors(B):
    with pytest.raises(B.BHRTError) as e:
        B.host_geometry(B.Spacetime(metric=0, chi=1.2))
    assert e.value.code == 2
    with pytest.raises(B.BHRTError) as e:
        B.host_geometry(B.Spacetime(metric=1, chi=0.7, lambda_E=0.3))
    assert e.value.code == 2


def test_argument_errors_return_before_device_work(B):
    """Validation happens on the host before anything is enqueued."""
    lib = B.lib()
    st = B.Spacetime(metric=0, chi=0.5)._c()
    cam = B.Camera()._c()
    em = B.Emission()._c()
    it = B.Integrator()._c()
    out = B._ImageOut()
    ws = C.c_void_p(0)
    # no workspace
    code = lib.bh_trace_image(C.byref(st), C.byref(cam), C.byref(em), C.byref(it), C.byref(out),
                              ws, 0, None)
    assert code in (1, 4)  # outputs missing (1) or workspace missing (4)
    bad = B.Spacetime(metric=0, chi=1.01)._c()
    code = lib.bh_trace_points(C.byref(bad), C.byref(cam), C.byref(em), C.byref(it), 0, None,
                               None, ws, 0, None)
    assert code == 2
    far = B.Camera(r_obs=5.0)._c()
    code = lib.bh_trace_points(C.byref(st), C.byref(far), C.byref(em), C.byref(it), 0, None,
                               None, ws, 0, None)
    assert code == 3
    for badint in (B.Integrator(precision=7)._c(), B.Integrator(promote_order=-1)._c(),
                   B.Integrator(promote_order=1001)._c(),
                   B.Integrator(promote_turning=-1e-3)._c(),
                   B.Integrator(promote_turning=1.5)._c(),
                   B.Integrator(promote_turning=float("nan"))._c()):
        code = lib.bh_trace_points(C.byref(st), C.byref(cam), C.byref(em), C.byref(badint), 0,
                                   None, None, ws, 0, None)
        assert code == 1
    assert lib.bh_plan_set_launch(None, 0, 1, 128, 0) == 1   # no plan
    incl = B.Camera(incl=math.pi)._c()
    code = lib.bh_trace_points(C.byref(st), C.byref(incl), C.byref(em), C.byref(it), 0, None,
                               None, ws, 0, None)
    assert code == 1
    # volumetric emission (Eq. 88): flag in {0, 1}, H0 > 0, h >= 0 and finite
    for kw in (dict(volumetric=2), dict(volumetric=1, H0=0.0), dict(volumetric=1, h=-1.0),
               dict(volumetric=1, h=float("inf"))):
        vem = B.Emission(**kw)._c()
        code = lib.bh_trace_points(C.byref(st), C.byref(cam), C.byref(vem), C.byref(it), 0,
                                   None, None, ws, 0, None)
        assert code == 1, kw
    vem = B.Emission(volumetric=1)._c()
    code = lib.bh_trace_points(C.byref(st), C.byref(cam), C.byref(vem), C.byref(it), 0, None,
                               None, ws, 0, None)
    assert code == 4   # arguments valid: only the workspace is missing
    # shadow boundary (Sec. 4.1): bracket, precision, spacetime, workspace
    def shadow(s, c, i, lo, hi, tol, lanes=0):
        return lib.bh_shadow_boundary(C.byref(s), C.byref(c), C.byref(i), 0, None, lo, hi, tol,
                                      lanes, None, None, None, None, ws, 0, None)
    for lo, hi, tol in ((3.0, 2.0, 1e-6), (-1.0, 2.0, 1e-6), (1.0, 2.0, 0.0),
                        (1.0, float("nan"), 1e-6), (1.0, 2.0, float("inf"))):
        assert shadow(st, cam, it, lo, hi, tol) == 1
    assert shadow(st, cam, B.Integrator(precision=1)._c(), 1.0, 9.0, 1e-6) == 1
    assert shadow(bad, cam, it, 1.0, 9.0, 1e-6) == 2
    assert shadow(st, far, it, 1.0, 9.0, 1e-6) == 3
    assert shadow(st, cam, it, 1.0, 9.0, 1e-6) == 4
    for lanes in (-1, 3, 64):
        assert shadow(st, cam, it, 1.0, 9.0, 1e-6, lanes) == 1
    # geometry scan (Sec. 2.3): sizes and missing arrays are rejected on the host
    assert lib.bh_geometry_scan(-1, None, 0, None, None, None, None, None, None, None,
                                None) == 1
    assert lib.bh_geometry_scan(4, None, 0, None, None, None, None, None, None, None,
                                None) == 1
    assert lib.bh_geometry_scan(0, None, -1, None, None, None, None, None, None, None,
                                None) == 1


def test_added_entry_points_host_checks(B):
    """Sizes and argument checks of the shadow, scan and amplitude-curve entry
    points, all answered on the host before any device work."""
    lib = B.lib()
    cam = B.Camera(nx=64, ny=48)._c()
    n = C.c_size_t(0)
    assert lib.bh_shadow_workspace_size(100, C.byref(n)) == 0 and n.value >= 256
    assert lib.bh_shadow_workspace_size(-1, C.byref(n)) == 1
    assert lib.bh_visibility_curves_workspace_size(C.byref(cam), 10, 16, C.byref(n)) == 0
    # room for the (u, v) set and the visibilities: 10 radii x 17 points + (0, 0)
    assert n.value >= 2 * (10 * 17 + 1) * 16
    for nq, nphi in ((-1, 16), (10, 0)):
        assert lib.bh_visibility_curves_workspace_size(C.byref(cam), nq, nphi, C.byref(n)) == 1
    fake = C.c_void_p(256)  # never dereferenced: every call below fails its checks first
    def curves(I, nq, nphi, mode, imax, ws, wsb):
        return lib.bh_visibility_curves(I, C.byref(cam), nq, fake if nq else None, nphi, mode,
                                        imax, fake if nq else None, fake if nq else None, ws,
                                        wsb, None)
    assert curves(None, 4, 8, 1, 1.0, fake, 1 << 30) == 1            # no image
    assert curves(fake, 4, 0, 1, 1.0, fake, 1 << 30) == 1            # no angles
    assert curves(fake, 4, 8, 3, 1.0, fake, 1 << 30) == 1            # unknown mode
    assert curves(fake, 4, 8, 1, 1.0, None, 0) == 4                  # no workspace


def test_workspace_sizes(B):
    cam = B.Camera(nx=64, ny=48, refine_levels=2)
    n64 = B.workspace_bytes([cam], B.Integrator(precision=0))
    nmx = B.workspace_bytes([cam], B.Integrator(precision=1))
    assert nmx > n64 > 64 * 48 * 32
    assert B.workspace_bytes([cam, cam], B.Integrator()) > n64
    with pytest.raises(B.BHRTError):
        B.workspace_bytes([cam, B.Camera(nx=32, ny=48, refine_levels=2)])


def test_status_strings(B):
    for code in range(9):
        assert B.status_string(code)


def test_visibility_call_validates_budget_and_mode(B):
    """bh_visibilities refuses a negative or non-finite time budget and an
    unknown mode before any device work (no workspace needed to see it)."""
    lib = B.lib()
    cam = B.Camera(nx=8, ny=8)._c()
    dummy = C.c_void_p(256)  # never dereferenced: validation fails first
    for budget, mode in ((-1.0, 1), (float("inf"), 1), (float("nan"), 1), (0.0, 3)):
        code = lib.bh_visibilities(dummy, C.byref(cam), dummy, 1, mode, 1.0, dummy, None, budget,
                                   None, 0, None)
        assert code == 1, (budget, mode)
