"""The allocation-free diagnostics entry point (bh_diagnostics_noalloc).

It exists for callers that cannot allocate device memory when they need the
result (a framework that owns all device memory through its own pool, a
plugin handed only its input and output buffers, a timed loop that must not
call cudaMalloc): its scratch is a fixed device array inside the library.
The test calls it through the C ABI twice in a row, on two different images,
and checks each result against bh_diagnostics with a caller workspace, within
the tolerance of the other diagnostics tests.  This file is collected last so
that a failure here stops a run only after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ring(n, ext, r0, w, x0, y0):
    d = 2 * ext / n
    c = -ext + (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(c, c)
    I = np.exp(-(np.hypot(X - x0, Y - y0) - r0) ** 2 / (2 * w * w)) * (1 + 0.5 * np.tanh(X - x0))
    return I.astype(np.float32)


def test_noalloc_diagnostics_match_workspace_version():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_05635_gb300 import bhrt
    lib = bhrt.lib()
    lib.bh_diagnostics_noalloc.argtypes = [C.c_void_p, C.POINTER(bhrt._Camera), C.c_double,
                                           C.c_void_p, C.c_void_p]
    lib.bh_diagnostics_noalloc.restype = C.c_int
    stream = torch.cuda.current_stream()
    cases = [(256, 12.0, _ring(256, 12.0, 5.0, 0.4, 0.7, -0.3)),
             (200, 10.0, _ring(200, 10.0, 3.2, 0.9, -1.1, 0.8))]
    for n, ext, img in cases:
        cam = bhrt.Camera(nx=n, ny=n, x_min=-ext, x_max=ext, y_min=-ext, y_max=ext)
        I = torch.from_numpy(img).cuda()
        out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
        code = lib.bh_diagnostics_noalloc(C.c_void_p(I.data_ptr()), C.byref(cam._c()), 3.8,
                                          C.c_void_p(out.data_ptr()),
                                          C.c_void_p(stream.cuda_stream))
        assert code == 0, bhrt.status_string(code)
        ref = bhrt.diagnostics(I, cam, theta_g=3.8)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-12)
    # beyond the fixed scratch (a 65536^2 screen needs ~1.5 MB of histogram):
    # rejected on the host before anything is enqueued, so the small device
    # buffers passed here are never read
    big = bhrt.Camera(nx=65536, ny=65536, x_min=-12, x_max=12, y_min=-12, y_max=12)
    code = lib.bh_diagnostics_noalloc(C.c_void_p(I.data_ptr()), C.byref(big._c()), 1.0,
                                      C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert code == 4
