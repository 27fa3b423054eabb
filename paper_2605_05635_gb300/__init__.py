"""GB300-native ray tracer for rotating dark-matter-dressed black holes.

The compute path is the CUDA library ``libbhrt.so`` (C ABI in
``include/bhrt.h``); :mod:`.bhrt` is the Python binding.
"""
from .bhrt import (CNFW, DIAG_NAMES, EINASTO, FP64, KERR, MIXED, VIS_BF16,  # noqa: F401
                   VIS_FP16, VIS_FP64, BHRTError, Camera, Emission, Integrator, Plan, Spacetime,
                   diagnostics, from_flat, host_geometry, lib, trace_batch, trace_image,
                   trace_points, shadow_boundary, geometry_scan, spacetime_array,
                   visibilities, visibilities_workspace, visibility_curves, visibilities_fp64, trace_backward, BHRender,
                   GRAD_NAMES, LOSS_DIAG_NAMES)
