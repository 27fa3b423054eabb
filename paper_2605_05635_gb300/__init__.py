"""GB300-native ray tracer for rotating dark-matter-dressed black holes.

The compute path is the CUDA library ``libbhrt.so`` (C ABI in
``include/bhrt.h``); :mod:`.bhrt` is the Python binding.
"""
from .bhrt import (CNFW, EINASTO, FP64, KERR, MIXED, BHRTError, Camera, Emission,  # noqa: F401
                   Integrator, Plan, Spacetime, from_flat, host_geometry, lib, trace_batch,
                   trace_image, trace_points)
