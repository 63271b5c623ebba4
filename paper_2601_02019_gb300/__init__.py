"""GB300 AeroSketch update path: a C-ABI CUDA library and its Python binding.

The library (lib/libaerosketch.so, built by build.py for sm_103a) implements
the AeroSketch update (persistent, fixed-threshold and P5 sites, with optional
probability amplification), the current-time and historical queries, merging,
the P5 coordinator, the sliding window, grouped updates of many sketches and
the serving runtime, and statistics; this package only
marshals arguments to it.  There is no CPU fallback: importing the binding
fails if the library has not been built.
"""
from .binding import (AS_BF16, AS_BF16X3, AS_BF16X6, AS_COORDINATOR, AS_FIXED_THETA, AS_FP32_PLAIN,  # noqa: F401
                      AS_PERSISTENT, AS_PROFILE, AS_SITE, AS_TRACE_DECISIONS, AsConfig, AsEvent, AsStats,
                      AeroSketchError, P5, Server, Sketch, SlidingWindow, footprint, lib, load_library,
                      update_grouped, update_many)
