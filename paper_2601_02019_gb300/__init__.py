"""GB300 AeroSketch update path: a C-ABI CUDA library and its Python binding.

The library (lib/libaerosketch.so, built by build.py for sm_103a) implements
the persistent AeroSketch update, query and statistics; this package only
marshals arguments to it.  There is no CPU fallback: importing the binding
fails if the library has not been built.
"""
from .binding import (AS_BF16, AS_BF16X3, AS_BF16X6, AS_FIXED_THETA, AS_FP32_PLAIN, AS_PERSISTENT, AS_PROFILE, AS_TRACE_DECISIONS,  # noqa: F401
                      AsConfig, AsEvent, AsStats, AeroSketchError, Sketch, lib, load_library)
