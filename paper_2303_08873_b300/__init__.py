"""Adaptive regions on one B300: variant selection by profiling and learned
models (arXiv 2303.08873), with hand-written sm_103a CUDA loop variants.

The package is a thin ctypes binding over ``libadaptive_region.so`` (C ABI in
``include/ar.h`` and ``include/ar_loops.h``).  Every step of the hot path runs
in that library's kernels and host runtime; importing the package fails if the
library is missing -- there is no fallback implementation.
"""
from .binding import *  # noqa: F401,F403
from .binding import ArError, lib, LIB_PATH  # noqa: F401
