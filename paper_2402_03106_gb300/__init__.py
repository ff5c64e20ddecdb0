"""DARTS transient path tracing on GB300 (sm_103a).

The hot path lives in libdarts.so (CUDA kernels behind the C ABI of
include/darts.h); ``paper_2402_03106_gb300.capi`` is its thin ctypes binding
and ``scenes`` holds the scene descriptions.  Importing the package loads
nothing native; the library is loaded on first use and a missing build
raises.
"""
from . import scenes  # noqa: F401
