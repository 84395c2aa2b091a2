"""GB300-native spectral point-mass filter (hot path of arXiv 2412.07240).

The filter runs in hand-written sm_103a CUDA kernels behind the C ABI of
include/pmf.h (libpmf.so, built in-tree by ``build.build()``); this package
is a thin ctypes binding with the same entry points.
"""
from ._binding import (  # noqa: F401
    Batch, Degenerate, Filter, PmfError, Server, Unsupported, fdm_transition, load, lib_path, make_config,
    make_meas, selftest_bounded_wait,
)
