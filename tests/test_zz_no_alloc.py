"""pmf_moments_noalloc: moments without device allocation, against pmf_moments.

This entry point exists for callers that cannot allocate device memory when
they need the moments (CUDA graph capture, hosts whose allocator owns the
device memory, real-time loops).  It must give the same mean and covariance
as the context's pmf_moments on the same weights, call after call (its
partial sums live in one shared static device array that each call reuses).
Collected last on purpose.
"""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _reference(sc, epochs):
    from paper_2412_07240_gb300 import Filter
    f = Filter(sc.cfg, precision="fp64")
    for k in range(epochs):
        f.meas_update(sc.meas, sc.z[k])
        f.time_update(sc.dt)
    m, C = f.moments()
    P, c, M = f.pdf()
    f.close()
    return m, C, P, c, M


@pytest.mark.parametrize("make", [lambda: w.small_2d_scenario(N=(48, 40), epochs=3),
                                  lambda: w.small_3d_scenario(N=(16, 24, 20), epochs=2)])
def test_noalloc_moments_match_context_moments_twice(make):
    import torch
    from paper_2412_07240_gb300._binding import moments_noalloc
    sc = make()
    m, C, P, c, M = _reference(sc, sc.epochs)
    n = sc.cfg.nx
    wdev = torch.from_numpy(P.ravel().copy()).cuda()
    for _ in range(2):                      # two calls in a row share the static scratch
        out = torch.full((1 + n + n * n,), float("nan"), dtype=torch.float64, device="cuda")
        moments_noalloc(wdev, P.shape, c, M, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert abs(o[0] * abs(np.linalg.det(M)) - 1.0) < TOL      # normalised weights
        assert np.abs(o[1:1 + n] - m).max() <= TOL * np.sqrt(np.trace(C)) + 1e-15
        assert np.abs(o[1 + n:].reshape(n, n) - C).max() <= TOL * np.abs(C).max()


def test_noalloc_rejects_oversized_grids():
    import ctypes
    from paper_2412_07240_gb300 import _binding
    lib = _binding.load()
    N = (ctypes.c_int * 2)(2048, 1024)      # 2^21 points > PMF_NOALLOC_MAX_POINTS
    c = (ctypes.c_double * 2)(0.0, 0.0)
    M = (ctypes.c_double * 4)(1.0, 0.0, 0.0, 1.0)
    rc = lib.pmf_moments_noalloc(ctypes.c_void_p(16), 2, N, c, M, ctypes.c_void_p(16), None)
    assert rc == _binding.ERR_ARG
