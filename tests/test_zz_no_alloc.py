"""pmf_moments_noalloc: moments without device allocation.

This entry point exists for callers that cannot allocate device memory when
they need the moments: hosts whose own allocator owns the device memory, and
real-time loops that must not pay for (or risk the failure of) a cudaMalloc.
It must give the mean and covariance of the point sums of the weights it is
given, call after call, although its block partial sums live in one static
device array that every call reuses.  The expected values here are numpy
point sums of the same weights, and the context's own pmf_moments.  The file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _point_sums(P, c, M):
    """S0, mean and covariance of the point masses P on the frame x = c + M u."""
    n = P.ndim
    u = np.meshgrid(*[np.arange(N) - 0.5 * (N - 1) for N in P.shape], indexing="ij")
    u = np.stack([a.ravel() for a in u])                    # (n, prod N)
    p = P.ravel()
    S0 = p.sum()
    mu = (u * p).sum(axis=1) / S0
    d = u - mu[:, None]
    Cu = (d * p) @ d.T / S0
    M = np.asarray(M).reshape(n, n)
    return S0, np.asarray(c) + M @ mu, M @ Cu @ M.T


def _call_twice(P, c, M):
    import torch
    from paper_2412_07240_gb300._binding import moments_noalloc
    n = P.ndim
    wdev = torch.from_numpy(P.ravel().copy()).cuda()
    outs = []
    for _ in range(2):                      # two calls in a row share the static scratch
        out = torch.full((1 + n + n * n,), float("nan"), dtype=torch.float64, device="cuda")
        moments_noalloc(wdev, P.shape, c, M, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    return outs


def _check(o, S0, m, C, n):
    assert abs(o[0] - S0) <= TOL * abs(S0)
    assert np.abs(o[1:1 + n] - m).max() <= TOL * np.sqrt(np.trace(C)) + 1e-15
    assert np.abs(o[1 + n:].reshape(n, n) - C).max() <= TOL * np.abs(C).max()


@pytest.mark.parametrize("make", [lambda: w.small_2d_scenario(N=(48, 40), epochs=3),
                                  lambda: w.small_3d_scenario(N=(16, 24, 20), epochs=2)])
def test_noalloc_moments_match_point_sums_and_context_twice(make):
    from paper_2412_07240_gb300 import Filter
    sc = make()
    f = Filter(sc.cfg, precision="fp64")
    for k in range(sc.epochs):
        f.meas_update(sc.meas, sc.z[k])
        f.time_update(sc.dt)
    m_ctx, C_ctx = f.moments()
    P, c, M = f.pdf()
    f.close()
    n = sc.cfg.nx
    S0, m, C = _point_sums(P, c, M)
    for o in _call_twice(P, c, M):
        _check(o, S0, m, C, n)
        _check(o, S0, m_ctx, C_ctx, n)
        assert abs(o[0] * abs(np.linalg.det(M)) - 1.0) < TOL      # the context's weights are normalised


def test_noalloc_largest_grid_uses_every_partial_block():
    """2^20 points: all 4096 partial blocks of the static array are written and summed."""
    rng = np.random.default_rng(11)
    P = rng.random((1024, 1024)) * np.exp(-np.linspace(-3, 3, 1024) ** 2)[:, None]
    c = np.array([0.3, -1.2])
    M = np.array([[0.02, 0.001], [-0.003, 0.015]])
    S0, m, C = _point_sums(P, c, M)
    for o in _call_twice(P, c, M):
        _check(o, S0, m, C, 2)
    # a smaller grid right after reuses only the first partials
    P2 = rng.random((24, 16, 8))
    M2 = np.diag([0.1, 0.2, 0.3])
    S0, m, C = _point_sums(P2, np.zeros(3), M2)
    for o in _call_twice(P2, np.zeros(3), M2):
        _check(o, S0, m, C, 3)


def test_noalloc_zero_mass_gives_nan_moments():
    P = np.zeros((32, 16))
    for o in _call_twice(P, np.zeros(2), np.eye(2)):
        assert o[0] == 0.0 and np.isnan(o[1:]).all()


def test_noalloc_rejects_oversized_grids():
    from paper_2412_07240_gb300 import _binding
    lib = _binding.load()
    c = (ctypes.c_double * 4)()
    M = (ctypes.c_double * 16)()
    N = (ctypes.c_int * 2)(2048, 1024)      # 2^21 points > PMF_NOALLOC_MAX_POINTS
    rc = lib.pmf_moments_noalloc(ctypes.c_void_p(16), 2, N, c, M, ctypes.c_void_p(16), None)
    assert rc == _binding.ERR_ARG
    big = 2 ** 31 - 1                       # the product of four such axes overflows 64 bits
    N4 = (ctypes.c_int * 4)(big, big, big, big)
    rc = lib.pmf_moments_noalloc(ctypes.c_void_p(16), 4, N4, c, M, ctypes.c_void_p(16), None)
    assert rc == _binding.ERR_ARG
