"""Finite-difference comparator on the GPU (eq. fdiff / eq. FST): parity with
the oracle, second-order convergence, and the spectral method's accuracy per
grid point against it (the Gaussian FPE closed form as the arbiter)."""
import numpy as np
import pytest

import workloads as w
from oracle import fdm

pytestmark = pytest.mark.gpu

A, Q, S0, TAU = -0.5, 0.5, 0.5, 0.5
VAR = np.exp(2 * A * TAU) * S0 ** 2 + Q * (np.exp(2 * A * TAU) - 1) / (2 * A)


def _gpu_fdm(P, q, a, dt, l, d0):
    import torch
    from paper_2412_07240_gb300 import fdm_transition
    count, N = P.shape
    Pin = torch.tensor(P, dtype=torch.float64, device="cuda")
    Pout = torch.empty_like(Pin)
    work = torch.empty(count * N + 4 * N + 2, dtype=torch.float64, device="cuda")
    fdm_transition(Pin, Pout, work, q, a, dt, l, d0)
    torch.cuda.synchronize()
    return Pout.cpu().numpy()


@pytest.mark.parametrize("N", [16, 63, 200])
def test_matches_oracle(N):
    rng = np.random.default_rng(N)
    P = rng.uniform(0.0, 1.0, size=(3, N))
    q, a, dt, l, d0 = 0.5, -0.5, 1e-3, 50, 0.2
    out = _gpu_fdm(P, q, a, dt, l, d0)
    for g in range(3):
        ref = fdm.fst_transition_apply(P[g], q, a, dt, l, d0)
        assert np.abs(out[g] - ref).max() <= 1e-12 * np.abs(ref).max()
        prod = fdm.fdm_transition(N, q, a, dt, l, d0) @ P[g]   # explicit product of eq. fdiff factors
        assert np.abs(out[g] - prod).max() <= 1e-10 * np.abs(prod).max()


def _fdm_error(N, dt=1e-3):
    L0 = 6 * np.sqrt(VAR) / np.exp(A * TAU) * 1.05
    d0 = 2 * L0 / N
    x0 = (np.arange(N) - (N - 1) / 2) * d0
    P = np.exp(-0.5 * x0 ** 2 / S0 ** 2) / np.sqrt(2 * np.pi * S0 ** 2)
    out = _gpu_fdm(P[None, :], Q, A, dt, int(round(TAU / dt)), d0)[0]
    xt = x0 * np.exp(A * TAU)
    ex = np.exp(-0.5 * xt ** 2 / VAR) / np.sqrt(2 * np.pi * VAR)
    return np.abs(out - ex).max() / ex.max()


def _spectral_error(N):
    from paper_2412_07240_gb300 import Filter
    cfg = w.FilterConfig(nx=1, N=(N,), A=np.array([[A]]), Q=np.array([[Q]]), m0=np.array([0.0]),
                         P0=np.array([[S0 ** 2]]))
    f = Filter(cfg, precision="fp64", psi_mode="exact")
    f.time_update(TAU)
    P, c, M = f.pdf()
    f.close()
    x = c[0] + M[0, 0] * (np.arange(N) - (N - 1) / 2)
    ex = np.exp(-0.5 * x ** 2 / VAR) / np.sqrt(2 * np.pi * VAR)
    return np.abs(P.ravel() - ex).max() / ex.max()


def test_fdm_second_order_and_spectral_accuracy_per_point():
    e = [_fdm_error(N) for N in (64, 128, 256)]
    for coarse, fine in zip(e, e[1:]):
        assert 3.0 < coarse / fine < 5.5, e          # O(delta^2)
    s24 = _spectral_error(24)
    assert s24 < 1e-7, s24                          # at the +-6 sigma wrap floor
    assert s24 < e[-1] / 1e3, (s24, e)              # 24 spectral points beat 256 FDM points
