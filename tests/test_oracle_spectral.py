"""Pins of the oracle's spectral operators (Sec. IV, V-A) against closed forms.

Each check is independent of the oracle's own construction: Trefethen's
closed-form periodic differentiation matrix (the paper's [Th:00]), exact
derivatives of a Gaussian, hand-evaluated tiny cases and brute-force sums.
"""
import os

import numpy as np
import pytest

from oracle import fdm, spectral

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


def trefethen_d2(N):
    """Closed-form periodic second-derivative matrix on [0, 2 pi), even N."""
    h = 2 * np.pi / N
    D = np.empty((N, N))
    for i in range(N):
        for j in range(N):
            d = i - j
            if d == 0:
                D[i, j] = -np.pi ** 2 / (3 * h ** 2) - 1.0 / 6.0
            else:
                D[i, j] = -((-1) ** d) / (2 * np.sin(d * h / 2) ** 2)
    return D


def test_wavenumbers_fftshift_golden():
    assert np.array_equal(spectral.wavenumbers(8), _golden("fftshift_n8.txt").astype(int))


def test_d2_golden_n4():
    D = spectral.spectral_d2_matrix(4, 2 * np.pi)
    np.testing.assert_allclose(D, _golden("d2_trefethen_n4.txt"), atol=1e-13)


@pytest.mark.parametrize("N", [4, 6, 8, 16, 32, 64])
def test_d2_matches_trefethen_closed_form(N):
    D = spectral.spectral_d2_matrix(N, 2 * np.pi)
    T = trefethen_d2(N)
    assert np.abs(D - T).max() <= 1e-11 * np.abs(T).max()


def test_d2_scaling_with_box_length():
    # d^2/dx^2 on a box of length L equals (2 pi / L)^2 times the [0, 2 pi) operator.
    N, L = 16, 3.7
    np.testing.assert_allclose(spectral.spectral_d2_matrix(N, L),
                               (2 * np.pi / L) ** 2 * trefethen_d2(N), atol=1e-11)


def test_dft_brute_force_n6():
    N = 6
    rng = np.random.default_rng(0)
    P = rng.standard_normal(N)
    F = spectral.dft_matrix(N) @ P
    for s in range(N):
        acc = 0j
        for j in range(N):
            acc += P[j] * complex(np.cos(2 * np.pi * j * s / N), -np.sin(2 * np.pi * j * s / N))
        assert abs(F[s] - acc / N) < 1e-14
    np.testing.assert_allclose(spectral.synthesis_matrix(N) @ F, P, atol=1e-14)


def _gauss(x, mu, s):
    return np.exp(-0.5 * ((x - mu) / s) ** 2)


def _gauss_d2(x, mu, s):
    return (((x - mu) ** 2) / s ** 4 - 1.0 / s ** 2) * _gauss(x, mu, s)


def test_d2_gaussian_spectral_vs_fdm_convergence():
    """Spectral error falls faster than any power of N; central differences fall as N^-2 (Sec. III-D, IV)."""
    L, mu, s = 20.0, 10.0, 1.0           # box of +-10 sigma: wrap floor ~ e^{-50}
    Ns = [16, 24, 32, 48, 64, 96]
    e_sp, e_fd = [], []
    for N in Ns:
        x = np.arange(N) * L / N
        f, d2 = _gauss(x, mu, s), _gauss_d2(x, mu, s)
        e_sp.append(np.abs(spectral.spectral_d2_matrix(N, L) @ f - d2).max())
        e_fd.append(np.abs(fdm.central_d2_matrix(N, L / N) @ f - d2).max())
    e_sp, e_fd = np.array(e_sp), np.array(e_fd)
    # FDM: log-log slope -2 over the last points
    slope = np.polyfit(np.log(Ns[2:]), np.log(e_fd[2:]), 1)[0]
    assert -2.2 < slope < -1.8
    # spectral: exponential decay; by N = 64 at round-off level
    assert e_sp[3] < 1e-4 * e_sp[0]
    assert e_sp[4] < 1e-10
    assert np.all(e_sp[2:] < e_fd[2:] * 1e-3)


def test_d1_gaussian_exact_derivative():
    L, mu, s, N = 20.0, 10.0, 1.0, 64
    x = np.arange(N) * L / N
    d1 = -(x - mu) / s ** 2 * _gauss(x, mu, s)
    assert np.abs(spectral.spectral_d1_matrix(N, L) @ _gauss(x, mu, s) - d1).max() < 1e-10


def test_d2_annihilates_constants_and_is_symmetric():
    for N in (6, 10, 32):
        D = spectral.spectral_d2_matrix(N, 1.0)
        assert np.abs(D @ np.ones(N)).max() < 1e-9 * np.abs(D).max()
        assert np.abs(D - D.T).max() < 1e-10 * np.abs(D).max()


def test_interp_reproduces_trig_polynomials():
    """The interpolant of eq. interFreq is exact on trig polynomials with |freq| < N/2 plus the Nyquist cosine."""
    N = 12
    rng = np.random.default_rng(1)
    a = rng.standard_normal(N // 2)
    b = rng.standard_normal(N // 2)
    cn = rng.standard_normal()

    def f(x):
        out = a[0] * np.ones_like(x) + cn * np.cos(np.pi * x)
        for k in range(1, N // 2):
            out += a[k] * np.cos(2 * np.pi * k * x / N) + b[k] * np.sin(2 * np.pi * k * x / N)
        return out

    nodes = np.arange(N, dtype=float)
    xq = rng.uniform(-2, N + 2, size=40)
    np.testing.assert_allclose(spectral.interp_matrix(N, xq) @ f(nodes), f(xq), atol=1e-12)


def test_interp_identity_at_nodes():
    N = 16
    np.testing.assert_allclose(spectral.interp_matrix(N, np.arange(N)), np.eye(N), atol=1e-13)


def test_interp_equals_periodic_sinc():
    """Trefethen's periodic sinc for even N: S(x) = sin(pi x) / (N tan(pi x / N))."""
    N = 10
    xq = np.array([0.3, 1.7, -2.2, 4.5])
    E = spectral.interp_matrix(N, xq)
    for i, x in enumerate(xq):
        for j in range(N):
            v = x - j
            ref = np.sin(np.pi * v) / (N * np.tan(np.pi * v / N))
            assert abs(E[i, j] - ref) < 1e-13
