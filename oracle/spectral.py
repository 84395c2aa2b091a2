"""Spectral differentiation of a periodic point-mass density (Sec. IV, V-A).

All routines are explicit O(N^2) matrix constructions in complex float64;
no FFT library is used.  Grid nodes are x_j = j * delta, j = 0..N-1 (the
paper's indexing from 0), with box length L = N * delta.
"""
from __future__ import annotations

import numpy as np


def wavenumbers(N: int) -> np.ndarray:
    """Integer frequency k_s of DFT index s: fftshift(-N/2 : N/2-1) (Sec. V-A).

    For even N this is [0, 1, ..., N/2-1, -N/2, ..., -1]; index s = N/2 is the
    Nyquist frequency -N/2.
    """
    if N % 2:
        raise ValueError("N must be even (Sec. IV)")
    k = np.arange(N)
    k[k >= N // 2] -= N
    return k


def dft_matrix(N: int) -> np.ndarray:
    """Eq. fourtrsf: P^(s) = (1/N) sum_j P^(j) exp(-2 pi i j s / N)."""
    j = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(j, j) / N) / N


def synthesis_matrix(N: int) -> np.ndarray:
    """Evaluate the trigonometric interpolant at the nodes: sum_s P^(s) e^{2 pi i j s/N}.

    At the nodes the Nyquist term P^(N/2) cos(pi j) equals P^(N/2) e^{i pi j},
    so this is the plain inverse of :func:`dft_matrix`.
    """
    j = np.arange(N)
    return np.exp(2j * np.pi * np.outer(j, j) / N)


def c2_coeffs(N: int, L: float) -> np.ndarray:
    """Second-derivative coefficients c'' = -(2 pi k / L)^2 (Sec. V-A), Nyquist included.

    At the Nyquist index the value -(pi N / L)^2 is the coefficient of the
    P^(N/2) (-1)^j term of eq. secDer.
    """
    return -(2.0 * np.pi / L * wavenumbers(N)) ** 2


def c1_coeffs(N: int, L: float) -> np.ndarray:
    """First-derivative coefficients c' = 2 pi i k / L for 0 < |k| < N/2, 0 at Nyquist.

    The first derivative of the interpolant (eq. interFreq) sums only over
    0 < s < N/2 and its mirror; the Nyquist cosine has zero slope at the nodes.
    """
    k = wavenumbers(N).astype(float)
    k[N // 2] = 0.0
    return 2j * np.pi / L * k


def spectral_d2_matrix(N: int, L: float) -> np.ndarray:
    """Matrix of eq. secDer: p'' at the nodes from P at the nodes."""
    D = synthesis_matrix(N) @ np.diag(c2_coeffs(N, L)) @ dft_matrix(N)
    return D.real


def spectral_d1_matrix(N: int, L: float) -> np.ndarray:
    """Matrix of the first spectral derivative at the nodes."""
    D = synthesis_matrix(N) @ np.diag(c1_coeffs(N, L)) @ dft_matrix(N)
    return D.real


def interp_matrix(N: int, x: np.ndarray) -> np.ndarray:
    """Eq. interFreq evaluated at positions x (index units, node j at x = j).

    p(x) = P^(0) + sum_{0<s<N/2} (P^(s) e^{2 pi i s x / N} + P^(N-s) e^{-2 pi i s x / N})
           + P^(N/2) cos(pi x),
    with L = N (unit spacing).  Returns the real matrix E F with p(x) = (E F) P.
    """
    x = np.asarray(x, dtype=float)
    s = np.arange(N)
    E = np.zeros((x.size, N), dtype=complex)
    E[:, 0] = 1.0
    for si in range(1, N // 2):
        E[:, si] = np.exp(2j * np.pi * si * x / N)
        E[:, N - si] = np.exp(-2j * np.pi * si * x / N)
    E[:, N // 2] = np.cos(np.pi * x)
    del s
    M = E @ dft_matrix(N)
    return M.real


def apply_along_axis(Mat: np.ndarray, X: np.ndarray, axis: int) -> np.ndarray:
    """Y[..., k, ...] = sum_j Mat[k, j] X[..., j, ...] along ``axis``."""
    Y = np.tensordot(Mat, X, axes=([1], [axis]))
    return np.moveaxis(Y, 0, axis)
