"""Finite-difference comparator on the moving grid (Sec. III-B, III-C).

One-dimensional model dx = a x dt + q dw on N interior nodes with zero
(Dirichlet) boundary values.  The explicit scheme with central differences
for diffusion, written as the tridiagonal matrix of eq. fdiff,

    F_diff(t) = tridiag(a_t, b_t, a_t),  a_t = q dt / (2 delta_t^2),
    b_t = 1 - q dt / delta_t^2 - dt a,

is applied once per sub-step while the spacing moves as
delta_n = e^{a dt} delta_{n-1} (eq. gridMov).  Its product over a time update
(eq. FKEnumSol) is compared with the sine-transform form of eq. FST: the
eigenvectors r^(j) = sin(i j pi / (N+1)) are constant, R^{-1} = 2/(N+1) R and
the eigenvalues are b_t + 2 a_t cos(j pi / (N+1)).

Reading: l explicit factors evaluated at the sub-step starts t_k + n dt,
n = 0..l-1 (the factor count printed in the two displayed products differs by
one).
"""
from __future__ import annotations

import numpy as np


def fdiff_matrix(N: int, q: float, a: float, dt: float, delta: float) -> np.ndarray:
    """Eq. fdiff for one sub-step."""
    at = q * dt / (2.0 * delta ** 2)
    bt = 1.0 - q * dt / delta ** 2 - dt * a
    F = np.diag(np.full(N, bt)) + np.diag(np.full(N - 1, at), 1) + np.diag(np.full(N - 1, at), -1)
    return F


def fdm_transition(N: int, q: float, a: float, dt: float, l: int, delta0: float) -> np.ndarray:
    """T_k of eq. FKEnumSol as an explicit product of l factors."""
    T = np.eye(N)
    delta = delta0
    for _ in range(l):
        T = fdiff_matrix(N, q, a, dt, delta) @ T
        delta = np.exp(a * dt) * delta
    return T


def sine_matrix(N: int) -> np.ndarray:
    """R with columns r^(j-1) = [sin(i j pi / (N+1))]_i, i, j = 1..N."""
    i = np.arange(1, N + 1)
    return np.sin(np.outer(i, i) * np.pi / (N + 1))


def fdiff_eigenvalues(N: int, q: float, a: float, dt: float, delta: float) -> np.ndarray:
    """lambda^(j-1) = b_t + 2 a_t cos(j pi / (N+1)), j = 1..N."""
    at = q * dt / (2.0 * delta ** 2)
    bt = 1.0 - q * dt / delta ** 2 - dt * a
    j = np.arange(1, N + 1)
    return bt + 2.0 * at * np.cos(j * np.pi / (N + 1))


def fst_transition_apply(P: np.ndarray, q: float, a: float, dt: float, l: int,
                         delta0: float) -> np.ndarray:
    """Eq. FST: P_{k+1} = S(diag(Lambda) . S(P)) with S the sine transform, Lambda = prod lambda."""
    N = P.size
    R = sine_matrix(N)
    lam = np.ones(N)
    delta = delta0
    for _ in range(l):
        lam = lam * fdiff_eigenvalues(N, q, a, dt, delta)
        delta = np.exp(a * dt) * delta
    return (2.0 / (N + 1)) * (R @ (lam * (R @ P)))


def central_d2_matrix(N: int, h: float, periodic: bool = True) -> np.ndarray:
    """Second-order central difference for the second derivative (the FDM's spatial operator)."""
    D = (np.diag(np.full(N, -2.0)) + np.diag(np.ones(N - 1), 1) + np.diag(np.ones(N - 1), -1))
    if periodic:
        D[0, -1] = D[-1, 0] = 1.0
    return D / h ** 2
