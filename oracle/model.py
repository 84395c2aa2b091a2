"""Model arithmetic of the oracle (Sec. I eqs. dynam/meas, Sec. II).

dx = A x dt + Q dw with E[dw dw^T] = I dt, Q read as the diffusion
(covariance-rate) matrix of the Fokker-Planck equation (eq. fokker);
z = h(x) + v, v ~ N(0, R).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def expm(X: np.ndarray) -> np.ndarray:
    """Matrix exponential (library primitive)."""
    return sla.expm(np.asarray(X, dtype=float))


def van_loan(A: np.ndarray, Q: np.ndarray, tau: float):
    """Phi = e^{A tau} and Q_d = int_0^tau e^{A s} Q e^{A^T s} ds.

    Van Loan (1978): expm([[-A, Q], [0, A^T]] tau) = [[., F12], [0, F22]] with
    F22 = Phi^T and F12 = Phi^{-1} Q_d, so Q_d = Phi F12.
    """
    n = A.shape[0]
    C = np.zeros((2 * n, 2 * n))
    C[:n, :n] = -A
    C[:n, n:] = Q
    C[n:, n:] = A.T
    E = expm(C * tau)
    Phi = E[n:, n:].T
    Qd = Phi @ E[:n, n:]
    return Phi, 0.5 * (Qd + Qd.T)


def backward_diffusion_integral(A: np.ndarray, Q: np.ndarray, tau: float) -> np.ndarray:
    """Q_b = int_0^tau e^{-A s} Q e^{-A^T s} ds = Phi^{-1} Q_d Phi^{-T}."""
    Phi, Qd = van_loan(A, Q, tau)
    Pi = np.linalg.inv(Phi)
    Qb = Pi @ Qd @ Pi.T
    return 0.5 * (Qb + Qb.T)


def terrain(params, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Smooth synthetic terrain altitude (stands in for the paper's map, Sec. VI):
    params[16] + sum_{i<4} params[4i] sin(params[4i+1] p_x + params[4i+2] p_y + params[4i+3])."""
    p = np.asarray(params, dtype=float)
    out = np.full(np.shape(px), p[16])
    for i in range(4):
        out = out + p[4 * i] * np.sin(p[4 * i + 1] * px + p[4 * i + 2] * py + p[4 * i + 3])
    return out


def gm_neg_log_lik(r: np.ndarray, params) -> np.ndarray:
    """-log of the two-component Gaussian mixture density of the residual r
    (Sec. VI): weight params[17] and 1 - params[17], means params[18], params[19],
    variances params[20], params[21]."""
    p = np.asarray(params, dtype=float)
    w = np.array([p[17], 1.0 - p[17]])
    mu, var = np.array([p[18], p[19]]), np.array([p[20], p[21]])
    with np.errstate(divide="ignore"):
        lg = (np.log(w)[None, :] - 0.5 * np.log(2.0 * np.pi * var)[None, :]
              - 0.5 * (np.asarray(r, dtype=float)[:, None] - mu[None, :]) ** 2 / var[None, :])
    return -np.logaddexp(lg[:, 0], lg[:, 1])


def h(kind: str, x: np.ndarray, H=None, params=None) -> np.ndarray:
    """Measurement function for points x of shape (P, n); returns (P, nz)."""
    if kind == "linear":
        return x @ np.asarray(H).T
    if kind == "range":
        return np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)[:, None]
    if kind == "bearing_linear3":
        return np.stack([np.arctan2(x[:, 1], x[:, 0]), x[:, 2]], axis=1)
    if kind == "terrain_gm":   # state [p_x, v_x, p_y, v_y]
        return terrain(params, x[:, 0], x[:, 2])[:, None]
    raise ValueError(kind)


def wrap_angle(r: np.ndarray) -> np.ndarray:
    """Wrap an angle residual to (-pi, pi]."""
    return r - 2.0 * np.pi * np.ceil((r - np.pi) / (2.0 * np.pi))


def residual(kind: str, z: np.ndarray, x: np.ndarray, H=None, params=None) -> np.ndarray:
    """z - h(x) with the bearing component wrapped to (-pi, pi]."""
    r = np.asarray(z, dtype=float)[None, :] - h(kind, x, H, params)
    if kind == "bearing_linear3":
        r[:, 0] = wrap_angle(r[:, 0])
    return r
