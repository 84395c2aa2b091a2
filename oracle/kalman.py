"""Continuous-discrete Kalman filter: the exact filter for linear h (Sec. II, Kalman-Bucy prediction).

For dx = A x dt + Q dw and z = H x + v the filtering density stays Gaussian;
its prediction over tau is N(Phi m, Phi P Phi^T + Q_d) with Phi = e^{A tau}
and Q_d from the Van Loan block exponential, and its Bayes update (eq. filt)
is the Kalman update.  The cycle matches the point-mass filter's: update at
t_0 on the prior, then predict to the next epoch.
"""
from __future__ import annotations

import numpy as np

from . import model


def kalman_update(m, P, H, R, z):
    S = H @ P @ H.T + R
    K = P @ H.T @ np.linalg.inv(S)
    m2 = m + K @ (z - H @ m)
    I = np.eye(P.shape[0])
    P2 = (I - K @ H) @ P @ (I - K @ H).T + K @ R @ K.T
    return m2, 0.5 * (P2 + P2.T)


def kalman_predict(m, P, A, Q, tau):
    Phi, Qd = model.van_loan(A, Q, tau)
    P2 = Phi @ P @ Phi.T + Qd
    return Phi @ m, 0.5 * (P2 + P2.T)


def run(m0, P0, A, Q, H, R, zs, tau):
    """Posterior (after each update) and predicted (after each prediction) moments."""
    m, P = np.asarray(m0, float), np.asarray(P0, float)
    post, pred = [], []
    for k, z in enumerate(zs):
        m, P = kalman_update(m, P, H, R, np.asarray(z, float))
        post.append((m.copy(), P.copy()))
        m, P = kalman_predict(m, P, A, Q, tau)
        pred.append((m.copy(), P.copy()))
    return post, pred
