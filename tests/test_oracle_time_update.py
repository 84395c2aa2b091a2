"""Pins of the oracle's spectral time update (Sec. II-B, V) against the Gaussian FPE solution.

For a Gaussian prior the Fokker-Planck equation (eq. fokker) has the closed
form N(e^{A tau} m, e^{A tau} P e^{A^T tau} + Q_d(tau)); the exact-in-time
multiplier must reproduce it at spectral accuracy on any frame, including a
sheared one (off-diagonal Q_u: cross terms and the Nyquist reading), and the
Euler multiplier must converge to it at first order in the sub-step.
"""
import math

import numpy as np
import pytest

from oracle import filter as of
from oracle import model
from workloads import FilterConfig


def _gauss_density(x, m, C):
    d = x - m[None, :]
    q = np.einsum("pi,ij,pj->p", d, np.linalg.inv(C), d)
    return np.exp(-0.5 * q) / math.sqrt((2 * math.pi) ** len(m) * np.linalg.det(C))


def _cfg(A, Q, m0, P0, N, span=10.0, dt_sub=0.01):
    return FilterConfig(nx=len(m0), N=tuple(N), A=np.array(A, float), Q=np.array(Q, float),
                        m0=np.array(m0, float), P0=np.array(P0, float), span=span, dt_sub=dt_sub)


def _closed_form_error(f, tau):
    m0, C0 = f.moments()
    f.spectral_step(tau)
    Phi, Qd = model.van_loan(f.A, f.Q, tau)
    ref = _gauss_density(f.points(), Phi @ m0, Phi @ C0 @ Phi.T + Qd)
    return np.abs(f.P.ravel() - ref).sum() / np.abs(ref).sum()


def test_gaussian_fpe_exact_time_1d():
    f = of.OracleFilter(_cfg([[-0.5]], [[0.5]], [1.0], [[0.25]], [64]), psi_mode="exact")
    assert _closed_form_error(f, 0.1) < 1e-12


def test_gaussian_fpe_exact_time_sheared_2d():
    """Non-normal A, full Q and a sheared frame: Q_u has off-diagonal terms."""
    A = [[0.0, 1.0], [-1.0, -0.2]]
    Q = [[0.1, 0.03], [0.03, 0.3]]
    P0 = [[0.25, 0.15], [0.15, 0.25]]
    f = of.OracleFilter(_cfg(A, Q, [2.0, 0.0], P0, [48, 40]), psi_mode="exact")
    Mi = np.linalg.inv(f.M)
    Qu = Mi @ np.array(Q) @ Mi.T
    assert abs(Qu[0, 1]) > 0.1 * math.sqrt(Qu[0, 0] * Qu[1, 1])
    assert _closed_form_error(f, 0.3) < 1e-9


def test_gaussian_fpe_exact_time_3d():
    rng = np.random.default_rng(7)
    from workloads import random_stable_matrix
    A = random_stable_matrix(3, rng)
    Q = np.diag([0.2, 0.2, 0.1])
    P0 = 0.25 * np.eye(3) + 0.05
    f = of.OracleFilter(_cfg(A, Q, [3.0, 1.0, 0.0], P0, [32, 36, 40], span=8.0), psi_mode="exact")
    assert _closed_form_error(f, 0.1) < 1e-8


def test_gaussian_fpe_exact_time_4d_degenerate_q():
    """Coordinated turn (Sec. VI): rotating velocity, diffusion on the velocity axes
    only (singular Q) and a correlated prior, so Q_u has cross terms and the
    4-D sign-flip orbits of the parity fix-up are all exercised."""
    a = np.deg2rad(30.0)
    A = [[0, 1, 0, 0], [0, 0, 0, -a], [0, 0, 0, 1], [0, a, 0, 0]]
    Q = np.diag([0.0, 1.0, 0.0, 1.0])
    sd = np.sqrt([9.0, 4.0, 9.0, 4.0])
    R = np.array([[1.0, 0.3, -0.2, 0.1], [0.3, 1.0, 0.25, -0.3], [-0.2, 0.25, 1.0, 0.2], [0.1, -0.3, 0.2, 1.0]])
    P0 = sd[:, None] * R * sd[None, :]
    f = of.OracleFilter(_cfg(A, Q, [0.0, 5.0, 0.0, 5.0], P0, [32, 30, 34, 28], span=7.0), psi_mode="exact")
    Mi = np.linalg.inv(f.M)
    Qu = Mi @ Q @ Mi.T
    # the first frame axis sees no diffusion (rank-2 Q); the other three pairs couple
    assert np.count_nonzero(np.abs(Qu[np.triu_indices(4, 1)]) > 0.1) == 3
    assert _closed_form_error(f, 0.5) < 3e-9


def test_euler_first_order_in_substep():
    A = [[0.0, 1.0], [-1.0, -0.2]]
    Q = [[0.1, 0.0], [0.0, 0.3]]
    errs = []
    for dt_sub in (0.02, 0.01, 0.005):
        f = of.OracleFilter(_cfg(A, Q, [2.0, 0.0], np.diag([0.05, 0.05]), [48, 48], dt_sub=dt_sub))
        errs.append(_closed_form_error(f, 0.2))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2, errs


@pytest.mark.parametrize("mode", ["exact", "euler"])
def test_mass_balance(mode):
    """Psi(0) = 1: the transform keeps sum P; the frame volume grows by e^{tr(A) tau}."""
    A = np.array([[-0.3, 0.4], [0.1, -0.6]])
    f = of.OracleFilter(_cfg(A, np.diag([0.1, 0.2]), [0.5, -0.5], 0.3 * np.eye(2), [32, 32]),
                        psi_mode=mode)
    tau = 0.1
    f.spectral_step(tau)
    trA = np.trace(A)
    if mode == "exact":
        assert abs(f.last_mass_ratio - 1.0) < 1e-13
    else:
        l = f.substeps(tau)
        expect = (1.0 - tau / l * trA) ** l * math.exp(trA * tau)
        assert abs(f.last_mass_ratio - expect) < 1e-13
        assert abs(f.last_mass_ratio - 1.0) < 1e-3


def test_even_prior_stays_even_without_drift():
    f = of.OracleFilter(_cfg([[0.0, 0.0], [0.0, 0.0]], np.diag([0.3, 0.1]), [0.0, 0.0],
                             np.eye(2), [32, 24]))
    f.spectral_step(0.2)
    np.testing.assert_allclose(f.P, f.P[::-1, ::-1], atol=1e-14 * f.P.max())


def test_no_drift_diagonal_q_is_separable_heat_kernel():
    """A = 0 and diagonal Q: the exact 2-D update is the outer product of two 1-D updates.

    (The Euler multiplier 1/(1 - dt/2 sum_m c''_m Q_mm) of the algorithm is not
    a product over axes, so this holds for the exact-in-time multiplier only.)
    """
    cfg2 = _cfg([[0.0, 0.0], [0.0, 0.0]], np.diag([0.3, 0.1]), [0.2, -0.1], np.diag([0.5, 0.2]),
                [32, 24])
    f2 = of.OracleFilter(cfg2, psi_mode="exact")
    f2.spectral_step(0.2)
    fa = of.OracleFilter(_cfg([[0.0]], [[0.3]], [0.2], [[0.5]], [32]), psi_mode="exact")
    fb = of.OracleFilter(_cfg([[0.0]], [[0.1]], [-0.1], [[0.2]], [24]), psi_mode="exact")
    fa.spectral_step(0.2)
    fb.spectral_step(0.2)
    np.testing.assert_allclose(f2.P, np.outer(fa.P, fb.P), atol=1e-13 * f2.P.max())


def test_imaginary_part_vanishes():
    """The update is real for a jointly even multiplier (assertion inside the oracle)."""
    A = [[0.0, 1.0], [-1.0, -0.2]]
    f = of.OracleFilter(_cfg(A, [[0.1, 0.05], [0.05, 0.3]], [2.0, 0.0],
                             [[0.25, 0.1], [0.1, 0.25]], [32, 32]))
    f.spectral_step(0.05)
    assert np.all(np.isfinite(f.P))


def test_rough_data_sheared_frame_is_real():
    """Data with Nyquist content on a sheared frame: the update stays real only if the
    cross terms use the first-derivative coefficients with the Nyquist term omitted."""
    A = [[0.0, 1.0], [-1.0, -0.2]]
    f = of.OracleFilter(_cfg(A, [[0.1, 0.05], [0.05, 0.3]], [2.0, 0.0],
                             [[0.25, 0.15], [0.15, 0.25]], [16, 12]))
    f.P = np.random.default_rng(4).uniform(size=f.N)
    f.normalise()
    f.spectral_step(0.05)       # raises if the inverse transform has an imaginary part
    assert np.all(np.isfinite(f.P))
