"""Pins of the oracle's model arithmetic: discretisation of eq. dynam and measurement functions."""
import numpy as np
import pytest

from oracle import fdm, model


def test_van_loan_scalar_closed_form():
    a, q, tau = -0.5, 0.5, 0.1
    Phi, Qd = model.van_loan(np.array([[a]]), np.array([[q]]), tau)
    assert abs(Phi[0, 0] - np.exp(a * tau)) < 1e-15
    assert abs(Qd[0, 0] - q * (np.exp(2 * a * tau) - 1) / (2 * a)) < 1e-15


def _quad_qd(A, Q, tau, n=2001):
    s = np.linspace(0.0, tau, n)
    w = np.full(n, 2.0)
    w[1::2] = 4.0
    w[0] = w[-1] = 1.0
    w *= (s[1] - s[0]) / 3.0
    acc = np.zeros_like(Q)
    for si, wi in zip(s, w):
        # Taylor series of e^{A s}, summed to convergence (independent of the library routine)
        E, term = np.eye(A.shape[0]), np.eye(A.shape[0])
        for k in range(1, 40):
            term = term @ (A * si) / k
            E = E + term
        acc += wi * E @ Q @ E.T
    return acc


def test_van_loan_matches_quadrature():
    A = np.array([[0.0, 1.0], [-1.0, -0.2]])
    Q = np.array([[0.1, 0.02], [0.02, 0.3]])
    tau = 0.37
    _, Qd = model.van_loan(A, Q, tau)
    np.testing.assert_allclose(Qd, _quad_qd(A, Q, tau), atol=1e-12)


def test_lyapunov_ode():
    """dQ_d/dtau = A Q_d + Q_d A^T + Q."""
    A = np.array([[-0.3, 0.8, 0.1], [-0.5, -0.2, 0.0], [0.2, 0.1, -0.7]])
    Q = np.diag([0.2, 0.2, 0.1])
    tau, h = 0.4, 1e-5
    _, Qp = model.van_loan(A, Q, tau + h)
    _, Qm = model.van_loan(A, Q, tau - h)
    _, Q0 = model.van_loan(A, Q, tau)
    np.testing.assert_allclose((Qp - Qm) / (2 * h), A @ Q0 + Q0 @ A.T + Q, atol=1e-8)


def test_backward_integral_identity():
    A = np.array([[0.0, 1.0], [-1.0, -0.2]])
    Q = np.diag([0.1, 0.3])
    tau = 0.05
    Qb = model.backward_diffusion_integral(A, Q, tau)
    np.testing.assert_allclose(Qb, _quad_qd(-A, Q, tau), atol=1e-13)


def test_wrap_angle():
    r = np.array([0.0, np.pi, -np.pi, 3 * np.pi, 2 * np.pi + 0.1, -2 * np.pi - 0.1])
    w = model.wrap_angle(r)
    np.testing.assert_allclose(w, [0.0, np.pi, np.pi, np.pi, 0.1, -0.1], atol=1e-12)
    assert np.all(w > -np.pi) and np.all(w <= np.pi)


def test_measurement_functions():
    x = np.array([[3.0, 4.0, 1.5], [-1.0, 0.0, -2.0]])
    np.testing.assert_allclose(model.h("range", x[:, :2]), [[5.0], [1.0]])
    np.testing.assert_allclose(model.h("bearing_linear3", x), [[np.arctan2(4, 3), 1.5], [np.pi, -2.0]])
    H = np.array([[1.0, 2.0, 0.0]])
    np.testing.assert_allclose(model.h("linear", x, H), [[11.0], [-1.0]])
    r = model.residual("bearing_linear3", np.array([-np.pi + 0.01, 0.0]), x[1:])
    assert abs(r[0, 0] - 0.01) < 1e-12


def test_gm_likelihood_is_the_mixture_density():
    """Sec. VI noise: exp(-gm_neg_log_lik) is w N(r; m1, v1) + (1 - w) N(r; m2, v2)."""
    from scipy.stats import norm
    p = np.zeros(24)
    p[17:22] = [0.3, -1.0, 20.0, 0.5, 4.0]
    r = np.linspace(-5.0, 30.0, 71)
    ref = 0.3 * norm.pdf(r, -1.0, np.sqrt(0.5)) + 0.7 * norm.pdf(r, 20.0, 2.0)
    np.testing.assert_allclose(np.exp(-model.gm_neg_log_lik(r, p)), ref, rtol=1e-13)
    # far tails stay finite in log form where the density itself underflows
    far = model.gm_neg_log_lik(np.array([1e4]), p)
    assert np.isfinite(far[0]) and far[0] > 700
    # weight 1 is a single Gaussian: -log N(r; m1, v1)
    p[17] = 1.0
    np.testing.assert_allclose(model.gm_neg_log_lik(r, p),
                               0.5 * np.log(2 * np.pi * 0.5) + 0.5 * (r + 1.0) ** 2 / 0.5, rtol=1e-13)


def test_terrain_measurement_special_values():
    """Terrain of four plane waves on a base; h reads positions from state axes 0 and 2."""
    p = np.zeros(24)
    p[16] = 500.0
    p[0:4] = [10.0, np.pi / 100.0, 0.0, 0.0]           # 10 sin(pi p_x / 100)
    p[4:8] = [3.0, 0.0, np.pi / 20.0, np.pi / 2.0]     # 3 cos(pi p_y / 20)
    x = np.array([[50.0, 7.0, 0.0, -2.0], [100.0, -1.0, 10.0, 5.0], [-50.0, 0.0, 20.0, 0.0]])
    np.testing.assert_allclose(model.h("terrain_gm", x, params=p)[:, 0], [513.0, 500.0, 487.0],
                               atol=1e-12)
    assert model.residual("terrain_gm", np.array([520.0]), x[:1], params=p)[0, 0] == pytest.approx(7.0)


def test_fst_inverse_and_eigenpairs():
    """R^{-1} = 2/(N+1) R and F_diff R = R diag(lambda) (Sec. III-C)."""
    N = 9
    R = fdm.sine_matrix(N)
    np.testing.assert_allclose(R @ R * (2.0 / (N + 1)), np.eye(N), atol=1e-13)
    F = fdm.fdiff_matrix(N, q=0.5, a=-0.5, dt=0.01, delta=0.3)
    lam = fdm.fdiff_eigenvalues(N, q=0.5, a=-0.5, dt=0.01, delta=0.3)
    np.testing.assert_allclose(F @ R, R @ np.diag(lam), atol=1e-12)


def test_fdm_product_equals_sine_transform_form():
    """Eq. FKEnumSol (explicit product) equals eq. FST (sine transforms) on the moving grid."""
    N, q, a, dt, l, d0 = 20, 0.5, -0.5, 0.01, 10, 0.3
    rng = np.random.default_rng(3)
    P = rng.uniform(size=N)
    T = fdm.fdm_transition(N, q, a, dt, l, d0)
    np.testing.assert_allclose(T @ P, fdm.fst_transition_apply(P, q, a, dt, l, d0), atol=1e-12)
