"""Pins of the oracle's cycle with nonlinear measurements (range, bearing),
against quantities computed here independently of the oracle's grid.

Bayes' rule (eq. filt) on a Gaussian prior with a range or bearing likelihood
has no closed form, but its moments are integrals that a quadrature in polar
(cylindrical) coordinates about the sensor evaluates to round-off: the
likelihood depends on the radius (range) or the angle (bearing) only, and
both integrands are smooth and, in the angle, periodic.  The time update that
follows is pinned twice: linear dynamics carry the first two moments of ANY
density exactly (m -> Phi m, C -> Phi C Phi^T + Q_d), and the predicted
density itself is the Chapman-Kolmogorov integral of the posterior against
the Gaussian transition kernel, evaluated here at sampled grid nodes.  Every
model quantity below (h, the angle wrap, Phi, Q_d) is written from its
definition in this file, not taken from the oracle.

The problems are chosen so that the oracle's grid resolves the posterior
(about two nodes per posterior standard deviation or more: trapezoid sums of
a smooth density are then accurate to round-off, and the band-limited regrid
interpolant to ~e^{-pi^2 (sigma/h)^2 / 2}), so the bars are tight and
planted mistakes in the oracle's h or wrap trip them.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as w
from oracle import filter as of
from oracle import model
from workloads import FilterConfig, MeasModel


def _gauss(x, m, C):
    """N(x; m, C) for points x of shape (..., n)."""
    d = x - m
    Ci = np.linalg.inv(C)
    q = np.einsum("...i,ij,...j->...", d, Ci, d)
    return np.exp(-0.5 * q) / np.sqrt((2 * np.pi) ** len(m) * np.linalg.det(C))


def _gl(a, b, n):
    t, wt = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * t + 0.5 * (b + a), 0.5 * (b - a) * wt


def _phi_qd(A, Q, tau, n=64):
    """e^{A tau} and Q_d = int_0^tau e^{A s} Q e^{A^T s} ds (Gauss-Legendre in s)."""
    s, ws = _gl(0.0, tau, n)
    Qd = sum(wk * sla.expm(A * sk) @ Q @ sla.expm(A * sk).T for sk, wk in zip(s, ws))
    return sla.expm(A * tau), 0.5 * (Qd + Qd.T)


def _moments(x, wq):
    S0 = wq.sum()
    m = (wq[:, None] * x).sum(axis=0) / S0
    d = x - m
    return m, (wq[:, None] * d).T @ d / S0


# --- range (n_x = 2) ---------------------------------------------------------------

def _range_problem(N=(64, 64)):
    P0 = np.array([[0.25, 0.08], [0.08, 0.2]])
    cfg = FilterConfig(nx=2, N=N, A=np.array([[0.0, 1.0], [-1.0, -0.2]]), Q=np.diag([0.1, 0.3]),
                       m0=np.array([2.0, 0.0]), P0=P0)
    meas = MeasModel("range", R=np.array([[0.15 ** 2]]))
    return cfg, meas, np.array([2.1])


def _range_nodes(cfg, z, sig, nr=400, nth=2048):
    """Polar quadrature nodes (x, weight incl. the Jacobian r) of the posterior
    p(x) ~ N(x; m0, P0) exp(-(z - |x|)^2 / (2 sig^2)), normalised weights."""
    r, wr = _gl(max(1e-9, z - 12 * sig), z + 12 * sig, nr)
    th = 2 * np.pi * np.arange(nth) / nth
    R_, T_ = np.meshgrid(r, th, indexing="ij")
    x = np.stack([(R_ * np.cos(T_)).ravel(), (R_ * np.sin(T_)).ravel()], axis=1)
    jac = (wr[:, None] * R_ * (2 * np.pi / nth)).ravel()
    rad = np.hypot(x[:, 0], x[:, 1])
    wq = jac * _gauss(x, cfg.m0, cfg.P0) * np.exp(-0.5 * (z - rad) ** 2 / sig ** 2)
    return x, wq / wq.sum()


def _range_oracle_cycle(cfg, meas, z, tau):
    f = of.OracleFilter(cfg, psi_mode="exact")
    f.meas_update(meas, z)
    post = f.moments()
    f.time_update(tau)
    return f, post, f.moments()


def _rel(m, C, mr, Cr):
    return (np.abs(m - mr).max() / np.sqrt(np.trace(Cr)), np.abs(C - Cr).max() / np.abs(Cr).max())


def _range_cycle_errors(span):
    """Oracle errors after the update and after the prediction, on a grid of
    16 nodes per prior sigma of box (posterior radial sigma ~ 2.4 nodes)."""
    cfg, meas, z = _range_problem((int(16 * span),) * 2)
    cfg.span = span
    tau = 0.05
    x, wq = _range_nodes(cfg, z[0], 0.15)
    mq, Cq = _moments(x, wq)
    f, (m, C), (mp, Cp) = _range_oracle_cycle(cfg, meas, z, tau)
    post = _rel(m, C, mq, Cq)
    # moments of any density move exactly under linear dynamics
    Phi, Qd = _phi_qd(cfg.A, cfg.Q, tau)
    pred = _rel(mp, Cp, Phi @ mq, Phi @ Cq @ Phi.T + Qd)
    # the predicted density at sampled nodes: int N(x; Phi y, Q_d) p_post(y) dy
    pts = f.points()
    Pf = f.P.ravel()
    idx = np.argsort(Pf)[::-1][:: max(1, Pf.size // 4000)][:48]      # spread over the mass
    y = x @ Phi.T
    ref = np.array([(wq * _gauss(y, xs, Qd)).sum() for xs in pts[idx]])
    return post, pred, np.abs(Pf[idx] - ref).max() / Pf.max()


def test_range_update_and_prediction_match_quadrature():
    """The update matches the quadrature to the truncation of the Gaussian
    prior by the +-6 sigma box (~e^-18); the prediction converges to the
    closed-form moments and the Chapman-Kolmogorov density as the box grows:
    the range posterior's tails along the arc are heavier than the Gaussian
    the box is sized for (+-span sigma of the predicted covariance), so at
    span 6 the re-sized box drops ~1e-3 of its covariance, a property of the
    grid rule (shared by the GPU paths), not of the arithmetic."""
    post6, pred6, _ = _range_cycle_errors(6.0)
    assert post6[0] < 1e-8 and post6[1] < 1e-7, post6
    assert pred6[1] < 3e-3, pred6
    post10, pred10, d10 = _range_cycle_errors(10.0)
    post14, pred14, d14 = _range_cycle_errors(14.0)
    assert max(post10 + post14) < 1e-11, (post10, post14)
    assert pred14[0] < 3e-7 and pred14[1] < 1.5e-6 and d14 < 5e-8, (pred14, d14)
    assert pred10[1] > 20 * pred14[1] and d10 > 20 * d14, (pred10, pred14, d10, d14)


def test_range_pin_trips_on_planted_mistakes(monkeypatch):
    cfg, meas, z = _range_problem()
    x, wq = _range_nodes(cfg, z[0], 0.15)
    mq, Cq = _moments(x, wq)
    good_h = model.h

    def bad_h(kind, xx, H=None, params=None):      # |x| of the first coordinate twice
        if kind == "range":
            return np.sqrt(xx[:, 0] ** 2 + xx[:, 0] ** 2)[:, None]
        return good_h(kind, xx, H, params)
    monkeypatch.setattr(model, "h", bad_h)
    f = of.OracleFilter(cfg, psi_mode="exact")
    f.meas_update(meas, z)
    em, ec = _rel(*f.moments(), mq, Cq)
    assert max(em, ec) > 1e-2, (em, ec)


# --- bearing + linear x3 (n_x = 3) -------------------------------------------------

def _bearing_problem():
    """Prior near the +-pi cut of atan2 and a measured bearing written on the
    other side of it, so the wrap of the residual decides the likelihood; the
    prior sits 12 sigma from the sensor, where the bearing is singular."""
    P0 = np.array([[0.25, 0.05, 0.02], [0.05, 0.2, 0.03], [0.02, 0.03, 0.3]])
    rng = np.random.default_rng(1003)
    A = w.random_stable_matrix(3, rng)
    cfg = FilterConfig(nx=3, N=(64, 64, 64), A=A, Q=np.diag([0.2, 0.2, 0.1]),
                       m0=np.array([-6.0, 0.25, 0.3]), P0=P0)
    meas = MeasModel("bearing_linear3", R=np.diag([0.12 ** 2, 0.25 ** 2]))
    z = np.array([-np.pi + 0.05, 0.2])
    return cfg, meas, z


def _wrap(a):
    """Angle to (-pi, pi] through the complex exponential (independent of the oracle's formula)."""
    out = np.angle(np.exp(1j * a))
    return np.where(out == -np.pi, np.pi, out)


def _bearing_moments(cfg, z, sb, s3, nr=240, nth=1024, n3=96):
    """Cylindrical quadrature (r, theta, x3) of the bearing + linear posterior moments."""
    r0 = np.hypot(cfg.m0[0], cfg.m0[1])
    r, wr = _gl(r0 - 5.0, r0 + 5.0, nr)
    th = 2 * np.pi * np.arange(nth) / nth - np.pi
    x3, w3 = _gl(z[1] - 12 * s3, z[1] + 12 * s3, n3)      # the linear likelihood confines x3
    S0, S1, S2 = 0.0, np.zeros(3), np.zeros((3, 3))
    T_, X3 = np.meshgrid(th, x3, indexing="ij")
    W3 = np.broadcast_to(w3[None, :], T_.shape)
    for ri, wri in zip(r, wr):
        x = np.stack([(ri * np.cos(T_)).ravel(), (ri * np.sin(T_)).ravel(), X3.ravel()], axis=1)
        lik = np.exp(-0.5 * _wrap(z[0] - T_.ravel()) ** 2 / sb ** 2 - 0.5 * (z[1] - X3.ravel()) ** 2 / s3 ** 2)
        wq = wri * ri * (2 * np.pi / nth) * W3.ravel() * _gauss(x, cfg.m0, cfg.P0) * lik
        S0 += wq.sum()
        S1 += wq @ x
        S2 += (wq[:, None] * x).T @ x
    m = S1 / S0
    return m, S2 / S0 - np.outer(m, m)


def test_bearing_update_and_prediction_match_quadrature():
    cfg, meas, z = _bearing_problem()
    mq, Cq = _bearing_moments(cfg, z, 0.12, 0.25)
    f = of.OracleFilter(cfg, psi_mode="exact")
    f.meas_update(meas, z)
    em, ec = _rel(*f.moments(), mq, Cq)
    assert em < 2e-8 and ec < 2e-7, (em, ec)          # the +-6 sigma truncation of the prior
    tau = 0.1
    f.time_update(tau)
    Phi, Qd = _phi_qd(cfg.A, cfg.Q, tau)
    em, ec = _rel(*f.moments(), Phi @ mq, Phi @ Cq @ Phi.T + Qd)
    assert em < 2e-8 and ec < 2e-7, (em, ec)


@pytest.mark.parametrize("mistake", ["wrap", "no_wrap"])
def test_bearing_pin_trips_on_planted_mistakes(monkeypatch, mistake):
    cfg, meas, z = _bearing_problem()
    mq, Cq = _bearing_moments(cfg, z, 0.12, 0.25, nr=120, nth=512, n3=48)
    if mistake == "wrap":        # wrapped to [0, 2 pi) instead of (-pi, pi]
        monkeypatch.setattr(model, "wrap_angle", lambda r: np.mod(r, 2 * np.pi))
    else:
        monkeypatch.setattr(model, "wrap_angle", lambda r: r)
    f = of.OracleFilter(cfg, psi_mode="exact")
    try:
        f.meas_update(meas, z)
    except of.Degenerate:
        return
    em, ec = _rel(*f.moments(), mq, Cq)
    assert max(em, ec) > 1e-2, (em, ec)


# --- terrain altitude with Gaussian-mixture noise (n_x = 4, Sec. VI) ---------------

def _terrain_problem(N=(128, 16, 32, 16)):
    """The coordinated turn in prior-relative coordinates with a position-velocity
    correlated prior; the grid resolves the likelihood's bands along the two
    position axes (the velocities enter the likelihood only through the prior)."""
    sc = w.c6_scenario(N=N, epochs=2, local=True)
    P0 = np.array(sc.cfg.P0, dtype=float)
    P0[0, 1] = P0[1, 0] = 60.0
    sc.cfg.P0 = P0
    return sc


def _terrain_lik(params, z, px, py):
    """Mixture density of z - h(p), h restated from the model's definition."""
    p = np.asarray(params, dtype=float)
    h = p[16] + sum(p[4 * i] * np.sin(p[4 * i + 1] * px + p[4 * i + 2] * py + p[4 * i + 3]) for i in range(4))
    r = z - h
    g = lambda mu, v: np.exp(-0.5 * (r - mu) ** 2 / v) / np.sqrt(2 * np.pi * v)
    return p[17] * g(p[18], p[20]) + (1.0 - p[17]) * g(p[19], p[21])


def _terrain_moments(sc, z, n=(900, 500)):
    """Posterior moments: a Gauss-Legendre quadrature over the positions (x0, x2)
    with their Gaussian prior marginal, and the velocities by Gaussian
    conditioning on the positions (exact, the likelihood depends on p only)."""
    m0, P0 = np.asarray(sc.cfg.m0, float), np.asarray(sc.cfg.P0, float)
    ip, iv = [0, 2], [1, 3]
    Cpp, Cvp, Cvv = P0[np.ix_(ip, ip)], P0[np.ix_(iv, ip)], P0[np.ix_(iv, iv)]
    sd = np.sqrt(np.diag(Cpp))
    a, wa = _gl(m0[0] - 8 * sd[0], m0[0] + 8 * sd[0], n[0])
    b, wb = _gl(m0[2] - 8 * sd[1], m0[2] + 8 * sd[1], n[1])
    PX, PY = np.meshgrid(a, b, indexing="ij")
    pts = np.stack([PX.ravel(), PY.ravel()], axis=1)
    wq = np.outer(wa, wb).ravel() * _gauss(pts, m0[ip], Cpp) * _terrain_lik(sc.meas.params, z, pts[:, 0], pts[:, 1])
    mp, Cp = _moments(pts, wq)
    K = Cvp @ np.linalg.inv(Cpp)
    mv = m0[iv] + K @ (mp - m0[ip])
    Cv = Cvv - K @ Cvp.T + K @ Cp @ K.T
    m = np.zeros(4)
    C = np.zeros((4, 4))
    m[ip], m[iv] = mp, mv
    C[np.ix_(ip, ip)], C[np.ix_(iv, iv)] = Cp, Cv
    C[np.ix_(iv, ip)] = K @ Cp
    C[np.ix_(ip, iv)] = (K @ Cp).T
    return m, C


def test_terrain_update_matches_quadrature():
    """The Sec. VI measurement (terrain altitude, two-component mixture noise)
    on a position-velocity correlated Gaussian prior: every moment to the
    truncation of the prior by the +-6 sigma box.  The grid resolves the
    likelihood's bands along the positions (16 nodes per velocity axis keep
    the velocities' trapezoid sums exact)."""
    sc = _terrain_problem(N=(128, 16, 32, 16))
    mq, Cq = _terrain_moments(sc, float(sc.z[0][0]))
    f = of.OracleFilter(sc.cfg, psi_mode="exact")
    f.meas_update(sc.meas, sc.z[0])
    em, ec = _rel(*f.moments(), mq, Cq)
    assert em < 1e-8 and ec < 1e-6, (em, ec)


def test_terrain_pin_trips_on_a_planted_mistake(monkeypatch):
    """The terrain read at (p_x, v_x) instead of (p_x, p_y)."""
    sc = _terrain_problem(N=(96, 16, 24, 16))
    z = float(sc.z[0][0])
    mq, Cq = _terrain_moments(sc, z, n=(500, 300))
    good = model.h

    def bad(kind, x, H=None, params=None):
        if kind == "terrain_gm":
            return model.terrain(params, x[:, 0], x[:, 1])[:, None]
        return good(kind, x, H, params)
    monkeypatch.setattr(model, "h", bad)
    f = of.OracleFilter(sc.cfg, psi_mode="exact")
    try:
        f.meas_update(sc.meas, sc.z[0])
    except of.Degenerate:
        return
    em, ec = _rel(*f.moments(), mq, Cq)
    assert max(em, ec) > 1e-2, (em, ec)
