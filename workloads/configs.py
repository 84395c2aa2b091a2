"""Workload definitions and seeded generators.

Model (Sec. I, eqs. dynam/meas): dx = A x dt + Q dw with E[dw dw^T] = I dt,
read as Q being the diffusion (covariance-rate) matrix, and z_k = h(x_k) + v_k.

The five workloads follow the model statement of the paper and the sizes of
the benchmark configurations:

* C1: n_x = 1, A = -0.5, Q = 0.5, prior N(1, 0.5^2), 64 points spanning
  +-6 sigma, linear z = x + v with v ~ N(0, 0.1^2), 20 epochs at dt = 0.1.
* C2: n_x = 2 damped oscillator, A = [[0, 1], [-1, -0.2]], Q = diag(0.1, 0.3),
  128 x 128 grid, prior N((2, 0), 0.25 I), range measurement with
  v ~ N(0, 0.05^2), 50 epochs at dt = 0.05.
* C3: n_x = 3, seeded random stable A (real eigenvalues in [-1, -0.1]),
  Q = diag(0.2, 0.2, 0.1), 96^3 grid, prior N((3, 1, 0), 0.25 I), bearing
  atan2(x2, x1) plus linear x3 with v ~ N(0, diag(0.02^2, 0.1^2)), 30 epochs
  at dt = 0.1.
* C4: 4096 independent n_x = 2 filters, each with its own seeded stable A,
  diagonal Q in [0.05, 0.5], axis sizes drawn from {32, 48, 64, 96, 128},
  linear z = x + v with R = 0.1^2 I, 100 epochs at dt = 0.05.

Truth trajectories are integrated with Euler-Maruyama on a fine step
(``fine`` sub-steps per epoch); this is input simulation, independent of how
the filter discretises the model.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

MEAS_KINDS = ("linear", "range", "bearing_linear3")


@dataclass
class FilterConfig:
    """Model and grid of one filter.

    N[m] is the number of grid points along axis m (even).  ``span`` is the
    half-width of the grid in standard deviations, ``dt_sub`` the Euler
    sub-step bound (l = ceil(dt / dt_sub) sub-steps per time update) and
    ``realign_rho`` the whitened-correlation threshold above which the grid
    frame is re-aligned to the predicted covariance, ``realign_mode`` how the
    re-aligned frame is filled ("multilinear", or "shear" for n_x = 2).
    """
    nx: int
    N: tuple
    A: np.ndarray
    Q: np.ndarray
    m0: np.ndarray
    P0: np.ndarray
    span: float = 6.0
    dt_sub: float = 0.01
    realign_rho: float = 0.5
    realign_mode: str = "multilinear"


@dataclass
class MeasModel:
    """Measurement model z = h(x) + v, v ~ N(0, R).

    kind: 'linear' (h = H x), 'range' (h = |x_{1:2}|), 'bearing_linear3'
    (h = [atan2(x2, x1), x3]) or 'terrain_gm' (n_x = 4, state [p_x, v_x, p_y,
    v_y]: a smooth terrain altitude under the position, two-component Gaussian
    mixture noise; ``params`` holds the terrain and mixture constants in the
    layout of pmf_meas.p, and R is the mixture's covariance for reference).
    """
    kind: str
    R: np.ndarray
    H: Optional[np.ndarray] = None
    params: Optional[np.ndarray] = None

    @property
    def nz(self) -> int:
        return self.R.shape[0]


@dataclass
class Scenario:
    name: str
    cfg: FilterConfig
    meas: MeasModel
    dt: float
    epochs: int
    truth: np.ndarray = field(default=None)
    z: np.ndarray = field(default=None)


def _h_true(meas: MeasModel, x: np.ndarray) -> np.ndarray:
    """Noise-free measurement of a true state (input simulation only)."""
    if meas.kind == "linear":
        return meas.H @ x
    if meas.kind == "range":
        return np.array([np.hypot(x[0], x[1])])
    if meas.kind == "bearing_linear3":
        return np.array([np.arctan2(x[1], x[0]), x[2]])
    raise ValueError(meas.kind)


def _psd_sqrt(S: np.ndarray) -> np.ndarray:
    """A square root L with L L^T = S for a symmetric PSD matrix."""
    w, V = np.linalg.eigh(0.5 * (S + S.T))
    return V * np.sqrt(np.clip(w, 0.0, None))


def simulate(cfg: FilterConfig, meas: MeasModel, dt: float, epochs: int,
             seed: int, fine: int = 200):
    """Seeded truth x_0..x_{K-1} and measurements z_0..z_{K-1}.

    x_0 ~ N(m0, P0); between epochs the SDE is integrated by Euler-Maruyama
    with ``fine`` steps; z_k = h(x_k) + v_k.
    """
    rng = np.random.default_rng(seed)
    n = cfg.nx
    Lp = np.linalg.cholesky(cfg.P0)
    Lq = _psd_sqrt(cfg.Q)
    Lr = np.linalg.cholesky(meas.R)
    x = cfg.m0 + Lp @ rng.standard_normal(n)
    h = dt / fine
    xs, zs = [], []
    for k in range(epochs):
        if k > 0:
            for _ in range(fine):
                x = x + h * (cfg.A @ x) + np.sqrt(h) * (Lq @ rng.standard_normal(n))
        xs.append(x.copy())
        zs.append(_h_true(meas, x) + Lr @ rng.standard_normal(meas.nz))
    return np.array(xs), np.array(zs)


def random_stable_matrix(n: int, rng, re_lo: float = -1.0, re_hi: float = -0.1,
                         complex_pairs: bool = False, max_cond: float = 10.0):
    """Seeded stable drift A = V diag-block(Lambda) V^{-1}.

    Eigenvalues (or real parts of complex pairs) are uniform in
    [re_lo, re_hi]; V is redrawn until cond(V) <= max_cond.
    """
    while True:
        V = rng.standard_normal((n, n))
        if np.linalg.cond(V) <= max_cond:
            break
    B = np.zeros((n, n))
    i = 0
    while i < n:
        a = rng.uniform(re_lo, re_hi)
        if complex_pairs and i + 1 < n and rng.uniform() < 0.5:
            b = rng.uniform(0.2, 2.0)
            B[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
            i += 2
        else:
            B[i, i] = a
            i += 1
    return V @ B @ np.linalg.inv(V)


def c1_scenario(seed: int = 1, epochs: int = 20, N: int = 64) -> Scenario:
    cfg = FilterConfig(nx=1, N=(N,), A=np.array([[-0.5]]), Q=np.array([[0.5]]),
                       m0=np.array([1.0]), P0=np.array([[0.25]]))
    meas = MeasModel("linear", R=np.array([[0.01]]), H=np.array([[1.0]]))
    sc = Scenario("c1_1d_n64", cfg, meas, dt=0.1, epochs=epochs)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, epochs, seed)
    return sc


def c2_scenario(seed: int = 2, epochs: int = 50, N=(128, 128)) -> Scenario:
    cfg = FilterConfig(nx=2, N=tuple(N), A=np.array([[0.0, 1.0], [-1.0, -0.2]]),
                       Q=np.diag([0.1, 0.3]), m0=np.array([2.0, 0.0]),
                       P0=np.diag([0.25, 0.25]))
    meas = MeasModel("range", R=np.array([[0.05 ** 2]]))
    sc = Scenario("c2_2d_osc_128x128", cfg, meas, dt=0.05, epochs=epochs)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, epochs, seed)
    return sc


def c3_scenario(seed: int = 3, epochs: int = 30, N=(96, 96, 96)) -> Scenario:
    rng = np.random.default_rng(1000 + seed)
    A = random_stable_matrix(3, rng)
    cfg = FilterConfig(nx=3, N=tuple(N), A=A, Q=np.diag([0.2, 0.2, 0.1]),
                       m0=np.array([3.0, 1.0, 0.0]), P0=0.25 * np.eye(3))
    meas = MeasModel("bearing_linear3", R=np.diag([0.02 ** 2, 0.1 ** 2]))
    sc = Scenario("c3_3d_96cube", cfg, meas, dt=0.1, epochs=epochs)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, epochs, seed)
    return sc


def small_2d_scenario(seed: int = 5, epochs: int = 6, N=(48, 32),
                      kind: str = "range") -> Scenario:
    """A reduced C2-like problem for parity tests that finish in seconds."""
    sc = c2_scenario(seed=seed, epochs=epochs, N=N)
    if kind == "linear":
        sc.meas = MeasModel("linear", R=0.1 ** 2 * np.eye(2), H=np.eye(2))
        sc.truth, sc.z = simulate(sc.cfg, sc.meas, sc.dt, epochs, seed)
    sc.name = f"small_2d_{N[0]}x{N[1]}_{kind}"
    return sc


def small_3d_scenario(seed: int = 6, epochs: int = 3, N=(16, 24, 32)) -> Scenario:
    """A reduced C3-like problem for parity tests that finish in seconds."""
    sc = c3_scenario(seed=seed, epochs=epochs, N=N)
    sc.name = f"small_3d_{N[0]}x{N[1]}x{N[2]}"
    return sc


def c4_batch(count: int = 4096, seed: int = 4, epochs: int = 100,
             sizes=(32, 48, 64, 96, 128), fine: int = 20):
    """C4: independent n_x = 2 filters with their own stable A and diagonal Q.

    Returns (configs, meas, dt, truth, z): a list of FilterConfig, the shared
    measurement model, the epoch spacing, truth of shape (count, epochs, 2)
    and measurements of shape (count, epochs, 2).  Axis sizes are drawn
    independently and uniformly from ``sizes``; priors have mean ~ N(0, I)
    and covariance 0.25 I; z = x + v with R = 0.1^2 I.
    """
    rng = np.random.default_rng(seed)
    meas = MeasModel("linear", R=0.1 ** 2 * np.eye(2), H=np.eye(2))
    dt = 0.05
    cfgs = []
    for _ in range(count):
        A = random_stable_matrix(2, rng, complex_pairs=True)
        Q = np.diag(rng.uniform(0.05, 0.5, size=2))
        N = tuple(int(s) for s in rng.choice(sizes, size=2))
        m0 = rng.standard_normal(2)
        cfgs.append(FilterConfig(nx=2, N=N, A=A, Q=Q, m0=m0, P0=0.25 * np.eye(2)))
    As = np.stack([c.A for c in cfgs])
    sq = np.stack([np.sqrt(np.diag(c.Q)) for c in cfgs])
    x = np.stack([c.m0 for c in cfgs]) + 0.5 * rng.standard_normal((count, 2))
    h = dt / fine
    truth = np.empty((count, epochs, 2))
    z = np.empty((count, epochs, 2))
    for k in range(epochs):
        if k > 0:
            for _ in range(fine):
                x = x + h * np.einsum("fij,fj->fi", As, x) \
                    + np.sqrt(h) * sq * rng.standard_normal((count, 2))
        truth[:, k] = x
        z[:, k] = x + 0.1 * rng.standard_normal((count, 2))
    return cfgs, meas, dt, truth, z


def _expm_batch(X: np.ndarray) -> np.ndarray:
    """Matrix exponentials of a stack (k, m, m): Taylor series after scaling
    by 2^-s (1-norm <= 1/4), then s squarings (input simulation only)."""
    k, m, _ = X.shape
    if k == 0:
        return X.copy()
    nrm = np.abs(X).sum(axis=1).max(axis=1)
    s = np.maximum(0, np.ceil(np.log2(np.maximum(nrm, 1e-300) / 0.25))).astype(int)
    Y = X / (2.0 ** s)[:, None, None]
    E = np.broadcast_to(np.eye(m), X.shape).copy()
    T = E.copy()
    for j in range(1, 19):
        T = T @ Y / j
        E = E + T
    for j in range(int(s.max())):
        sel = s > j
        E[sel] = E[sel] @ E[sel]
    return E


@dataclass
class ServingWorkload:
    """Resident filters and a request log replayed in real time.

    Request i arrives at t_arrival[i] (seconds, ascending) for filter ids[i]:
    measurement z[i] (nx values, zero-padded to 3) of the filter's truth at its
    current model time, then a time update over taus[i], the time to the
    filter's next measurement.
    """
    cfgs: list
    meas: list
    t_arrival: np.ndarray
    ids: np.ndarray
    z: np.ndarray
    taus: np.ndarray
    truth: list = field(default_factory=list)


def c5_serving(n_filters: int = 10000, rate: float = 200e3, duration: float = 60.0, seed: int = 5,
               frac=(0.6, 0.35, 0.05), n1=(64, 512), n2=(32, 128), n3=(32, 64),
               tau_mean: float = 0.1) -> ServingWorkload:
    """C5: 60% n_x = 1 filters with N in [64, 512] (multiples of 8), 35% n_x = 2
    with each axis in [32, 128] (multiples of 16, the tensor-core tile), 5%
    n_x = 3 with each axis in [32, 64] (multiples of 16); each with its own
    seeded stable A, diagonal Q in [0.05, 0.5], prior N(m0 ~ N(0, I), 0.25 I)
    and z = x + v, R = 0.1^2 I.  Requests arrive as a Poisson process of the
    given aggregate rate for ``duration`` seconds, each for a uniformly drawn
    filter, with the time to that filter's next measurement drawn from an
    exponential distribution of mean ``tau_mean``.  The truth advances by the
    exact discretisation x <- e^{A tau} x + w, w ~ N(0, Q_d(tau)).
    """
    rng = np.random.default_rng(seed)
    counts = [int(round(frac[0] * n_filters)), int(round(frac[1] * n_filters))]
    counts.append(n_filters - counts[0] - counts[1])
    grids = {1: np.arange(n1[0], n1[1] + 1, 8), 2: np.arange(n2[0], n2[1] + 1, 16),
             3: np.arange(n3[0], n3[1] + 1, 16)}
    cfgs, meas = [], []
    for nx, cnt in zip((1, 2, 3), counts):
        for _ in range(cnt):
            if nx == 1:
                A = np.array([[rng.uniform(-1.0, -0.1)]])
            else:
                A = random_stable_matrix(nx, rng, complex_pairs=(nx == 2))
            Q = np.diag(rng.uniform(0.05, 0.5, size=nx))
            N = tuple(int(v) for v in rng.choice(grids[nx], size=nx))
            cfgs.append(FilterConfig(nx=nx, N=N, A=A, Q=Q, m0=rng.standard_normal(nx), P0=0.25 * np.eye(nx)))
            meas.append(MeasModel("linear", R=0.1 ** 2 * np.eye(nx), H=np.eye(nx)))
    n_req = int(rng.poisson(rate * duration))
    t_arrival = np.sort(rng.uniform(0.0, duration, size=n_req))
    ids = rng.integers(0, n_filters, size=n_req).astype(np.int32)
    taus = rng.exponential(tau_mean, size=n_req)
    z = np.zeros((n_req, 3))
    # truth per filter, advanced request by request ("round" k = k-th request of each filter)
    order = np.argsort(ids, kind="stable")
    first = np.searchsorted(ids[order], np.arange(n_filters))
    rank = np.empty(n_req, dtype=np.int64)
    rank[order] = np.arange(n_req) - first[ids[order]]
    nxs = np.array([c.nx for c in cfgs])
    x = [cfgs[f].m0 + 0.5 * rng.standard_normal(cfgs[f].nx) for f in range(n_filters)]
    X = {d: np.array([x[f] for f in range(n_filters) if nxs[f] == d]).reshape(-1, d) for d in (1, 2, 3)}
    pos = np.zeros(n_filters, dtype=np.int64)
    for d in (1, 2, 3):
        pos[nxs == d] = np.arange((nxs == d).sum())
    As = {d: np.array([cfgs[f].A for f in range(n_filters) if nxs[f] == d]).reshape(-1, d, d) for d in (1, 2, 3)}
    Qs = {d: np.array([cfgs[f].Q for f in range(n_filters) if nxs[f] == d]).reshape(-1, d, d) for d in (1, 2, 3)}
    by_rank = np.argsort(rank, kind="stable")
    bounds = np.searchsorted(rank[by_rank], np.arange(int(rank.max(initial=-1)) + 2))
    for k in range(len(bounds) - 1):
        req = by_rank[bounds[k]:bounds[k + 1]]
        for d in (1, 2, 3):
            r = req[nxs[ids[req]] == d]
            if r.size == 0:
                continue
            p = pos[ids[r]]
            z[r, :d] = X[d][p] + 0.1 * rng.standard_normal((r.size, d))
            A = As[d][p]
            tau = taus[r][:, None, None]
            m = 2 * d
            C = np.zeros((r.size, m, m))
            C[:, :d, :d] = -A * tau
            C[:, :d, d:] = Qs[d][p] * tau
            C[:, d:, d:] = np.transpose(A, (0, 2, 1)) * tau
            E = _expm_batch(C)
            Phi = np.transpose(E[:, d:, d:], (0, 2, 1))
            Qd = Phi @ E[:, :d, d:]
            Qd = 0.5 * (Qd + np.transpose(Qd, (0, 2, 1)))
            w, V = np.linalg.eigh(Qd)
            L = V * np.sqrt(np.maximum(w, 0.0))[:, None, :]
            X[d][p] = np.einsum("kij,kj->ki", Phi, X[d][p]) + np.einsum("kij,kj->ki", L, rng.standard_normal((r.size, d)))
    return ServingWorkload(cfgs, meas, t_arrival, ids, z, taus)


def terrain_params(seed: int = 6) -> np.ndarray:
    """Seeded smooth terrain and the Sec. VI noise mixture, in the pmf_meas.p
    layout: four plane waves (amplitude 20-60 m, wavelength 300-1500 m, random
    direction and phase) on a 500 m base; mixture weights 1/2, 1/2, means 0 and
    20 m, unit variances.  Stands in for the paper's terrain map, which is not
    available."""
    rng = np.random.default_rng(1000 + seed)
    p = np.zeros(24)
    for i in range(4):
        amp, lam, th = rng.uniform(20.0, 60.0), rng.uniform(300.0, 1500.0), rng.uniform(0.0, 2 * np.pi)
        k = 2 * np.pi / lam
        p[4 * i:4 * i + 4] = [amp, k * np.cos(th), k * np.sin(th), rng.uniform(0.0, 2 * np.pi)]
    p[16] = 500.0
    p[17:22] = [0.5, 0.0, 20.0, 1.0, 1.0]
    return p


def c6_scenario(seed: int = 6, epochs: int = 20, N=34, dt_sub: float = 0.05,
                terrain_seed: int = 6, local: bool = False) -> Scenario:
    """The paper's numerical illustration (Sec. VI): coordinated turn with known
    turn rate alpha = 30 deg/s, state [p_x, v_x, p_y, v_y], diffusion on the
    velocity axes only (Q = diag(0, 1, 0, 1)), prior N([36569, 50, 55581, 50],
    diag(90, 160, 5, 5)), sampling period 1 s, N_pa = 34 points per axis;
    terrain-altitude measurement with two-component Gaussian-mixture noise
    (synthetic terrain, see terrain_params; one terrain shared by every seed
    of the trajectory).  The truth advances by the exact discretisation
    x <- e^{A T} x + w, w ~ N(0, Q_d(T)).

    local=True states the same problem in positions relative to the prior mean
    (the terrain's wave phases absorb the offset), so that grid coordinates are
    O(100) m instead of O(50 km)."""
    rng = np.random.default_rng(600 + seed)
    a = np.deg2rad(30.0)
    A = np.array([[0.0, 1.0, 0.0, 0.0], [0.0, 0.0, 0.0, -a], [0.0, 0.0, 0.0, 1.0], [0.0, a, 0.0, 0.0]])
    Q = np.diag([0.0, 1.0, 0.0, 1.0])
    m0 = np.array([36569.0, 50.0, 55581.0, 50.0])
    P0 = np.diag([90.0, 160.0, 5.0, 5.0])
    Ns = tuple(int(v) for v in (N if np.ndim(N) else (N,) * 4))
    cfg = FilterConfig(nx=4, N=Ns, A=A, Q=Q, m0=m0, P0=P0, dt_sub=dt_sub)
    params = terrain_params(terrain_seed)
    meas = MeasModel("terrain_gm", R=np.array([[1.0]]), params=params)
    sc = Scenario("c6_4d_coordinated_turn", cfg, meas, dt=1.0, epochs=epochs)
    C = np.zeros((1, 8, 8))
    C[0, :4, :4] = -A * sc.dt
    C[0, :4, 4:] = Q * sc.dt
    C[0, 4:, 4:] = A.T * sc.dt
    E = _expm_batch(C)[0]
    Phi = E[4:, 4:].T
    Qd = Phi @ E[:4, 4:]
    w_, V_ = np.linalg.eigh(0.5 * (Qd + Qd.T))
    Lq = V_ * np.sqrt(np.maximum(w_, 0.0))[None, :]
    x = m0 + np.linalg.cholesky(P0) @ rng.standard_normal(4)
    truth, z = [], []
    for _ in range(epochs):
        comp = rng.uniform() >= params[17]
        v = params[19 if comp else 18] + np.sqrt(params[21 if comp else 20]) * rng.standard_normal()
        alt = params[16] + sum(params[4 * i] * np.sin(params[4 * i + 1] * x[0] + params[4 * i + 2] * x[2]
                                                      + params[4 * i + 3]) for i in range(4))
        truth.append(x.copy())
        z.append(np.array([alt + v]))
        x = Phi @ x + Lq @ rng.standard_normal(4)
    sc.truth, sc.z = np.array(truth), np.array(z)
    if local:
        o = np.array([m0[0], 0.0, m0[2], 0.0])
        p = params.copy()
        for i in range(4):
            p[4 * i + 3] = np.mod(p[4 * i + 3] + p[4 * i + 1] * o[0] + p[4 * i + 2] * o[2], 2 * np.pi)
        sc.cfg.m0 = m0 - o
        sc.meas = MeasModel("terrain_gm", R=np.array([[1.0]]), params=p)
        sc.truth = sc.truth - o[None, :]
        sc.name = "c6_4d_coordinated_turn_local"
    return sc
