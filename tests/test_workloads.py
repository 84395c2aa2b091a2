"""Seeded input generators: the serving workload has the composition, sizes
and arrival statistics it states."""
import numpy as np

import workloads as w


def test_c5_composition_and_sizes():
    wl = w.c5_serving(n_filters=2000, rate=50e3, duration=1.0, seed=11)
    nx = np.array([c.nx for c in wl.cfgs])
    assert np.bincount(nx, minlength=4)[1:].tolist() == [1200, 700, 100]
    for c in wl.cfgs:
        N = np.array(c.N)
        if c.nx == 1:
            assert 64 <= N[0] <= 512 and N[0] % 8 == 0
        elif c.nx == 2:
            assert np.all((32 <= N) & (N <= 128) & (N % 16 == 0))
        else:
            assert np.all((32 <= N) & (N <= 64) & (N % 16 == 0))
        assert np.all(np.linalg.eigvals(c.A).real < 0)


def test_c5_arrivals_and_horizons():
    wl = w.c5_serving(n_filters=500, rate=40e3, duration=2.0, seed=12)
    n = wl.ids.size
    assert abs(n - 80e3) < 5 * np.sqrt(80e3)            # Poisson count
    assert np.all(np.diff(wl.t_arrival) >= 0) and wl.t_arrival[-1] <= 2.0
    gaps = np.diff(wl.t_arrival)
    assert abs(gaps.mean() * 40e3 - 1.0) < 0.02           # exponential gaps of mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.03
    assert abs(wl.taus.mean() - 0.1) < 0.003
    nx = np.array([c.nx for c in wl.cfgs])[wl.ids]
    assert np.all(wl.z[nx == 1, 1:] == 0) and np.all(wl.z[nx == 2, 2] == 0)


def test_c5_truth_is_the_exact_discretisation():
    # a 1-D filter's measurements: z_{k+1} - e^{a tau_k} z_k has variance
    # Q_d(tau_k) + (1 + e^{2 a tau_k}) R on average
    wl = w.c5_serving(n_filters=10, rate=20e3, duration=2.0, seed=13, frac=(1.0, 0.0, 0.0))
    res, var = [], []
    for f, c in enumerate(wl.cfgs):
        r = np.nonzero(wl.ids == f)[0]
        a, q = c.A[0, 0], c.Q[0, 0]
        e = np.exp(a * wl.taus[r[:-1]])
        res.append(wl.z[r[1:], 0] - e * wl.z[r[:-1], 0])
        var.append(q * (np.exp(2 * a * wl.taus[r[:-1]]) - 1) / (2 * a) + (1 + e ** 2) * 0.01)
    res, var = np.concatenate(res), np.concatenate(var)
    assert abs(np.mean(res ** 2 / var) - 1.0) < 0.05


def test_c6_local_coordinates_state_the_same_problem():
    """The local form shifts positions by the prior mean and moves the offset into
    the terrain phases: same altitudes at the same physical points, same z."""
    from oracle import model
    a = w.c6_scenario(epochs=5)
    b = w.c6_scenario(epochs=5, local=True)
    np.testing.assert_array_equal(a.z, b.z)
    ha = model.h("terrain_gm", a.truth, params=a.meas.params)
    hb = model.h("terrain_gm", b.truth, params=b.meas.params)
    np.testing.assert_allclose(hb, ha, rtol=0, atol=1e-9)
    np.testing.assert_allclose(b.truth + np.array([36569.0, 0, 55581.0, 0]), a.truth, rtol=1e-15)
    assert np.allclose(b.cfg.m0, [0.0, 50.0, 0.0, 50.0])
