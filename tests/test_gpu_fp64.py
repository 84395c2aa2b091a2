"""GPU parity of the plain float64 path against the float64 oracle (bar: relative L1 <= 1e-12).

Both sides run the same seeded inputs update by update; the CUDA path is
called through the C-ABI binding.  Cases span 1-D, 2-D (range, linear with
re-alignment) and 3-D (bearing) grids, both diffusion multipliers, ragged
(non-square, non-power-of-two) sizes and the smallest even grid.
"""
import numpy as np
import pytest

import workloads as w
from tests._parity import max_errors
from workloads import FilterConfig, MeasModel, Scenario, simulate

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _check(worst, tol=TOL):
    assert worst["l1"] <= tol, worst
    assert worst["frame"] <= tol, worst
    assert worst["mean"] <= tol and worst["cov"] <= 10 * tol, worst


def test_c1_full_run():
    worst, log = max_errors(w.c1_scenario())
    _check(worst)


def test_c1_exact_multiplier():
    worst, _ = max_errors(w.c1_scenario(epochs=8), psi_mode="exact")
    _check(worst)


def test_small_2d_range_ragged():
    worst, _ = max_errors(w.small_2d_scenario(N=(48, 40), epochs=5))
    _check(worst)


def test_2d_realignment_path():
    cfg = FilterConfig(nx=2, N=(40, 48), A=np.array([[0.0, 1.0], [0.0, 0.0]]), Q=np.diag([0.01, 0.1]),
                       m0=np.array([0.0, 1.0]), P0=np.diag([0.5, 0.5]))
    meas = MeasModel("linear", R=np.array([[0.3 ** 2]]), H=np.array([[1.0, 0.0]]))
    sc = Scenario("cv", cfg, meas, dt=0.2, epochs=6)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=11)
    worst, log = max_errors(sc)
    assert any(s.endswith("R") for s, _ in log), "re-alignment not exercised"
    _check(worst, 1e-11)


def test_small_3d_bearing():
    worst, _ = max_errors(w.small_3d_scenario(N=(16, 24, 20), epochs=3))
    _check(worst)


def test_minimal_grid_n4():
    """Four nodes: the posterior collapses onto about one node, so its variance is a
    cancellation of O(1) sums; weights and frame are compared, not the moments."""
    sc = w.c1_scenario(N=4, epochs=3)
    worst, _ = max_errors(sc)
    assert worst["l1"] <= 1e-11 and worst["frame"] <= 1e-11, worst


def test_c2_full_size_first_epochs():
    worst, _ = max_errors(w.c2_scenario(epochs=4))
    _check(worst)


def test_invalid_measurement_rejected():
    from paper_2412_07240_gb300 import Filter, PmfError
    sc = w.c1_scenario()
    f = Filter(sc.cfg)
    with pytest.raises(PmfError):
        f.meas_update(sc.meas, np.array([np.nan]))
    m0, _ = f.moments()
    assert np.all(np.isfinite(m0))


def test_2d_shear_realignment_path():
    cfg = FilterConfig(nx=2, N=(40, 48), A=np.array([[0.0, 1.0], [0.0, 0.0]]), Q=np.diag([0.01, 0.1]),
                       m0=np.array([0.0, 1.0]), P0=np.diag([0.5, 0.5]), realign_mode="shear")
    meas = MeasModel("linear", R=np.array([[0.3 ** 2]]), H=np.array([[1.0, 0.0]]))
    sc = Scenario("cv", cfg, meas, dt=0.2, epochs=6)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=11)
    worst, log = max_errors(sc)
    assert any(s.endswith("R") for s, _ in log), "re-alignment not exercised"
    _check(worst, 1e-11)


def _cv3(mode, N=(20, 24, 16), epochs=6):
    A = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.3, -0.5]])
    cfg = FilterConfig(nx=3, N=N, A=A, Q=np.diag([0.01, 0.1, 0.05]), m0=np.array([0.0, 1.0, 0.5]),
                       P0=np.diag([0.5, 0.5, 0.3]), realign_mode=mode)
    meas = MeasModel("linear", R=np.diag([0.3 ** 2, 0.4 ** 2]), H=np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]]))
    sc = Scenario("cv3", cfg, meas, dt=0.2, epochs=epochs)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=12)
    return sc


def test_3d_shear_realignment_path():
    """Band-limited re-alignment in 3-D: three line-wise passes on the float64 path."""
    worst, log = max_errors(_cv3("shear"))
    assert sum(s.endswith("R") for s, _ in log) >= 2, "re-alignment not exercised"
    _check(worst, 1e-11)

