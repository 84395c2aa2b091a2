"""GPU parity of the 3-D tensor-core pipelines against the float64 oracle.

Cases: non-cubic grids whose axis-0 line tiles are ragged (N2/2 + 1 not a
multiple of 32), the bearing + linear measurement, a linear 3-D model with a
sheared frame, the exact-in-time multiplier, and the full 96^3 workload.  Bar: FP16X3 relative L1 <= 1e-5.
"""
import numpy as np
import pytest

import workloads as w
from tests._parity import max_errors

pytestmark = pytest.mark.gpu


def _check(worst, bar=1e-5):
    assert worst["l1"] <= bar, worst
    assert worst["frame"] <= bar, worst
    assert worst["mean"] <= bar and worst["cov"] <= 10 * bar, worst


@pytest.mark.parametrize("N", [(16, 32, 48), (32, 48, 80)])
def test_small_3d_bearing_fp16x3(N):
    worst, _ = max_errors(w.small_3d_scenario(N=N, epochs=3), precision="fp16x3")
    print(N, worst)
    _check(worst)


def test_3d_linear_fp16x3():
    from workloads import FilterConfig, MeasModel, Scenario, simulate
    rng = np.random.default_rng(21)
    A = w.random_stable_matrix(3, rng)
    cfg = FilterConfig(nx=3, N=(32, 32, 48), A=A, Q=np.diag([0.2, 0.1, 0.15]),
                       m0=np.array([0.5, -0.2, 0.1]), P0=np.array([[0.3, 0.1, 0.0], [0.1, 0.25, 0.05],
                                                                   [0.0, 0.05, 0.2]]))
    meas = MeasModel("linear", R=0.3 ** 2 * np.eye(3), H=np.eye(3))
    sc = Scenario("lin3", cfg, meas, dt=0.1, epochs=3)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=22)
    worst, _ = max_errors(sc, precision="fp16x3")
    _check(worst)


def test_3d_exact_multiplier_fp16x3():
    # the exact-in-time multiplier on the 8-point orbits (cross terms of both signs)
    worst, _ = max_errors(w.small_3d_scenario(N=(32, 48, 80), epochs=3), precision="fp16x3", psi_mode="exact")
    _check(worst)


def test_c3_full_size_two_epochs():
    worst, _ = max_errors(w.c3_scenario(epochs=2), precision="fp16x3")
    print(worst)
    _check(worst)


def test_far_measurement_tiny_slices_fp16x3():
    """A measurement ~2 sigma off the prior leaves 3-D slices with only denormal
    weights; their per-slice operand scale must stay finite."""
    from workloads import FilterConfig, MeasModel, Scenario
    cfg = FilterConfig(nx=3, N=(32, 32, 32), A=np.zeros((3, 3)), Q=np.diag([0.2, 0.1, 0.15]),
                       m0=np.array([0.5, -0.2, 0.1]), P0=0.25 * np.eye(3))
    meas = MeasModel("linear", R=0.09 * np.eye(3), H=np.eye(3))
    sc = Scenario("far", cfg, meas, dt=0.1, epochs=2)
    sc.z = np.array([[-0.386, -0.368, -1.032], [-0.5, -0.4, -1.1]])
    worst, _ = max_errors(sc, precision="fp16x3")
    _check(worst)


def test_repeatable_bitwise():
    # two filters fed the same inputs agree bit for bit (self-mirrored
    # frequency lines are written back once, by one thread)
    from paper_2412_07240_gb300 import Filter
    wl = w.c5_serving(n_filters=40, rate=8000.0, duration=0.05, seed=7, n1=(16, 96), n2=(16, 48), n3=(16, 32))
    f = next(i for i, c in enumerate(wl.cfgs) if c.nx == 3)
    outs = []
    for _ in range(2):
        g = Filter(wl.cfgs[f], precision="fp16x3")
        for k in range(3):
            g.step(wl.meas[f], wl.z[k, :3] * 0 + wl.cfgs[f].m0, 0.1)
        outs.append(g.pdf())
        g.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])


@pytest.mark.parametrize("prec,bar", [("bf16x3", 1e-4), ("tf32", 3e-2)])
def test_small_3d_bearing_other_precisions(prec, bar):
    """The 3-D pipelines in the other operand formats (bars as for 2-D: BF16X3
    keeps ~16 bits of each operand, TF32 ~11)."""
    worst, _ = max_errors(w.small_3d_scenario(N=(16, 32, 48), epochs=3), precision=prec)
    assert worst["l1"] <= bar, worst
    assert worst["mean"] <= bar, worst


def test_3d_shear_realignment_fp16x3():
    """Band-limited re-alignment in the 3-D pipelines (three batched line-wise
    passes in float32) against the oracle's passes."""
    from tests.test_gpu_fp64 import _cv3
    worst, log = max_errors(_cv3("shear", N=(32, 32, 16)), precision="fp16x3")
    assert sum(s.endswith("R") for s, _ in log) >= 2, "re-alignment not exercised"
    _check(worst)
