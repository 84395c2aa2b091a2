"""Edge cases of the update calls on every path, against the float64 oracle:
zero horizons, measurement-only steps, repeated measurement updates, a
horizon of exactly one sub-step, and the largest grids per axis."""
import numpy as np
import pytest

import workloads as w
from oracle.filter import OracleFilter
from tests._parity import check_own_decisions, compare, displacement_bound, max_errors

pytestmark = pytest.mark.gpu

# (scenario, precision, bar) per path: float64, fused 2-D, 1-D, 3-D pipelines, float32 4-D
PATHS = [
    (lambda: w.small_2d_scenario(N=(32, 48), epochs=3), "fp64", 1e-12),
    (lambda: w.small_2d_scenario(N=(32, 48), epochs=3), "fp16x3", 1e-5),
    (lambda: w.c1_scenario(N=64, epochs=3), "fp16x3", 1e-5),
    (lambda: w.small_3d_scenario(N=(16, 32, 16), epochs=3), "fp16x3", 1e-5),
    (lambda: w.c6_scenario(N=(10, 8, 12, 8), epochs=3, local=True), "fp16x3", 1e-5),
]
IDS = ["fp64-2d", "fused-2d", "1d", "3d", "4d-f32"]


@pytest.mark.parametrize("make,prec,bar", PATHS, ids=IDS)
def test_zero_horizon_and_measurement_only_steps(make, prec, bar):
    """tau = 0 leaves the weights as they are; a step with tau = 0 is the
    measurement update alone; two measurement updates in a row compose."""
    from paper_2412_07240_gb300 import Filter
    sc = make()
    gpu = Filter(sc.cfg, precision=prec)
    orc = OracleFilter(sc.cfg)
    P0 = gpu.pdf()[0]
    gpu.time_update(0.0)
    assert np.array_equal(gpu.pdf()[0], P0)
    gpu.step(sc.meas, sc.z[0], 0.0)
    orc.meas_update(sc.meas, sc.z[0])
    e = compare(gpu, orc)
    assert e["l1"] <= bar and e["frame"] <= bar, e
    gpu.meas_update(sc.meas, sc.z[1])
    orc.meas_update(sc.meas, sc.z[1])
    e = compare(gpu, orc)
    assert e["l1"] <= bar and e["frame"] <= bar, e
    gpu.close()


@pytest.mark.parametrize("make,prec,bar", PATHS, ids=IDS)
def test_horizon_of_one_substep(make, prec, bar):
    """tau equal to dt_sub: a single Euler factor (l = 1)."""
    from paper_2412_07240_gb300 import Filter
    sc = make()
    tau = sc.cfg.dt_sub
    gpu = Filter(sc.cfg, precision=prec)
    orc = OracleFilter(sc.cfg)
    gpu.meas_update(sc.meas, sc.z[0])
    orc.meas_update(sc.meas, sc.z[0])
    gpu.time_update(tau)
    orc.time_update(tau)
    e = compare(gpu, orc)
    _, c, M = gpu.pdf()
    # both on their own regrid decisions (see check_own_decisions)
    shift = displacement_bound(orc, c, M) if prec != "fp64" else 0.0
    assert e["l1"] <= bar + 2.0 * shift and e["frame"] <= max(bar, 1e-3 if shift else 0.0), e
    gpu.close()


def test_largest_grids_per_axis():
    """The largest axis each path holds (1-D 512, fused 2-D 128, 3-D 128 on one
    axis, 4-D float32 64 on one axis), two epochs each."""
    cases = [(w.c1_scenario(N=512, epochs=2), "fp16x3", {}),
             (w.small_2d_scenario(N=(128, 16), epochs=2), "fp16x3", {}),
             (w.small_3d_scenario(N=(128, 16, 32), epochs=2), "fp16x3", {}),
             (w.c6_scenario(N=(64, 6, 8, 6), epochs=2, local=True), "fp16x3", {})]
    for sc, prec, kw in cases:
        worst, log = max_errors(sc, precision=prec, **kw)
        check_own_decisions(log, 1e-5)
