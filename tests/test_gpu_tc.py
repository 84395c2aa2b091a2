"""GPU parity of the fused tensor-core path against the float64 oracle.

Bars (relative L1 of the weights after every update, and moments):
  FP16X3  <= 1e-5   (the mixed-precision target)
  BF16X6  <= 1e-5   (three BF16 pieces, six products: the BF16 split at the target)
  BF16X3  <= 1e-4   (reported; the 2-term bf16 split keeps ~16 bits)
  TF32    <= 3e-2   (reported; single TF32 products keep ~11 bits)
Cases: ragged non-square grids (48 x 32, 64 x 112), the full 128 x 128 range
workload, the linear model with frame re-alignment, the exact multiplier, and
the fused single-launch epoch (pmf_step) against the two separate calls.
"""
import numpy as np
import pytest

import workloads as w
from tests._parity import max_errors
from workloads import FilterConfig, MeasModel, Scenario, simulate

pytestmark = pytest.mark.gpu

BARS = {"fp16x3": 1e-5, "bf16x6": 1e-5, "bf16x3": 1e-4, "tf32": 3e-2}


def _check(worst, prec):
    bar = BARS[prec]
    assert worst["l1"] <= bar, worst
    assert worst["frame"] <= bar, worst
    assert worst["mean"] <= bar and worst["cov"] <= 10 * bar, worst


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x6", "bf16x3", "tf32"])
def test_small_2d_range(prec):
    worst, log = max_errors(w.small_2d_scenario(N=(48, 32), epochs=5), precision=prec)
    print(prec, worst)
    _check(worst, prec)


def test_ragged_2d_linear_fp16x3():
    sc = w.small_2d_scenario(N=(64, 112), kind="linear", epochs=4)
    worst, _ = max_errors(sc, precision="fp16x3")
    _check(worst, "fp16x3")


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x6"])
def test_c2_full_size(prec):
    worst, _ = max_errors(w.c2_scenario(epochs=6), precision=prec)
    print(prec, worst)
    _check(worst, prec)


def test_c2_sixty_epochs_bf16x6():
    """The 128 x 128 range workload over 60 epochs in the BF16 split at the
    target: the error stays at the bar over the whole run, not just per epoch."""
    worst, _ = max_errors(w.c2_scenario(epochs=60), precision="bf16x6")
    print(worst)
    _check(worst, "bf16x6")


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x6"])
def test_realignment(prec):
    cfg = FilterConfig(nx=2, N=(48, 64), A=np.array([[0.0, 1.0], [0.0, 0.0]]), Q=np.diag([0.01, 0.1]),
                       m0=np.array([0.0, 1.0]), P0=np.diag([0.5, 0.5]))
    meas = MeasModel("linear", R=np.array([[0.3 ** 2]]), H=np.array([[1.0, 0.0]]))
    sc = Scenario("cv", cfg, meas, dt=0.2, epochs=6)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=11)
    worst, log = max_errors(sc, precision=prec)
    assert any(s.endswith("R") for s, _ in log), "re-alignment not exercised"
    _check(worst, prec)


def test_exact_multiplier_fp16x3():
    worst, _ = max_errors(w.small_2d_scenario(N=(64, 48), epochs=4), precision="fp16x3",
                          psi_mode="exact")
    _check(worst, "fp16x3")


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x6"])
def test_fused_step(prec):
    worst, _ = max_errors(w.small_2d_scenario(N=(48, 48), epochs=5), precision=prec,
                          fused_step=True)
    _check(worst, prec)


def test_shear_realignment_bf16x6():
    cfg = FilterConfig(nx=2, N=(64, 112), A=np.array([[0.0, 1.0], [0.0, 0.0]]), Q=np.diag([0.01, 0.1]),
                       m0=np.array([0.0, 1.0]), P0=np.diag([0.5, 0.5]), realign_mode="shear")
    meas = MeasModel("linear", R=np.array([[0.3 ** 2]]), H=np.array([[1.0, 0.0]]))
    sc = Scenario("cv", cfg, meas, dt=0.2, epochs=6)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=11)
    worst, log = max_errors(sc, precision="bf16x6")
    assert any(s.endswith("R") for s, _ in log), "re-alignment not exercised"
    _check(worst, "bf16x6")


def test_unsupported_sizes_are_rejected():
    from paper_2412_07240_gb300 import Filter, Unsupported
    sc = w.small_2d_scenario(N=(40, 48))
    with pytest.raises(Unsupported):
        Filter(sc.cfg, precision="fp16x3")


def test_shear_realignment_fp16x3():
    cfg = FilterConfig(nx=2, N=(48, 64), A=np.array([[0.0, 1.0], [0.0, 0.0]]), Q=np.diag([0.01, 0.1]),
                       m0=np.array([0.0, 1.0]), P0=np.diag([0.5, 0.5]), realign_mode="shear")
    meas = MeasModel("linear", R=np.array([[0.3 ** 2]]), H=np.array([[1.0, 0.0]]))
    sc = Scenario("cv", cfg, meas, dt=0.2, epochs=6)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=11)
    worst, log = max_errors(sc, precision="fp16x3")
    assert any(s.endswith("R") for s, _ in log), "re-alignment not exercised"
    _check(worst, "fp16x3")


def test_shear_realignment_batch_equals_single():
    """The band-limited re-alignment in the batch's size-64 transform kernel
    equals the single-filter kernel's to float32 rounding, on the same frames."""
    from paper_2412_07240_gb300 import Batch, Filter
    from tests._parity import rel_l1
    cfg = FilterConfig(nx=2, N=(48, 64), A=np.array([[0.0, 1.0], [0.0, 0.0]]), Q=np.diag([0.01, 0.1]),
                       m0=np.array([0.0, 1.0]), P0=np.diag([0.5, 0.5]), realign_mode="shear")
    meas = MeasModel("linear", R=0.3 ** 2 * np.eye(2), H=np.eye(2))
    sc = Scenario("cv", cfg, meas, dt=0.2, epochs=6)
    sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=11)
    b = Batch([cfg], [meas])
    g = Filter(cfg, precision="fp16x3")
    for k in range(sc.epochs):
        b.step([0], sc.z[k][None, :], sc.dt)
        g.step(meas, sc.z[k], sc.dt)
    Pb, cb, Mb = b.pdf(0)
    Ps, cs, Ms = g.pdf()
    assert np.array_equal(cb, cs) and np.array_equal(Mb, Ms)
    assert rel_l1(Pb, Ps) <= 2e-6, rel_l1(Pb, Ps)
