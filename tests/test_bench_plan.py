"""The benchmark's argument and scenario plumbing, without a GPU.

Every leg of a bench run (warm-up and timed steps, the end-to-end loop, the
float64 comparator, the oracle parity sample) indexes into a seeded scenario;
these tests build the scenarios the way bench.py does, for the usual
arguments (--steps 20 --warmup 5) and for edge cases, and check that each
leg stays inside.
"""
import numpy as np
import pytest

import bench
import workloads as w


def test_default_workload_is_the_batch():
    args = bench.make_parser().parse_args([])
    assert args.workload == "c4"
    assert args.gpus == 1 and args.impl == "native"
    # split-BF16 differentiation where the kernels have it (2-D), FP16X3 elsewhere
    assert args.precision is None
    assert [bench.default_precision(x) for x in ("c2", "c3", "c4", "c5", "c6")] == \
        ["bf16x6", "fp16x3", "bf16x6", "bf16x6", "fp16x3"]


@pytest.mark.parametrize("workload", ["c2", "c3", "c6"])
@pytest.mark.parametrize("steps,warmup", [(20, 5), (1, 3), (200, 10), (3, 100)])
def test_single_filter_legs_fit_their_scenario(workload, steps, warmup):
    warmup = max(3, warmup)
    legs = bench.leg_epochs(workload, steps, warmup)
    sc = bench._scenario(workload, max(legs.values()) + 1)
    for name, n in legs.items():
        assert len(sc.z) >= n, (name, n, len(sc.z))
    # the oracle subprocess builds the same scenario (same expression, same length)
    expr = bench._scenario_expr(workload, max(legs["parity"], len(sc.z)))
    sc2 = eval(expr, {"w": w})
    assert len(sc2.z) == len(sc.z)
    np.testing.assert_array_equal(sc2.z, sc.z)


@pytest.mark.parametrize("steps,warmup", [(20, 5), (1, 3), (200, 10)])
def test_batch_legs_fit(steps, warmup):
    warmup = max(3, warmup)
    epochs = warmup + steps + 1
    cfgs, meas, dt, truth, z = w.c4_batch(count=8, epochs=epochs)
    # timed steps and the end-to-end loop read z[:, warmup + k]
    assert warmup + steps - 1 < z.shape[1]
    assert warmup + min(5, steps) - 1 < z.shape[1]
    # the oracle sample and the parity batch (their own c4_batch call over the
    # whole horizon) see the same measurements as the timed batch's first
    # epochs: draws are made epoch by epoch
    _, _, _, _, z8 = w.c4_batch(count=8, epochs=8)
    np.testing.assert_array_equal(z8[:, :min(8, epochs)], z[:, :min(8, epochs)])
    ids = bench.c4_sample_ids(4096)
    assert len(ids) == 256 and ids[0] == 0 and ids[-1] == 4095 and len(set(ids)) == 256
    assert len(bench.c4_sample_ids(100)) == 100


def test_executed_mma_flops_closed_form(monkeypatch):
    """Issued tensor-core flops of one epoch: 128 lanes x N x K per stage and
    split product; six stages in the GEMM form, the two regrid stages in the
    FFT form."""
    cfgs = [w.FilterConfig(nx=2, N=(32, 64), A=np.zeros((2, 2)), Q=np.eye(2), m0=np.zeros(2), P0=np.eye(2)),
            w.FilterConfig(nx=2, N=(128, 128), A=np.zeros((2, 2)), Q=np.eye(2), m0=np.zeros(2), P0=np.eye(2))]
    sq = 32 ** 2 + 64 ** 2 + 2 * 128 ** 2
    monkeypatch.setenv("PMF_2D_FORM", "gemm")
    assert bench.executed_mma_flops(cfgs, "bf16x6") == 6 * 2 * 128 * 3 * sq
    assert bench.executed_mma_flops(cfgs, "fp16x3") == 3 * 2 * 128 * 3 * sq
    assert bench.executed_mma_flops(cfgs, "tf32") == 1 * 2 * 128 * 3 * sq
    monkeypatch.setenv("PMF_2D_FORM", "fft")
    assert bench.executed_mma_flops(cfgs, "fp16x3") == 3 * 2 * 128 * 1 * sq
