"""The shared-memory FFT form of the 2-D Hartley transforms (steps 1 and 5 of
the Sec. V-B algorithm on the fused and batched tensor-core paths), against
the float64 oracle, and the per-size autotuner that chooses between it and
the tensor-core GEMMs."""
import json
import os

import numpy as np
import pytest

import workloads as w
from tests._parity import check_own_decisions, max_errors, rel_l1

pytestmark = pytest.mark.gpu

BAR = {"fp16x3": 1e-5, "bf16x3": 1e-4}


@pytest.mark.parametrize("N", [(32, 48), (96, 64), (48, 128), (16, 96)])
def test_fft_form_matches_oracle(N):
    """Range measurement (sharp posteriors), every update, oracle on its own decisions."""
    sc = w.small_2d_scenario(N=N, epochs=5)
    _, log = max_errors(sc, precision="fp16x3", transform="fft")
    check_own_decisions(log, BAR["fp16x3"])


def test_fft_form_c2_full_size():
    """The 128 x 128 oscillator with the range measurement, 60 epochs, fused steps."""
    sc = w.c2_scenario(epochs=60)
    _, log = max_errors(sc, precision="fp16x3", transform="fft", fused_step=True)
    check_own_decisions(log, BAR["fp16x3"])


@pytest.mark.parametrize("prec", ["bf16x3"])
def test_fft_form_other_formats_and_exact_multiplier(prec):
    sc = w.small_2d_scenario(N=(64, 48), epochs=4)
    _, log = max_errors(sc, precision=prec, transform="fft")
    check_own_decisions(log, BAR[prec])
    _, log = max_errors(sc, precision="fp16x3", transform="fft", psi_mode="exact")
    check_own_decisions(log, BAR["fp16x3"])


def test_fft_form_with_realignment():
    """Multilinear and band-limited re-alignment ahead of the FFT-form transforms."""
    from workloads import FilterConfig, MeasModel, Scenario, simulate
    for mode in ("multilinear", "shear"):
        cfg = FilterConfig(nx=2, N=(64, 48), A=np.array([[0.0, 1.0], [0.0, 0.0]]), Q=np.diag([0.01, 0.1]),
                           m0=np.array([0.0, 1.0]), P0=np.diag([0.5, 0.5]), realign_mode=mode)
        meas = MeasModel("linear", R=np.array([[0.3 ** 2]]), H=np.array([[1.0, 0.0]]))
        sc = Scenario("cv", cfg, meas, dt=0.2, epochs=8)
        sc.truth, sc.z = simulate(cfg, meas, sc.dt, sc.epochs, seed=11)
        _, log = max_errors(sc, precision="fp16x3", transform="fft")
        assert any(s.endswith("R") for s, _ in log), "re-alignment not exercised"
        check_own_decisions(log, BAR["fp16x3"])


def test_fft_form_in_batches_equals_single_filters():
    """Both size classes of the batched transform kernels run the FFT form."""
    from paper_2412_07240_gb300 import Batch, Filter
    cfgs, meas, dt, truth, z = w.c4_batch(count=10, epochs=4)
    b = Batch(cfgs, [meas] * len(cfgs), transform="fft")
    singles = [Filter(c, precision="fp16x3", transform="fft") for c in cfgs]
    ids = np.arange(len(cfgs))
    for k in range(4):
        b.step(ids, z[:, k], dt)
        for i, f in enumerate(singles):
            f.step(meas, z[i, k], dt)
    for i, f in enumerate(singles):
        Pb, cb, Mb = b.pdf(i)
        Ps, cs, Ms = f.pdf()
        assert np.array_equal(cb, cs) and np.array_equal(Mb, Ms), i
        assert rel_l1(Pb, Ps) <= 5e-6, (i, rel_l1(Pb, Ps))


def test_fft_and_gemm_forms_agree_with_each_other():
    """Same filter in both forms, every update: both within the bar of the
    oracle, so within twice the bar of each other."""
    sc = w.small_2d_scenario(N=(96, 96), kind="linear", epochs=4)
    _, lf = max_errors(sc, precision="fp16x3", transform="fft")
    _, lg = max_errors(sc, precision="fp16x3", transform="gemm")
    for (sf, ef), (sg, eg) in zip(lf, lg):
        assert sf == sg and ef["frame"] < 1e-9 and eg["frame"] < 1e-9
        assert ef["l1"] <= 1e-5 and eg["l1"] <= 1e-5


def test_autotuner_records_both_forms_per_size(monkeypatch):
    """The 2-D autotuner times both forms the first time a size is used and
    keeps its choice and timings beside the library."""
    from paper_2412_07240_gb300 import Filter, lib_path
    monkeypatch.delenv("PMF_2D_FORM", raising=False)
    for N in ((32, 32), (64, 48)):
        f = Filter(w.small_2d_scenario(N=N, epochs=1).cfg, precision="fp16x3")
        f.close()
    rec = json.load(open(os.path.join(os.path.dirname(lib_path()), "autotune_2d.json")))
    for N in ((32, 32), (64, 48)):
        e = rec[f"2d:{N[0]}x{N[1]}:4"]
        assert e["form"] in (0, 1) and e["gemm_us"] > 0 and e["fft_us"] > 0
        assert e["form"] == int(e["fft_us"] < e["gemm_us"])
