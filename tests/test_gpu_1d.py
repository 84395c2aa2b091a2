"""1-D CUDA-core kernel (n_x = 1, float32) against the float64 oracle, through the C ABI."""
import numpy as np
import pytest

import workloads as w
from tests._parity import max_errors

pytestmark = pytest.mark.gpu

BAR = 1e-5   # relative L1 of the weights, float32 path


def test_c1_all_epochs_fused_step():
    sc = w.c1_scenario()
    worst, log = max_errors(sc, precision="fp16x3", fused_step=True)
    assert worst["l1"] < BAR, log
    assert worst["mean"] < BAR and worst["cov"] < 10 * BAR, worst


def test_c1_separate_updates_and_path():
    from paper_2412_07240_gb300 import Filter
    sc = w.c1_scenario()
    f = Filter(sc.cfg, precision="fp16x3")
    assert f.path == 3
    f.close()
    worst, log = max_errors(sc, precision="fp16x3", epochs=8)
    assert worst["l1"] < BAR, log


@pytest.mark.parametrize("N", [16, 200, 512])
def test_grid_sizes(N):
    # ragged (200 = 8 * 25) and the largest supported grid, a few epochs
    sc = w.c1_scenario(N=N, epochs=6)
    worst, log = max_errors(sc, precision="fp16x3", fused_step=True)
    assert worst["l1"] < BAR, log


def test_exact_multiplier():
    sc = w.c1_scenario(epochs=6)
    worst, log = max_errors(sc, precision="fp16x3", fused_step=True, psi_mode="exact")
    assert worst["l1"] < BAR, log


def test_unsupported_size_rejected():
    from paper_2412_07240_gb300 import Filter, Unsupported
    sc = w.c1_scenario(N=1000)
    with pytest.raises(Unsupported):
        Filter(sc.cfg, precision="fp16x3")


@pytest.mark.parametrize("form", ["fft", "matvec"])
@pytest.mark.parametrize("N", [64, 512])
def test_transform_forms(form, N, monkeypatch):
    # both Hartley forms (shared-memory FFT and matrix-vector) against the oracle
    monkeypatch.setenv("PMF_1D_FORM", form)
    sc = w.c1_scenario(N=N, epochs=6)
    worst, log = max_errors(sc, precision="fp16x3", fused_step=True)
    assert worst["l1"] < BAR, log


@pytest.mark.parametrize("form", ["fft", "gemm"])
def test_transform_form_from_the_config(form, monkeypatch):
    monkeypatch.delenv("PMF_1D_FORM", raising=False)
    sc = w.c1_scenario(N=128, epochs=6)
    worst, log = max_errors(sc, precision="fp16x3", fused_step=True, transform=form)
    assert worst["l1"] < BAR, log


def test_fft_form_only_where_it_exists():
    from paper_2412_07240_gb300 import Filter, Unsupported
    with pytest.raises(Unsupported):                         # not a power of two
        Filter(w.c1_scenario(N=200).cfg, precision="fp16x3", transform="fft")
    with pytest.raises(Unsupported):                         # float64 path
        Filter(w.c1_scenario(N=64).cfg, precision="fp64", transform="fft")
    with pytest.raises(Unsupported):                         # 2-D axis not 2^a 3^b
        Filter(w.small_2d_scenario(N=(80, 32), epochs=1).cfg, precision="fp16x3", transform="fft")
    with pytest.raises(Unsupported):                         # 3-D pipelines
        Filter(w.small_3d_scenario(N=(16, 16, 16), epochs=1).cfg, precision="fp16x3", transform="fft")


def test_autotuner_records_its_choice(monkeypatch):
    import json
    import os
    from paper_2412_07240_gb300 import Filter, lib_path
    monkeypatch.delenv("PMF_1D_FORM", raising=False)
    sc = w.c1_scenario(N=128, epochs=2)
    f = Filter(sc.cfg, precision="fp16x3")
    f.step(sc.meas, sc.z[0], sc.dt)
    f.close()
    path = os.path.join(os.path.dirname(lib_path()), "autotune.json")
    entry = json.load(open(path))["1d:128"]
    assert entry["mode"] in (0, 1)
