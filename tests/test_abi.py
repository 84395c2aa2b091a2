"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/pmf.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pmf_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2412_07240_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert len(_declared()) >= 13


def test_binding_signatures_cover_header():
    from paper_2412_07240_gb300 import _binding
    bound = {s[0] for s in _binding.SIGNATURES}
    assert _declared() <= bound | {"pmf_config_defaults"}, _declared() - bound


def test_config_defaults_and_struct_layout():
    from paper_2412_07240_gb300 import _binding
    lib = _binding.load()
    c = _binding.PmfConfig()
    lib.pmf_config_defaults(ctypes.byref(c))
    assert c.span_sigma == 6.0 and c.dt_sub == 0.01 and c.realign_rho == 0.5
    assert c.precision == 0 and c.psi_mode == 0
    # int nx, int N[4] (+4 padding) | A, Q | m0 | P0 | span, dt_sub, rho | precision, psi_mode,
    # realign_mode (+4 padding)
    assert ctypes.sizeof(_binding.PmfConfig) == 24 + 128 + 128 + 32 + 128 + 24 + 16
    assert _binding.PmfConfig.transform.offset == 476
    # int kind, nz | z[3] | R[9] | H[12] | p[24]
    assert ctypes.sizeof(_binding.PmfMeas) == 8 + 24 + 72 + 96 + 192


def test_invalid_config_rejected_without_gpu():
    """Validation happens on the host before any CUDA call."""
    from paper_2412_07240_gb300 import _binding
    lib = _binding.load()
    c = _binding.PmfConfig()
    lib.pmf_config_defaults(ctypes.byref(c))
    c.nx = 2
    c.N[0], c.N[1] = 33, 32      # odd size
    c.P0[0] = c.P0[3] = 1.0
    h = ctypes.c_void_p()
    assert lib.pmf_create(ctypes.byref(h), ctypes.byref(c), None) == _binding.ERR_ARG
    c.N[0] = 32
    c.P0[0] = -1.0               # not positive definite
    assert lib.pmf_create(ctypes.byref(h), ctypes.byref(c), None) == _binding.ERR_ARG
    c.nx = 1
    c.P0[0] = 1.0
    c.realign_mode = _binding.REALIGN["shear"]   # band-limited re-alignment needs n_x >= 2
    assert lib.pmf_create(ctypes.byref(h), ctypes.byref(c), None) == _binding.ERR_ARG
    assert not h.value


def test_product_path_does_not_import_oracle():
    import subprocess
    import sys
    code = ("import sys, paper_2412_07240_gb300 as p; p.load(); "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules)")
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)


def test_marshalling_of_config_and_measurement():
    import numpy as np

    import workloads as w
    from paper_2412_07240_gb300 import _binding
    sc = w.small_3d_scenario()
    c = _binding.make_config(sc.cfg, "fp16x3", "exact")
    assert c.nx == 3 and tuple(c.N[:3]) == (16, 24, 32)
    assert np.allclose(np.array(c.A[:9]).reshape(3, 3), sc.cfg.A)
    assert np.allclose(np.array(c.P0[:9]).reshape(3, 3), sc.cfg.P0)
    assert c.precision == 4 and c.psi_mode == 1
    m = _binding.make_meas(sc.meas, sc.z[0], 3)
    assert m.kind == 2 and m.nz == 2 and np.allclose(m.z[:2], sc.z[0])
    assert np.allclose(np.array(m.R[:4]).reshape(2, 2), sc.meas.R)
    sc1 = w.c1_scenario()
    c1 = _binding.make_config(sc1.cfg)
    assert c1.nx == 1 and c1.N[0] == 64 and c1.A[0] == -0.5 and c1.Q[0] == 0.5
    m1 = _binding.make_meas(sc1.meas, sc1.z[0], 1)
    assert m1.kind == 0 and m1.H[0] == 1.0 and m1.R[0] == 0.01


def test_unassigned_precision_rejected_without_gpu():
    """Precision code 2 is not assigned (no split-TF32 path is built)."""
    from paper_2412_07240_gb300 import _binding
    lib = _binding.load()
    c = _binding.PmfConfig()
    lib.pmf_config_defaults(ctypes.byref(c))
    c.nx = 2
    c.N[0], c.N[1] = 32, 32
    c.P0[0] = c.P0[3] = 1.0
    c.precision = 2
    h = ctypes.c_void_p()
    assert lib.pmf_create(ctypes.byref(h), ctypes.byref(c), None) == _binding.ERR_ARG
    assert "tf32x3" not in _binding.PREC


def test_bf16x6_scope_without_gpu():
    """BF16X6 (three BF16 pieces, six products) is a 2-D format: a 3-D filter
    and the FFT form are refused before any device work; code 6 is unknown."""
    from paper_2412_07240_gb300 import _binding
    lib = _binding.load()
    assert _binding.PREC["bf16x6"] == 5
    c = _binding.PmfConfig()
    lib.pmf_config_defaults(ctypes.byref(c))
    c.nx = 3
    c.N[0], c.N[1], c.N[2] = 32, 32, 32
    c.P0[0] = c.P0[4] = c.P0[8] = 1.0
    c.precision = 5
    h = ctypes.c_void_p()
    assert lib.pmf_create(ctypes.byref(h), ctypes.byref(c), None) == _binding.ERR_UNSUPPORTED
    c.nx = 2
    c.N[2] = 0
    c.P0[:] = [0.0] * len(c.P0)
    c.P0[0] = c.P0[3] = 1.0
    c.transform = 2                              # PMF_TRANSFORM_FFT
    assert lib.pmf_create(ctypes.byref(h), ctypes.byref(c), None) == _binding.ERR_UNSUPPORTED
    c.transform = 0
    c.precision = 6
    assert lib.pmf_create(ctypes.byref(h), ctypes.byref(c), None) == _binding.ERR_ARG


def test_batch_refuses_three_component_linear_without_gpu():
    """The 2-D tensor-core kernels form the likelihood of at most two
    measurement components: a batch whose 2-D filter has a three-component
    linear model is refused (PMF_ERR_UNSUPPORTED) before any device work."""
    import numpy as np
    from paper_2412_07240_gb300 import _binding
    from workloads import FilterConfig, MeasModel
    lib = _binding.load()
    cfg = FilterConfig(nx=2, N=(32, 32), A=np.zeros((2, 2)), Q=np.eye(2), m0=np.zeros(2), P0=np.eye(2))
    three = MeasModel("linear", R=np.eye(3), H=np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]))
    carr = (_binding.PmfConfig * 1)(_binding.make_config(cfg, "bf16x6", "euler", "auto"))
    marr = (_binding.PmfMeas * 1)(_binding.make_meas(three, np.zeros(3), 2))
    h = ctypes.c_void_p()
    assert lib.pmf_batch_create(ctypes.byref(h), carr, marr, 1, 0, None) == _binding.ERR_UNSUPPORTED
    assert not h.value
