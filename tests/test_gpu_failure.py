"""Bounded device waits: a wait whose completion never comes ends its kernel
with PMF_ERR_TIMEOUT instead of hanging the GPU, and the context stays usable.

The wait is the one every tensor-core kernel uses on its mbarriers (bulk
copies, MMA completion); the failure is made by a barrier that nothing
arrives at, with a small poll limit, never by a fault or an endless loop.
"""
import pytest

import workloads as w
from tests._parity import max_errors

pytestmark = pytest.mark.gpu


def test_wait_completes_when_the_arrival_happened():
    from paper_2412_07240_gb300 import _binding, selftest_bounded_wait
    assert selftest_bounded_wait(1 << 12, arrive=True) == _binding.OK


def test_wait_gives_up_and_reports_timeout_then_work_continues():
    from paper_2412_07240_gb300 import _binding, selftest_bounded_wait
    assert selftest_bounded_wait(1 << 10, arrive=False) == _binding.ERR_TIMEOUT
    assert selftest_bounded_wait(1 << 12, arrive=True) == _binding.OK
    # the same process keeps running filters on the tensor-core path
    worst, _ = max_errors(w.small_2d_scenario(N=(48, 32), epochs=2), precision="fp16x3")
    assert worst["l1"] <= 1e-5, worst


def test_invalid_poll_limit_rejected():
    from paper_2412_07240_gb300 import _binding, selftest_bounded_wait
    assert selftest_bounded_wait(0, arrive=True) == _binding.ERR_ARG
