"""Failure detection on the GPU without a fault: a bounded wait runs out.

The tensor-core GEMM waits on mbarriers with an iteration limit.  The
self-test leaves one pipeline stage unloaded (the flag its consumer waits for is
never set), so the MMA issuer's wait gives up.  The kernel records the timeout,
unwinds (copies and MMAs in flight drained, TMEM freed), the call reports
CCSD_ERR_TIMEOUT, and the context keeps working."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(lib):
    from paper_1911_00242_gb300 import binding
    assert lib.ccsd_tc_timeout_selftest() == binding.CCSD_ERR_TIMEOUT
    err = ctypes.c_double(-1.0)
    assert lib.ccsd_tc_selftest(200, 300, 100, 3, 5, ctypes.byref(err)) == 0
    assert 0 <= err.value < 2e-6
    assert lib.ccsd_tc_timeout_selftest() == binding.CCSD_ERR_TIMEOUT
