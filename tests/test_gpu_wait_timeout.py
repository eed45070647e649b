"""Failure path of the library's bounded device waits, exercised on demand
without a GPU fault.  A warp waits on an mbarrier that nothing arrives on and
gives up after its limit.  The give-up is counted and reported by
s2dw_wait_timeouts: status S2DW_ETIMEOUT through the C ABI, the count
through the binding.  The context stays usable: a mixed round trip
afterwards (through the tensor-core kernels) is exact and reports no
timeout."""
import ctypes

import numpy as np
import pytest

from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian
from tests.gpu_helpers import relerr, run_analysis, run_synthesis, torch_cuda

pytestmark = pytest.mark.gpu


def test_wait_probe_is_reported_and_context_survives():
    torch_cuda()
    B.s2dw_wait_timeouts()  # reset
    B.s2dw_wait_probe(200_000)  # about 0.1 ms
    assert B.s2dw_wait_timeouts() == 1
    assert B.s2dw_wait_timeouts() == 0  # read and reset
    B.s2dw_wait_probe(1_000)
    B.s2dw_wait_probe(1_000)
    c = ctypes.c_int()
    assert B.lib().s2dw_wait_timeouts(ctypes.byref(c)) == -4  # S2DW_ETIMEOUT
    assert c.value == 2
    assert B.lib().s2dw_wait_timeouts(ctypes.byref(c)) == 0 and c.value == 0
    L, N = 40, 3
    f = flm_gaussian(L, 6, "unit")
    p = B.Plan(L, N, 2.0, 0, "mixed")
    try:
        W, Wphi = run_analysis(p, f)
        fr = run_synthesis(p, W, Wphi)
        assert relerr(fr, f) < 1e-5
        assert np.isfinite(W).all()
    finally:
        p.close()
    assert B.s2dw_wait_timeouts() == 0
