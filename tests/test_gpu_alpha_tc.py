"""Direct alpha sums of the small-band scales (L_j <= 32) on the tensor cores
(FP32 plans): kind::tf32 matrix products with the three-product split, so
FP32-level results.  Analysis against the oracle's Eq. (20) / Eq. (30) on
every row, synthesis of arbitrary coefficients against the oracle's
Eqs. (32)-(41), the mixed path against the FP64 plan at the level FP32 sums
reach (a single TF32 product, 10-bit mantissa, would miss it by two orders),
odd row counts and partial tiles, and no bounded wait giving up."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian, w_random
from tests.gpu_helpers import relerr, run_analysis, run_synthesis

pytestmark = pytest.mark.gpu


def direct_scales(p):
    return [j for j in range(p.nscale + 1) if p.alpha_method(j, 0)[0] == 0]


@pytest.mark.parametrize("L,N,lam,J0,mw", [(64, 3, 2.0, 0, False), (100, 5, 2.0, 0, False),
                                           (45, 2, 1.5, 0, False), (33, 5, 2.0, 0, True)])
def test_direct_scales_vs_oracle(L, N, lam, J0, mw):
    f = flm_gaussian(L, 31, "unit")
    kern = O.kernels(L, N, lam, J0)
    p = B.Plan(L, N, lam, J0, "mixed", mw=mw)
    try:
        ds = direct_scales(p)
        assert ds
        W, Wphi = run_analysis(p, f)
        Wo, Wpo = (O.analysis_mw if mw else O.analysis)(f, L, N, lam, J0, kern)
        for j in ds:
            got, ref = (Wphi, Wpo) if j == p.nscale else (W[j], Wo[j])
            assert relerr(got, ref) < 1e-5, (j, relerr(got, ref))
        nb = L if mw else 2 * L
        Wr, Wpr = w_random(L, N, W.shape[0], 9 + L, nb=nb)
        fo = (O.synthesis_mw if mw else O.synthesis)(Wr, Wpr, L, N, lam, J0, kern)
        fg = run_synthesis(p, Wr, Wpr)
        assert relerr(fg, fo) < 1e-5, relerr(fg, fo)
    finally:
        p.close()
    assert B.s2dw_wait_timeouts() == 0


def test_direct_scales_fp32_level_at_L256():
    """Mixed against FP64 on the direct scales: analysis W (K <= 64 terms)
    within 3e-6 and the synthesis stage V (2L - 1 = 511 terms, FP32
    accumulation) within 2e-5, both far below what one TF32 product per term
    would give (relative 2^-11 ~ 5e-4)."""
    L, N = 256, 5
    f = flm_gaussian(L, 8, "cl")
    pm = B.Plan(L, N, 2.0, 0, "mixed")
    p64 = B.Plan(L, N, 2.0, 0, "fp64")
    try:
        Wm, Wpm = run_analysis(pm, f)
        W64, Wp64 = run_analysis(p64, f)
        worst = 0.0
        for j in direct_scales(pm):
            got, ref = (Wpm, Wp64) if j == pm.nscale else (Wm[j], W64[j])
            worst = max(worst, relerr(got, ref))
        assert worst < 3e-6, worst
        # synthesis of the same (FP64) coefficients: stage V after the alpha step
        run_synthesis(pm, W64, Wp64)
        run_synthesis(p64, W64, Wp64)
        for j in direct_scales(pm):
            vm = pm.stage(1, j)
            v64 = p64.stage(1, j)
            assert relerr(vm, v64) < 2e-5, (j, relerr(vm, v64))
    finally:
        pm.close()
        p64.close()
    assert B.s2dw_wait_timeouts() == 0


def test_direct_scales_rows_at_L1024():
    """The headline sizes: three beta rows of every direct scale against the
    oracle (first, middle, last row: partial sample tile a >= 1920)."""
    L, N = 1024, 5
    f = flm_gaussian(L, 2, "cl")
    rows = [0, 1023, 2047]
    Wo, Wpo, _ = O.analysis_rows(f, L, N, 2.0, 0, rows, O.kernels(L, N, 2.0, 0))
    p = B.Plan(L, N, 2.0, 0, "mixed")
    try:
        W, Wphi = run_analysis(p, f)
        for j in direct_scales(p):
            if j == p.nscale:
                got, ref = Wphi[rows, :], Wpo
            else:
                got, ref = W[j][:, rows, :], Wo[j]
            if np.abs(ref).max() > 0:
                assert relerr(got, ref) < 1e-5, (j, relerr(got, ref))
    finally:
        p.close()
    assert B.s2dw_wait_timeouts() == 0
