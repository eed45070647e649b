"""Wavelet transforms sampled with L beta samples (S2DW_MW; the McEwen-Wiaux
grid that Sec. 4 names as the replacement of the DH grid): analysis against
the oracle's Eq. (20) at beta_b = (2b+1) pi/(2L-1), synthesis against the
oracle's exact resampling + DH synthesis, exact round trips.  Includes odd
row counts (N L odd), non-power-of-two L (chirp-z beta), even N, J0 > 0 with
the scaling part active, the segmented chirp-z range (L = 255, 256) and a
spot check at L = 1024."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian, w_random
from tests.gpu_helpers import relerr, run_analysis, run_synthesis

pytestmark = pytest.mark.gpu

CASES = [(8, 3, 2.0, 0), (9, 3, 2.0, 1), (16, 4, 3.0, 0), (33, 5, 2.0, 0), (40, 1, 2.0, 2), (64, 5, 2.0, 0)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,N,lam,J0", CASES)
def test_mw_analysis_synthesis_vs_oracle(L, N, lam, J0, prec):
    tol = 1e-11 if prec == "fp64" else 1e-5
    f = flm_gaussian(L, 21, "unit")
    kern = O.kernels(L, N, lam, J0)
    p = B.Plan(L, N, lam, J0, prec, mw=True)
    try:
        assert p.w_shape == (p.nscale, N, L, 2 * L - 1) and p.wphi_shape == (L, 2 * L - 1)
        W, Wphi = run_analysis(p, f)
        Wo, Wpo = O.analysis_mw(f, L, N, lam, J0, kern)
        for j in range(W.shape[0]):
            assert relerr(W[j], Wo[j]) < tol, (j, relerr(W[j], Wo[j]))
        assert np.abs(Wphi - Wpo).max() < tol * max(1.0, np.abs(Wpo).max())
        # synthesis of arbitrary coefficients: the oracle's resampling + DH synthesis
        Wr, Wpr = w_random(L, N, W.shape[0], 5 + L, nb=L)
        fo = O.synthesis_mw(Wr, Wpr, L, N, lam, J0, kern)
        fg = run_synthesis(p, Wr, Wpr)
        assert relerr(fg, fo) < tol, relerr(fg, fo)
        # exact round trip
        fr = run_synthesis(p, W, Wphi)
        assert np.abs(fr - f).max() < (1e-12 if prec == "fp64" else 1e-5) * np.abs(f).max()
    finally:
        p.close()


@pytest.mark.parametrize("L,N", [(255, 5), (256, 5)])
def test_mw_round_trip_and_rows_mid_size(L, N):
    """Scales in the segmented chirp-z range, an odd row count (L = 255):
    beta rows against the oracle and the round trip, both precisions."""
    f = flm_gaussian(L, 4, "cl")
    kern = O.kernels(L, N, 2.0, 0)
    rows = [0, L // 2, L - 1]
    Wo, _, _ = O.analysis_rows(f, L, N, 2.0, 0, rows, kern, betas=O.mw_betas(L))
    for prec in ("fp64", "mixed"):
        p = B.Plan(L, N, 2.0, 0, prec, mw=True)
        try:
            W, Wphi = run_analysis(p, f)
            for j in range(W.shape[0]):
                den = np.abs(Wo[j]).max()
                if den > 0:
                    err = np.abs(W[j][:, rows, :] - Wo[j]).max() / den
                    assert err < (1e-11 if prec == "fp64" else 1e-5), (prec, j, err)
            fr = run_synthesis(p, W, Wphi)
            assert np.abs(fr - f).max() < (1e-12 if prec == "fp64" else 1e-5) * np.abs(f).max()
        finally:
            p.close()


def test_mw_at_L1024():
    """The headline sizes on the MW grid: a beta row of every scale against the
    oracle and the round trip (mixed)."""
    L, N = 1024, 5
    f = flm_gaussian(L, 2, "cl")
    Wo, _, _ = O.analysis_rows(f, L, N, 2.0, 0, [700], O.kernels(L, N, 2.0, 0), betas=O.mw_betas(L))
    p = B.Plan(L, N, 2.0, 0, "mixed", mw=True)
    try:
        W, Wphi = run_analysis(p, f)
        for j in range(W.shape[0]):
            den = np.abs(Wo[j]).max()
            if den > 0:
                assert np.abs(W[j][:, [700], :] - Wo[j]).max() / den < 1e-5
        fr = run_synthesis(p, W, Wphi)
        assert np.abs(fr - f).max() < 1e-5 * np.abs(f).max()
    finally:
        p.close()


def test_mw_flag_errors():
    with pytest.raises(B.S2dwError):
        B.Plan(64, 3, 2.0, 0, "mixed", multires=True, mw=True)


def test_mw_steer_reproduces_samples_and_oracle():
    """Steering on the MW grid (Eq. (10)): the output has L beta rows per
    orientation; the sampled orientations give W back, and any orientation
    equals the oracle's interpolation of the same W."""
    import torch
    L, N = 16, 3
    p = B.Plan(L, N, 2.0, 0, "mixed", mw=True)
    try:
        f = torch.from_numpy(flm_gaussian(L, 8, "unit")).to(torch.complex64).cuda()
        W, Wphi = p.alloc_w()
        p.analysis(f, W, Wphi)
        gam = np.concatenate([np.pi * np.arange(N) / N, [0.37, -2.1]])
        out = p.steer(W, gam)
        torch.cuda.synchronize()
        assert tuple(out.shape) == (p.nscale, len(gam), L, 2 * L - 1)
        Wn = W.double().cpu().numpy()
        got = out.double().cpu().numpy()
        assert np.abs(got[:, :N] - Wn).max() <= 1e-5 * max(1.0, np.abs(Wn).max())
        ref = O.steer(Wn, N, gam)
        for j in range(got.shape[0]):
            assert relerr(got[j], ref[j]) < 1e-5, j
    finally:
        p.close()
