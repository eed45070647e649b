"""How each scale's alpha sums are evaluated (s2dw_alpha_method) at L=1024,
N=5, lambda=2: the two full-band scales by one chirp-z convolution of
length 4096, the scales with 64 <= L_j <= 512 by the segmented chirp-z
(S + 1 FFTs of a shorter length M' >= 2 L_j - 2 + P covering all 2L-1
samples), the rest by direct sums; and the segmented path reproduces the
oracle at sampled alpha positions of every segment."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian
from tests.gpu_helpers import run_analysis

pytestmark = pytest.mark.gpu


def test_methods_at_L1024():
    p = B.Plan(1024, 5, 2.0, 0, "mixed")
    n = 2 * 1024 - 1
    try:
        for j in range(p.nscale + 1):
            Lj = p.support(j)[1] + 1 if j < p.nscale else None
            for d in (0, 1):
                method, M, S, P = p.alpha_method(j, d)
                if j < 2:
                    assert (method, M, S) == (1, 4096, 1)
                elif j < p.nscale and Lj > 32:
                    assert method == 2 and M < 4096 and S >= 2
                    assert P == M - 2 * Lj + 2 and S * P >= n and (S - 1) * P < n
                else:
                    assert method == 0
        with pytest.raises(B.S2dwError):
            p.alpha_method(p.nscale + 1, 0)
        with pytest.raises(B.S2dwError):
            p.alpha_method(0, 2)
    finally:
        p.close()


def test_segmented_scales_match_oracle_at_L256():
    """L=256: the scales with L_j = 64, 128 use two segments of length 512;
    one beta row of every scale against the oracle in float64 (1e-11)."""
    L, N = 256, 5
    f = flm_gaussian(L, 5, "cl")
    p = B.Plan(L, N, 2.0, 0, "fp64")
    try:
        segd = [j for j in range(p.nscale) if p.alpha_method(j, 0)[0] == 2]
        assert segd, "no segmented scale at L=256"
        W, _ = run_analysis(p, f)
        rows = [0, 255, 511]
        Wo, _, _ = O.analysis_rows(f, L, N, 2.0, 0, rows, O.kernels(L, N, 2.0, 0))
        for j in segd:
            err = np.abs(W[j][:, rows, :] - Wo[j]).max() / np.abs(Wo[j]).max()
            assert err < 1e-11, (j, err)
    finally:
        p.close()
