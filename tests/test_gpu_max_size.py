"""The largest band-limit the library accepts, L = 2048 (Fourier axes of
2L - 1 = 4095, FFT length 8192 in the beta and alpha stages, the largest
shared-memory configurations), with N = 3, lambda = 2, J0 = 0 and the
C_l = 1/(l(l+1)) spectrum.

Both precisions: one beta row of every scale against the oracle (normwise
per scale, 1e-11 for float64, 1e-5 for mixed), and the exact round trip of
Sec. 3.4 with the coefficients kept on the device (1e-12 / 1e-5)."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian
from tests.gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

L, N, LAM, J0 = 2048, 3, 2.0, 0
ROW = 1500


@pytest.fixture(scope="module")
def oracle_row():
    f = flm_gaussian(L, 11, "cl")
    kern = O.kernels(L, N, LAM, J0)
    Wo, _, _ = O.analysis_rows(f, L, N, LAM, J0, [ROW], kern)
    return f, Wo


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_max_band_limit(prec, oracle_row):
    torch = torch_cuda()
    f, Wo = oracle_row
    p = B.Plan(L, N, LAM, J0, prec)
    try:
        cd, rd = p.torch_dtypes()
        fd = torch.from_numpy(f).to(cd).cuda()
        W, Wphi = p.alloc_w()
        p.analysis(fd, W, Wphi)
        fr = p.alloc_flm()
        p.synthesis(W, Wphi, fr)
        torch.cuda.synchronize()
        row = W[:, :, ROW, :].double().cpu().numpy()
        for j in range(row.shape[0]):
            den = np.abs(Wo[j]).max()
            err = np.abs(row[j] - Wo[j][:, 0, :]).max() / den if den > 0 else np.abs(row[j]).max()
            assert err < (1e-11 if prec == "fp64" else 1e-5), (prec, j, err)
        eps = (fr.to(torch.complex128).cpu() - torch.from_numpy(f)).abs().max().item() / np.abs(f).max()
        assert eps < (1e-12 if prec == "fp64" else 1e-5), (prec, eps)
        assert torch.isfinite(W).all().item()
    finally:
        p.close()
