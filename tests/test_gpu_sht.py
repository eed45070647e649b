"""Spherical harmonic transforms on the DH grid through the C ABI: the
device inverse SHT equals the oracle's pixel sums, the forward SHT recovers
f_lm exactly (DH quadrature), for FP64 and mixed plans."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,N", [(8, 3), (16, 1), (33, 5), (64, 2)])
def test_sht_matches_oracle(L, N, prec):
    import torch
    tol = 1e-12 if prec == "fp64" else 1e-5
    p = B.Plan(L, N, 2.0, 0, prec)
    cd, rd = p.torch_dtypes()
    f = flm_gaussian(L, 90 + L, "unit")
    fd = torch.from_numpy(f).to(cd).cuda()
    pix = p.alloc_pix()
    p.sht_inverse(fd, pix)
    torch.cuda.synchronize()
    ref = O.sht_inverse(f, L)
    assert np.abs(ref.imag).max() < 1e-12
    assert relerr(pix.double().cpu().numpy(), ref.real) < tol
    # forward SHT of the oracle's pixels recovers f_lm (exact quadrature)
    back = p.alloc_flm()
    p.sht_forward(torch.from_numpy(np.ascontiguousarray(ref.real)).to(rd).cuda(), back)
    torch.cuda.synchronize()
    assert relerr(back.to(torch.complex128).cpu().numpy(), f) < tol
    # device round trip
    back2 = p.alloc_flm()
    p.sht_forward(pix, back2)
    torch.cuda.synchronize()
    assert relerr(back2.to(torch.complex128).cpu().numpy(), f) < (1e-12 if prec == "fp64" else 2e-5)
    p.close()


def test_sht_then_wavelets():
    """Starting from pixel values: analysis(sht_forward(pix)) equals the
    analysis of the band-limited signal the pixels sample."""
    import torch
    L, N = 24, 3
    p = B.Plan(L, N, 2.0, 0, "fp64")
    f = flm_gaussian(L, 5, "cl")
    pix = torch.from_numpy(np.ascontiguousarray(O.sht_inverse(f, L).real)).cuda()
    flm = p.alloc_flm()
    p.sht_forward(pix, flm)
    W1, Wp1 = p.alloc_w()
    p.analysis(flm, W1, Wp1)
    W2, Wp2 = p.alloc_w()
    p.analysis(torch.from_numpy(f).cuda(), W2, Wp2)
    torch.cuda.synchronize()
    assert relerr(W1.cpu().numpy(), W2.cpu().numpy()) < 1e-12
    p.close()
