"""Steering (Eq. (10)) through the C ABI: the device interpolation of the N
sampled orientations equals the oracle's, and steering the device W equals
the oracle's analysis at those orientations."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu

CASES = [(16, 3, 2.0, 0), (24, 5, 2.0, 1), (20, 1, 3.0, 0), (32, 8, 2.0, 0), (17, 2, 1.7, 0)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,N,lam,J0", CASES)
def test_steer_matches_oracle(L, N, lam, J0, prec):
    import torch
    tol = 1e-12 if prec == "fp64" else 1e-5
    p = B.Plan(L, N, lam, J0, prec)
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    f = flm_gaussian(L, 21 + L, "cl")
    W, Wp = p.alloc_w()
    p.analysis(torch.from_numpy(f).to(cd).cuda(), W, Wp)
    rng = np.random.default_rng(L * N)
    gammas = np.concatenate([np.pi * np.arange(N) / N, rng.uniform(-4, 4, 7)])
    out = p.steer(W, gammas)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    # interpolation parity on the device's own W
    ref = O.steer(W.double().cpu().numpy(), N, gammas)
    for j in range(got.shape[0]):
        assert relerr(got[j], ref[j]) < tol, (j, relerr(got[j], ref[j]))
    # the sample orientations reproduce W exactly (up to rounding)
    assert np.abs(got[:, :N] - W.double().cpu().numpy()).max() <= tol * max(1.0, float(W.abs().max()))
    # against the oracle's analysis steered to the same angles
    Wo, _ = O.analysis(f, L, N, lam, J0)
    refo = O.steer(Wo, N, gammas)
    for j in range(got.shape[0]):
        if np.abs(refo[j]).max() > 0:
            assert relerr(got[j], refo[j]) < (1e-11 if prec == "fp64" else 1e-5)
    p.close()


def test_steer_arguments():
    import torch
    p = B.Plan(16, 3, 2.0, 0, "mixed")
    W, _ = p.alloc_w()
    out = torch.empty((p.J + 1, 33, 32, 31), dtype=torch.float32, device="cuda")
    for ng in (0, 33):
        with pytest.raises(B.S2dwError):
            B.s2dw_steer(p.handle, W, np.zeros(ng), out)
    B.s2dw_steer(p.handle, W, np.zeros(32), out)  # the largest count is accepted
    torch.cuda.synchronize()
    p.close()
