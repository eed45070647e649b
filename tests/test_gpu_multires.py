"""Multi-resolution plans (S2DW_MULTIRES): every scale on the grid of its
own band-limit, compared with the oracle's multi-resolution transforms; the
round trip stays exact, batches mix multi- and full-resolution plans."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu

CASES = [(16, 3, 2.0, 0), (24, 2, 2.0, 1), (20, 1, 3.0, 0), (37, 4, 1.7, 1), (64, 5, 2.0, 0)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,N,lam,J0", CASES)
def test_multires_matches_oracle(L, N, lam, J0, prec):
    import torch
    tol = 1e-11 if prec == "fp64" else 1e-5
    p = B.Plan(L, N, lam, J0, prec, multires=True)
    cd, rd = p.torch_dtypes()
    Ls, Lp = O.band_limits(L, N, lam, J0)
    assert [g[0] for g in p.grids[:-1]] == Ls and p.grids[-1][0] == Lp
    f = flm_gaussian(L, 60 + L, "unit")
    W, Wp = p.alloc_w()
    p.analysis(torch.from_numpy(f).to(cd).cuda(), W, Wp)
    torch.cuda.synchronize()
    Wo, Wpo = O.analysis_multires(f, L, N, lam, J0)
    for j in range(p.nscale):
        got = p.w_scale(W, j).double().cpu().numpy()
        assert got.shape == Wo[j].shape
        assert relerr(got, Wo[j]) < tol, (j, relerr(got, Wo[j]))
    if np.abs(Wpo).max() > 0:
        assert relerr(Wp.double().cpu().numpy(), Wpo) < tol
    # synthesis of the oracle's coefficients, and the device round trip
    Wd = torch.cat([torch.from_numpy(np.ascontiguousarray(w)).reshape(-1) for w in Wo]).to(rd).cuda()
    fo = p.alloc_flm()
    p.synthesis(Wd, torch.from_numpy(np.ascontiguousarray(Wpo)).to(rd).cuda(), fo)
    fr = p.alloc_flm()
    p.synthesis(W, Wp, fr)
    torch.cuda.synchronize()
    assert relerr(fo.to(torch.complex128).cpu().numpy(), f) < (1e-12 if prec == "fp64" else 2e-5)
    assert relerr(fr.to(torch.complex128).cpu().numpy(), f) < (1e-12 if prec == "fp64" else 2e-5)
    p.close()


def test_multires_batch_and_steer():
    import torch
    specs = [(32, 3, 2.0, 0, True), (32, 3, 2.0, 0, False), (20, 2, 3.0, 1, True)]
    plans = [B.Plan(L, N, lam, J0, "mixed", multires=mr) for (L, N, lam, J0, mr) in specs]
    fs = [torch.from_numpy(flm_gaussian(p.L, 7 + i, "cl")).to(torch.complex64).cuda() for i, p in enumerate(plans)]
    Wb = [p.alloc_w() for p in plans]
    B.s2dw_analysis_batch([p.handle for p in plans], fs, [w[0] for w in Wb], [w[1] for w in Wb])
    for p, f, w in zip(plans, fs, Wb):
        W1, Wp1 = p.alloc_w()
        p.analysis(f, W1, Wp1)
        torch.cuda.synchronize()
        assert torch.equal(W1, w[0]) and torch.equal(Wp1, w[1])
    fb = [p.alloc_flm() for p in plans]
    B.s2dw_synthesis_batch([p.handle for p in plans], [w[0] for w in Wb], [w[1] for w in Wb], fb)
    torch.cuda.synchronize()
    for p, f, g in zip(plans, fs, fb):
        assert relerr(g.to(torch.complex128).cpu().numpy(), f.to(torch.complex128).cpu().numpy()) < 2e-5
    # steering a multi-resolution W: per-scale blocks, against the oracle's interpolation
    p, W = plans[0], Wb[0][0]
    gam = [0.4, 2.9]
    out = p.steer(W, gam)
    torch.cuda.synchronize()
    for j in range(p.nscale):
        Lg, off, n = p.grids[j]
        blk = out[(off // p.N) * len(gam):(off // p.N) * len(gam) + len(gam) * 2 * Lg * (2 * Lg - 1)]
        ref = O.steer(p.w_scale(W, j).double().cpu().numpy()[None], p.N, gam)[0]
        assert relerr(blk.view(len(gam), 2 * Lg, 2 * Lg - 1).double().cpu().numpy(), ref) < 1e-5
    for q in plans:
        q.close()
