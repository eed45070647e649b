"""The measured workloads at full size (GPU vs oracle on what the oracle can
compute one by one): L=256 and L=1024 with N=5, lambda=2, J0=0 and the
C_l = 1/(l(l+1)) spectrum, and the 64-signal batch of mixed L and N.

Per-scale errors are normwise, max|x - x_ref| / max|x_ref|, with the float64
path within 1e-11 and the mixed path within 1e-5."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian, w_random
from tests.gpu_helpers import run_analysis, run_synthesis

pytestmark = pytest.mark.gpu


def _per_scale_err(W, Wo):
    errs = []
    for j in range(W.shape[0]):
        den = np.abs(Wo[j]).max()
        errs.append(np.abs(W[j] - Wo[j]).max() / den if den > 0 else np.abs(W[j]).max())
    return np.array(errs)


@pytest.mark.parametrize("L,seed,rows", [(256, 1, [0, 97, 300, 511]), (1024, 2, [0, 700, 2047])])
def test_analysis_spot_rows(L, seed, rows):
    N, lam, J0 = 5, 2.0, 0
    f = flm_gaussian(L, seed, "cl")
    kern = O.kernels(L, N, lam, J0)
    Wo, Wpo, _ = O.analysis_rows(f, L, N, lam, J0, rows, kern)
    out = {}
    for prec in ("fp64", "mixed"):
        p = B.Plan(L, N, lam, J0, prec)
        W, Wphi = run_analysis(p, f)
        out[prec] = W
        err = _per_scale_err(W[:, :, rows, :], Wo)
        assert err.max() < (1e-11 if prec == "fp64" else 1e-5), (prec, err)
        # scaling coefficients vanish: C_0 = C_1 = 0 and Phi lives on l = 0 only
        assert np.abs(Wphi).max() < 1e-12
        p.close()
    # mixed against float64 on the whole arrays, per scale
    W64, Wm = out["fp64"], out["mixed"]
    nz = [j for j in range(W64.shape[0]) if np.abs(W64[j]).max() > 0]
    e = max(np.abs(Wm[j] - W64[j]).max() / np.abs(W64[j]).max() for j in nz)
    assert e < 1e-5


@pytest.mark.parametrize("L", [256, 1024])
def test_synthesis_spot_modes_and_round_trip(L):
    N, lam, J0 = 5, 2.0, 0
    J = O.n_scales(L, lam, J0)
    W, Wphi = w_random(L, N, J + 1, 7 + L)
    lm = [(0, 0), (1, 1), (5, 3), (L // 2, 0), (L // 2, 17), (L - 1, L - 1), (L - 1, 2)]
    kern = O.kernels(L, N, lam, J0)
    ref = O.synthesis_modes(W, Wphi, L, N, lam, J0, lm, kern)
    scale = max(abs(v) for v in ref.values())
    for prec in ("fp64", "mixed"):
        p = B.Plan(L, N, lam, J0, prec)
        f = run_synthesis(p, W, Wphi)
        for (l, m), v in ref.items():
            tol = 1e-11 if prec == "fp64" else 1e-5
            assert abs(f[l * l + l + m] - v) < tol * scale, (prec, l, m)
        # exact round trip (Sec. 3.4 metric) of a signal
        fs = flm_gaussian(L, 3, "cl")
        Wd, Wpd = run_analysis(p, fs)
        fr = run_synthesis(p, Wd, Wpd)
        eps = np.abs(fr - fs).max() / np.abs(fs).max()
        assert eps < (1e-12 if prec == "fp64" else 1e-5), (prec, eps)
        p.close()


def test_batch_workload_64_signals():
    """64 real signals, L from {64,128,256,512}, N from {1,3,5}: one batched
    launch set equals the single runs, and every round trip is exact."""
    import torch
    rng = np.random.default_rng(3)
    Ls = rng.choice([64, 128, 256, 512], 64)
    Ns = rng.choice([1, 3, 5], 64)
    plans = [B.Plan(int(L), int(N), 2.0, 0, "mixed") for L, N in zip(Ls, Ns)]
    fs = [torch.from_numpy(flm_gaussian(p.L, 300 + i, "cl")).to(torch.complex64).cuda() for i, p in enumerate(plans)]
    Ws = [p.alloc_w() for p in plans]
    B.s2dw_analysis_batch([p.handle for p in plans], fs, [w[0] for w in Ws], [w[1] for w in Ws])
    fr = [p.alloc_flm() for p in plans]
    B.s2dw_synthesis_batch([p.handle for p in plans], [w[0] for w in Ws], [w[1] for w in Ws], fr)
    torch.cuda.synchronize()
    for i in (0, 17, 63):
        p = plans[i]
        W1, Wp1 = p.alloc_w()
        p.analysis(fs[i], W1, Wp1)
        torch.cuda.synchronize()
        assert torch.equal(W1, Ws[i][0])
    for i, p in enumerate(plans):
        ref = flm_gaussian(p.L, 300 + i, "cl")
        eps = np.abs(fr[i].to(torch.complex128).cpu().numpy() - ref).max() / np.abs(ref).max()
        assert eps < 1e-5
    # one member against the oracle on a beta row
    i = int(np.argmin(Ls))
    p = plans[i]
    Wo, _, _ = O.analysis_rows(flm_gaussian(p.L, 300 + i, "cl"), p.L, p.N, 2.0, 0, [5])
    got = Ws[i][0][:, :, [5], :].double().cpu().numpy()
    nz = [j for j in range(Wo.shape[0]) if np.abs(Wo[j]).max() > 0]
    assert max(np.abs(got[j] - Wo[j]).max() / np.abs(Wo[j]).max() for j in nz) < 1e-5
    for p in plans:
        p.close()
