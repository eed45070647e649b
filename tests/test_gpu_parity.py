"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances: float64 path 1e-11 normwise relative, mixed path 1e-5
(max|x - x_ref| / max|x_ref| per output array); round trip
eps = max|f_rec - f| <= 1e-12 (float64).
"""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian, flm_uniform, w_random
from tests.gpu_helpers import relerr, run_analysis, run_synthesis, torch_cuda

pytestmark = pytest.mark.gpu

TOL64, TOLMIX = 1e-11, 1e-5

SMALL = [  # (L, N, lam, J0, spectrum, seed)
    (32, 3, 2.0, 0, "unit", 0),       # small configuration of the workload set
    (32, 3, 2.0, 2, "unit", 1),       # scaling part active
    (16, 2, 2.0, 1, "unit", 2),       # eta = i
    (20, 1, 3.0, 0, "unit", 3),       # N = 1, lambda = 3, non power-of-two L
    (37, 4, 1.7, 1, "cl", 4),         # odd L, non-integer lambda
    (2, 1, 2.0, 0, "unit", 5),        # smallest band-limit
    (8, 8, 2.0, 0, "unit", 6),        # N = L
    (24, 5, 2.0, 4, "unit", 7),       # J0 = J_max - 1: two wavelet scales
]


@pytest.fixture(scope="module")
def cache():
    return {}


def _plan(L, N, lam, J0, prec):
    return B.Plan(L, N, lam, J0, prec)


@pytest.mark.parametrize("L,N,lam,J0,spec,seed", SMALL)
def test_kernels_match_oracle(L, N, lam, J0, spec, seed):
    torch_cuda()
    p = _plan(L, N, lam, J0, "fp64")
    psi, phi = p.kernels()
    psi_o, phi_o = O.kernels(L, N, lam, J0)
    assert psi.shape == psi_o.shape
    assert np.abs(psi - psi_o).max() < 1e-13
    assert np.abs(phi - phi_o).max() < 1e-13
    p.close()


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 5, 7, 31, 64, 257])
def test_delta_table(l):
    torch_cuda()
    p = _plan(max(l + 1, 2), 1, 2.0, 0, "fp64")
    D = p.delta_slab(l)
    ms = np.arange(l + 1)
    ref = O.delta(l + 1, ms[:, None], ms[None, :])[l]
    assert np.abs(D - ref).max() < 1e-13
    p.close()


@pytest.mark.parametrize("l", [1023, 2047])
def test_delta_table_large_sampled(l):
    torch_cuda()
    p = _plan(l + 1, 1, 2.0, 0, "fp64")
    D = p.delta_slab(l)
    rng = np.random.default_rng(l)
    mp = rng.integers(0, l + 1, 300)
    m = rng.integers(0, l + 1, 300)
    mp[:4] = [0, l, l, 0]
    m[:4] = [0, l, 0, l]
    ref = O.delta(l + 1, mp, m)[l]
    assert np.abs(D[mp, m] - ref).max() < 1e-12
    # orthogonality of the full matrix (Delta_{-m',m} = (-1)^(l+m) Delta_{m'm})
    full = np.vstack([D[1:][::-1] * ((-1.0) ** (l + np.arange(l + 1)))[None, :], D])
    assert np.abs(full.T @ full - np.eye(l + 1)).max() < 1e-11
    p.close()


def _flm(L, spec, seed):
    return flm_uniform(L, seed) if spec == "uniform" else flm_gaussian(L, seed, spec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,N,lam,J0,spec,seed", SMALL)
def test_analysis_vs_oracle(L, N, lam, J0, spec, seed, prec):
    f = _flm(L, spec, seed)
    p = _plan(L, N, lam, J0, prec)
    W, Wphi = run_analysis(p, f)
    Wo, Wpo = O.analysis(f, L, N, lam, J0)
    tol = TOL64 if prec == "fp64" else TOLMIX
    for j in range(W.shape[0]):
        assert relerr(W[j], Wo[j]) < tol, (j, relerr(W[j], Wo[j]))
    if np.abs(Wpo).max() > 0:
        assert relerr(Wphi, Wpo) < tol
    else:
        assert np.abs(Wphi).max() < 1e-12
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,N,lam,J0,spec,seed", SMALL)
def test_synthesis_vs_oracle(L, N, lam, J0, spec, seed, prec):
    """Synthesis of arbitrary real coefficients (not in the range of the analysis)."""
    J = O.n_scales(L, lam, J0)
    W, Wphi = w_random(L, N, J + 1, 100 + seed)
    p = _plan(L, N, lam, J0, prec)
    f = run_synthesis(p, W, Wphi)
    fo = O.synthesis(W, Wphi, L, N, lam, J0)
    tol = TOL64 if prec == "fp64" else TOLMIX
    assert relerr(f, fo) < tol
    p.close()


@pytest.mark.parametrize("L,N,lam,J0,spec,seed", SMALL + [(64, 5, 2.0, 0, "cl", 9), (33, 3, 2.0, 0, "uniform", 10)])
def test_round_trip_fp64(L, N, lam, J0, spec, seed):
    f = _flm(L, spec, seed)
    p = _plan(L, N, lam, J0, "fp64")
    W, Wphi = run_analysis(p, f)
    fr = run_synthesis(p, W, Wphi)
    assert np.abs(fr - f).max() < 1e-12 * max(1.0, np.abs(f).max())
    p.close()


def test_stage_fourier_cube_fp64():
    """Contraction + gamma epilogue against the Fourier cube of Eq. (27)."""
    L, N, lam, J0 = 16, 3, 2.0, 0
    f = flm_gaussian(L, 21)
    p = _plan(L, N, lam, J0, "fp64")
    run_analysis(p, f)
    for j in range(p.nscale):
        lo, hi = p.support(j)
        Lj = hi + 1
        Y = p.stage(0, j).reshape(N, Lj, Lj)
        U = O.fourier_cube(f, L, N, lam, J0, j)          # [m][m'][k]
        ns = O.n_orders(N)
        gam = np.pi * np.arange(N) / N
        for g in range(N):
            ref = np.einsum("mpk,k->mp", U[L - 1:L - 1 + Lj, L - 1:L - 1 + Lj, :], np.exp(1j * ns * gam[g]))
            assert np.abs(Y[g] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    p.close()
