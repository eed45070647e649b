"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module holds random-number generation and array layout only: none of the
transform's arithmetic.  All generators use numpy's PCG64 with an explicit
seed, so the GPU path and the CPU oracle see identical inputs.

Workload recipe (the paper's experiments are synthetic too, Sec. 3.4):
  * "unit": f_lm complex Gaussian with E|f_lm|^2 = 1;
  * "cl":   E|f_lm|^2 = C_l with C_l = 1/(l(l+1)) for l >= 2, C_0 = C_1 = 0;
  * "uniform": Re and Im uniform in [-1, 1] (the Sec. 3.4 experiment), made
    real-signal symmetric;
every signal is real on the sphere: f_{l,-m} = (-1)^m conj(f_lm), f_l0 real.
For m > 0, Re and Im are each drawn with half the variance; f_l0 carries the
full variance.
"""
from __future__ import annotations

import numpy as np


def _spectrum(L: int, kind: str) -> np.ndarray:
    ell = np.arange(L, dtype=np.float64)
    if kind == "unit":
        return np.ones(L)
    if kind == "cl":
        c = np.zeros(L)
        c[2:] = 1.0 / (ell[2:] * (ell[2:] + 1.0))
        return c
    raise ValueError(kind)


def flm_gaussian(L: int, seed: int, spectrum: str = "unit") -> np.ndarray:
    """Real-signal Gaussian harmonic coefficients, flat index l*l + l + m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cl = _spectrum(L, spectrum)
    f = np.zeros(L * L, dtype=np.complex128)
    for l in range(L):
        sd = np.sqrt(cl[l])
        base = l * l + l
        f[base] = rng.standard_normal() * sd
        if l > 0:
            re = rng.standard_normal(l) * sd / np.sqrt(2.0)
            im = rng.standard_normal(l) * sd / np.sqrt(2.0)
            pos = re + 1j * im
            m = np.arange(1, l + 1)
            f[base + m] = pos
            f[base - m] = ((-1.0) ** m) * np.conj(pos)
    return f


def flm_uniform(L: int, seed: int) -> np.ndarray:
    """Re, Im uniform in [-1, 1] for m > 0, f_l0 uniform real, real-signal symmetric."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = np.zeros(L * L, dtype=np.complex128)
    for l in range(L):
        base = l * l + l
        f[base] = rng.uniform(-1.0, 1.0)
        if l > 0:
            pos = rng.uniform(-1.0, 1.0, l) + 1j * rng.uniform(-1.0, 1.0, l)
            m = np.arange(1, l + 1)
            f[base + m] = pos
            f[base - m] = ((-1.0) ** m) * np.conj(pos)
    return f


def w_random(L: int, N: int, n_scale: int, seed: int, nb: int = None):
    """Arbitrary real wavelet coefficients [n_scale][N][nb][2L-1] and scaling
    coefficients [nb][2L-1] (nb beta samples, default 2L), standard normal;
    inputs for synthesis-only checks."""
    nb = 2 * L if nb is None else nb
    rng = np.random.Generator(np.random.PCG64(seed))
    W = rng.standard_normal((n_scale, N, nb, 2 * L - 1))
    Wphi = rng.standard_normal((nb, 2 * L - 1))
    return W, Wphi


def flm_positive_m(f: np.ndarray, L: int) -> np.ndarray:
    """The m >= 0 half of a real-signal f_lm (layout only), flat l*l + l + m."""
    return f.copy()
