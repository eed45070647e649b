"""The seeded input recipe: every generated signal is real on the sphere
(f_{l,-m} = (-1)^m conj(f_lm), f_l0 real), has the stated spectrum, and the
same seed gives the same array."""
import numpy as np
import pytest

from paper_1308_5706_gb300.inputs import flm_gaussian, flm_uniform, w_random


def _real_signal_symmetric(f, L):
    for l in range(L):
        b = l * l + l
        assert f[b].imag == 0.0
        for m in range(1, l + 1):
            assert f[b - m] == ((-1) ** m) * np.conj(f[b + m])


@pytest.mark.parametrize("gen", ["unit", "cl", "uniform"])
def test_real_signal_symmetry_and_seeding(gen):
    L = 24
    make = (lambda s: flm_uniform(L, s)) if gen == "uniform" else (lambda s: flm_gaussian(L, s, gen))
    f = make(5)
    assert f.shape == (L * L,) and f.dtype == np.complex128
    _real_signal_symmetric(f, L)
    assert np.array_equal(f, make(5))
    assert not np.array_equal(f, make(6))


def test_spectra():
    L = 400
    f = flm_gaussian(L, 2, "cl")
    assert np.all(f[:4] == 0)  # C_0 = C_1 = 0
    # E|f_lm|^2 = C_l = 1/(l(l+1)): the mean over 2l+1 orders of many l
    ls = np.arange(2, L)
    power = np.array([np.mean(np.abs(f[l * l:(l + 1) * (l + 1)]) ** 2) for l in ls])
    ratio = power * ls * (ls + 1.0)
    assert abs(ratio.mean() - 1.0) < 0.02
    g = flm_gaussian(L, 3, "unit")
    assert abs(np.mean(np.abs(g) ** 2) - 1.0) < 0.02
    u = flm_uniform(L, 4)
    assert np.abs(u.real).max() <= 1.0 and np.abs(u.imag).max() <= 1.0
    # Re, Im uniform on [-1, 1]: mean square 1/3 each
    pos = np.concatenate([u[l * l + l + 1:(l + 1) * (l + 1)] for l in range(1, L)])
    assert abs(np.mean(pos.real ** 2) - 1 / 3) < 0.01 and abs(np.mean(pos.imag ** 2) - 1 / 3) < 0.01


def test_w_random_shapes():
    W, Wp = w_random(8, 3, 4, seed=1)
    assert W.shape == (4, 3, 16, 15) and Wp.shape == (16, 15)
    W2, _ = w_random(8, 3, 4, seed=1, nb=8)
    assert W2.shape == (4, 3, 8, 15)
