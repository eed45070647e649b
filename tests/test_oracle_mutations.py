"""Planted mistakes in the CPU oracle must make at least one pin fail.

Each case replaces one oracle function by a plausible wrong variant (a
transposed operand, a dropped term, a wrong sign or grid) and runs a set of
the pins of test_oracle_pins.py; the mistake must be caught.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.s2dw_oracle as OS
import tests.test_oracle_pins as P

_orig_wigner_d = OS.wigner_d
_orig_kernels = OS.kernels
_orig_dh = OS.dh_weights
_orig_grids = OS.grids
_orig_k = OS.k_lambda


def _wigner_transposed(beta, L, m, n):
    return _orig_wigner_d(beta, L, n, m)


_orig_rows = OS.analysis_rows
_orig_synth = OS.synthesis


def _analysis_noconj(flm, L, N, lam, J0, b_list, kern=None, **kw):
    psi, phi = kern if kern is not None else _orig_kernels(L, N, lam, J0)
    return _orig_rows(flm, L, N, lam, J0, b_list, (np.conj(psi), phi), **kw)


def _synthesis_conj(W, Wphi, L, N, lam, J0, kern=None):
    psi, phi = kern if kern is not None else _orig_kernels(L, N, lam, J0)
    return _orig_synth(W, Wphi, L, N, lam, J0, (np.conj(psi), phi))


def _dh_no_sin(L):
    _, theta, _ = _orig_grids(L, 1)
    k = np.arange(L)
    s = np.sin(np.outer(theta, 2 * k + 1)) / (2 * k + 1)
    return 2.0 / L * s.sum(axis=1)


def _grids_gamma_2pi(L, N):
    a, b, g = _orig_grids(L, N)
    return a, b, 2.0 * g


def _grids_alpha_2L(L, N):
    a, b, g = _orig_grids(L, N)
    return 2.0 * np.pi * np.arange(2 * L - 1) / (2 * L), b, g


def _k_bad_norm(t, lam):
    t = float(t)
    if t <= 1.0 / lam:
        return 1.0
    if t >= 1.0:
        return 0.0
    return OS._I(t, lam) / OS._I(1.0 / lam, lam) * 0.9


def _wigner_sign(beta, L, m, n):
    return _orig_wigner_d(beta, L, m, -np.asarray(n))


_orig_steer = OS.steer


def _steer_2pi_spacing(W, N, gammas):
    # samples taken as if gamma_g = 2 pi g / N (the full circle)
    W = np.asarray(W, dtype=np.float64)
    ns = OS.n_orders(N)
    x = np.asarray(gammas)[:, None] - 2 * np.pi * np.arange(N)[None, :] / N
    z = np.real(np.exp(1j * x[:, :, None] * ns[None, None, :]).sum(axis=2)) / N
    return np.einsum("tg,jgba->jtba", z, W)


def _steer_no_norm(W, N, gammas):
    return _orig_steer(W, N, gammas) * N


_orig_mw_to_dh = OS._mw_beta_to_dh


def _mw_reflection_unsigned(U, L, sigma, band=None):
    # reflection 2 pi - beta taken without the (-1)^{m-n} sign
    return _orig_mw_to_dh(U, L, np.ones_like(sigma), band)


def _mw_pole_unweighted(U, L, sigma, band=None):
    # the pole sample beta = pi counted as an ordinary sample (no (1 + sigma)/2 weight)
    n = 2 * L - 1
    band = L if band is None else band
    bet = np.pi * (2 * np.arange(n) + 1) / n
    U = np.array(U, dtype=np.complex128)
    ext = np.concatenate([U, sigma * U[..., L - 2::-1, :]], axis=-2)
    p = np.arange(-(band - 1), band)
    c = np.einsum("...bm,pb->...pm", ext, np.exp(-1j * np.outer(p, bet))) / n
    _, bdh, _ = OS.grids(L, 1)
    return np.einsum("...pm,tp->...tm", c, np.exp(1j * np.outer(bdh, p)))


_orig_modes = OS.synthesis_modes


def _modes_no_phi(W, Wphi, L, N, lam, J0, lm_list, kern=None):
    # the scaling term of Eq. (41) dropped
    return _orig_modes(W, np.zeros_like(Wphi), L, N, lam, J0, lm_list, kern)


def _modes_q_shifted(W, Wphi, L, N, lam, J0, lm_list, kern=None):
    # each beta row paired with the quadrature weight of its neighbour
    return _orig_modes(np.roll(W, 1, axis=2), np.roll(Wphi, 1, axis=0), L, N, lam, J0, lm_list, kern)


def _modes_wrong_2l1(W, Wphi, L, N, lam, J0, lm_list, kern=None):
    # the wavelet part scaled by (2l+1)/(4 pi) instead of (2l+1)/(8 pi^2)
    out = _orig_modes(W, np.zeros_like(Wphi), L, N, lam, J0, lm_list, kern)
    ph = _orig_modes(np.zeros_like(W), Wphi, L, N, lam, J0, lm_list, kern)
    return {k: v * 2 * np.pi + ph[k] for k, v in out.items()}


def _mw_betas_2L(L):
    return np.pi * (2 * np.arange(L) + 1) / (2 * L)


PINS = [
    lambda: P.test_single_mode_analysis_closed_form(3, 2.0, 0),
    lambda: P.test_single_mode_analysis_closed_form(2, 2.0, 1),
    lambda: P.test_single_mode_synthesis_closed_form(3),
    lambda: P.test_single_mode_synthesis_closed_form(4),
    lambda: P.test_round_trip_exact(8, 3, 2.0, 0, "unit"),
    lambda: P.test_round_trip_exact(16, 2, 2.0, 1, "uniform"),
    lambda: P.test_wigner_closed_forms(),
    lambda: P.test_dh_weights(5),
    lambda: P.test_k_lambda_limits_and_derivative(),
    lambda: P.test_realness_and_steerability(),
    lambda: P.test_steer_reproduces_samples(3),
    lambda: P.test_sht_round_trip_exact(9),
    lambda: P.test_sht_textbook_harmonics(1, 1),
    lambda: P.test_multires_round_trip_exact(16, 3, 2.0, 0),
    lambda: P.test_mw_single_mode_analysis_closed_form(3),
    lambda: P.test_mw_resampling_and_round_trip_exact(8, 3, 2.0, 0),
    lambda: P.test_mw_pole_only_component(1, True),
    lambda: P.test_synthesis_modes_round_trip_exact(8, 3, 2.0, 1),
]


@pytest.mark.parametrize("name,attr,bad", [
    ("transposed d operand", "wigner_d", _wigner_transposed),
    ("analysis without conj(Psi)", "analysis_rows", _analysis_noconj),
    ("synthesis with conj(Psi)", "synthesis", _synthesis_conj),
    ("DH weights without sin(theta)", "dh_weights", _dh_no_sin),
    ("gamma grid on [0, 2pi)", "grids", _grids_gamma_2pi),
    ("alpha grid 2L points", "grids", _grids_alpha_2L),
    ("k_lambda normalisation", "k_lambda", _k_bad_norm),
    ("sign of n in d", "wigner_d", _wigner_sign),
    ("steering samples on [0, 2pi)", "steer", _steer_2pi_spacing),
    ("steering without z_n = 1/N", "steer", _steer_no_norm),
    ("MW reflection without its sign", "_mw_beta_to_dh", _mw_reflection_unsigned),
    ("MW beta grid of spacing pi/L", "mw_betas", _mw_betas_2L),
    ("MW pole sample without the (1 + sigma)/2 weight", "_mw_beta_to_dh", _mw_pole_unweighted),
    ("per-mode synthesis without the scaling term", "synthesis_modes", _modes_no_phi),
    ("per-mode synthesis with q_b of the next row", "synthesis_modes", _modes_q_shifted),
    ("per-mode synthesis with (2l+1)/(4 pi) on the wavelet part", "synthesis_modes", _modes_wrong_2l1),
])
def test_planted_mistake_is_caught(monkeypatch, name, attr, bad):
    monkeypatch.setattr(OS, attr, bad)
    monkeypatch.setattr(O, attr, bad, raising=False)
    OS._I.cache_clear()
    caught = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, KeyError, ValueError, IndexError):
            caught += 1
    assert caught > 0, f"planted mistake '{name}' passed every pin"
