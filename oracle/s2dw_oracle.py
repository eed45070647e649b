"""Plain, slow, float64 CPU oracle (test infrastructure only; never product code).

Every function states the passage of McEwen, Vandergheynst & Wiaux (2013) it
writes out.  Equation numbers follow the order of the paper's displayed
equations: (1) analysis, (3) scaling analysis, (4) synthesis, (6)
admissibility, (7) factorised wavelet, (11) directionality coefficients,
(12)-(16) kernel construction, (17)-(19) quadrature, (20) harmonic analysis,
(24)-(25) Wigner decomposition and Fourier expansion, (27) Fourier cube,
(31) scaling harmonics, (32)-(33) harmonic synthesis, (41) scaling synthesis.

Index conventions (shared with the C ABI, by specification only):
  * f_lm is a flat array indexed l*l + l + m, |m| <= l < L.
  * n_k = -(N-1) + 2k, k = 0..N-1: the azimuthal orders with s_ln != 0.
  * W has shape [J+1][N][2L][2L-1] = [scale j][gamma g][beta b][alpha a].
  * W^Phi has shape [2L][2L-1] = [theta t][phi p].
  * On the grid of mw_betas (L beta samples) the beta axes have L entries.
"""
from __future__ import annotations

import functools
import math
import warnings

import numpy as np
from scipy import integrate

__all__ = [
    "PARITY", "j_max", "n_scales", "n_orders", "bump", "s_lambda", "k_lambda",
    "kappa_lambda", "kappa", "phi_l", "s_dir", "kernels", "dh_weights", "grids",
    "wigner_d", "delta", "flm_to_grid", "grid_to_flm", "analysis",
    "analysis_rows", "synthesis", "synthesis_modes", "fourier_cube",
    "support", "steer", "sht_inverse", "sht_forward",
    "band_limits", "analysis_multires", "synthesis_multires",
    "mw_betas", "analysis_mw", "resample_mw_to_dh", "synthesis_mw",
]

# How each public function is pinned to something other than itself (tests
# named in tests/test_oracle_pins.py; planted mistakes in
# tests/test_oracle_mutations.py).  No function is "parity unpinned".
PARITY = {
    "j_max": "closed values from the definition in Sec. 2.2 (L=1024, lam=2 -> 10; L=1000, lam=3 -> 7)",
    "n_scales": "closed values J = J_max - J0 and the J0 > J_max error",
    "n_orders": "closed order lists of Eq. (11) for N = 1, 4, 5",
    "bump": "admissibility Eq. (6) and the k_lambda derivative pin (s^2 enters both)",
    "s_lambda": "k_lambda derivative -s_lam^2/t/I(1/lam) by finite differences; support ends of kappa",
    "kappa_lambda": "peak of unity at t = 1 (kappa^j(lam^-j L) = 1); admissibility Eq. (6)",
    "kappa": "hand-typed supports of Sec. 2.2 (tests/golden/supports_*.txt): zero at and outside the ends",
    "phi_l": "admissibility Eq. (6); band-limit of Phi derived by hand",
    "s_dir": "explicit s_ln values and sum_n |s_ln|^2 = 1 (Eq. (8))",
    "grids": "single-mode closed-form D at the grid samples (planted 2L-point alpha / 2pi gamma grids caught)",
    "flm_to_grid": "index placement of a single mode; inverse of grid_to_flm",
    "grid_to_flm": "inverse of flm_to_grid",
    "analysis_rows": "the rows of analysis (same pins: closed-form D, realness, steerability)",
    "synthesis_modes": "exact round trip at every (l, m) with the scaling term live; equals synthesis on arbitrary arrays",
    "fourier_cube": "Eq. (26) applied to the cube reproduces the (pinned) analysis",
    "support": "hand-typed values of the Sec. 2.2 formula at L=1024, lam=2 and L=100, lam=3",
    "band_limits": "closed values derived by hand at L=1024, lam=2 and L=100, lam=3 (J0 = 0, 1)",
    "k_lambda": "limits k=1 below 1/lam, 0 above 1; derivative vs -s^2/t/I by finite differences",
    "kernels": "admissibility Eq. (6); sum_n |s_ln|^2 = 1 (Eq. (8)); support edges (Sec. 2.2)",
    "dh_weights": "sum q = 2; exact integration of sin(t)cos(kt), k < 2L (Eq. (17))",
    "wigner_d": "textbook closed forms at l=1,2; Wigner's explicit sum in 60-digit arithmetic; orthogonality up to l=2047",
    "delta": "symmetries of d(pi/2); Fourier expansion Eq. (25) reproduces d(beta)",
    "analysis": "single-mode closed-form D at l=1,2; realness for real signals; steerability Eq. (10)",
    "synthesis": "exact round trip with analysis (Sec. 3.4 metric) to 1e-12",
    "steer": "reproduces the samples at gamma = gamma_g; equals the direct sum of Eq. (20) at off-grid gamma",
    "sht_inverse": "textbook Y_lm (Condon-Shortley) at l <= 2; exact round trip with sht_forward",
    "sht_forward": "textbook Y_lm maps give unit coefficients; exact round trip with sht_inverse",
    "analysis_multires": "equals the full-resolution W at the samples the two grids share; exact round trip",
    "synthesis_multires": "exact round trip with analysis_multires (Sec. 3.4 metric)",
    "mw_betas": "closed values (last sample beta = pi)",
    "analysis_mw": "closed-form D^l_mn at the MW beta samples (l <= 2)",
    "resample_mw_to_dh": "equals the DH analysis of the same signal (exact resampling)",
    "synthesis_mw": "exact round trip with analysis_mw (Sec. 3.4 metric)",
}


# ---------------------------------------------------------------------------
# Scales and kernels (Sec. 2.2)
# ---------------------------------------------------------------------------

def j_max(L: int, lam: float) -> int:
    """Largest useful scale J_L(lam) = ceil(log_lam L) (Sec. 2.2): the smallest
    integer J with lam**-J * L <= 1, found by an integer loop."""
    J, p = 0, 1.0
    while p < L:
        p *= lam
        J += 1
    return J


def n_scales(L: int, lam: float, J0: int) -> int:
    """J = J_max - J0 (scales j = 0..J); J0 counts the coarse scales left to
    the scaling function."""
    J = j_max(L, lam) - J0
    if J < 0:
        raise ValueError("J0 exceeds J_max")
    return J


def n_orders(N: int) -> np.ndarray:
    """Azimuthal orders n with beta_(N,n) = 1 and |n| < N (Sec. 2.2, Eq. (11))."""
    return np.arange(-(N - 1), N, 2)


def bump(x):
    """s(x) = exp(-(1-x^2)^-1) on (-1, 1), zero outside (Sec. 2.2, Eq. (12))."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    inside = np.abs(x) < 1.0
    out[inside] = np.exp(-1.0 / (1.0 - x[inside] ** 2))
    return out


def s_lambda(t, lam: float):
    """s_lam(t) = s(2 lam/(lam-1) (t - 1/lam) - 1), support [1/lam, 1] (Eq. (12))."""
    t = np.asarray(t, dtype=np.float64)
    return bump(2.0 * lam / (lam - 1.0) * (t - 1.0 / lam) - 1.0)


@functools.lru_cache(maxsize=None)
def _I(t: float, lam: float) -> float:
    """I(t) = int_t^1 s_lam(u)^2 / u du by adaptive Gauss-Kronrod (QUADPACK)."""
    return _Iab(max(t, 1.0 / lam), 1.0, lam)


@functools.lru_cache(maxsize=None)
def _Iab(lo: float, hi: float, lam: float) -> float:
    """int_lo^hi s_lam(u)^2 / u du (adaptive Gauss-Kronrod), 0 if lo >= hi."""
    lo = max(lo, 1.0 / lam)
    hi = min(hi, 1.0)
    if lo >= hi:
        return 0.0
    c = 2.0 * lam / (lam - 1.0)

    def f(u):
        x = c * (u - 1.0 / lam) - 1.0
        if abs(x) >= 1.0:
            return 0.0
        return math.exp(-2.0 / (1.0 - x * x)) / u

    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, _ = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1.2e-14, limit=1000)
    return val


def k_lambda(t: float, lam: float) -> float:
    """k_lam(t) = I(t) / I(1/lam) (Eq. (13)); 1 for t < 1/lam, 0 for t > 1."""
    t = float(t)
    if t <= 1.0 / lam:
        return 1.0
    if t >= 1.0:
        return 0.0
    return _I(t, lam) / _I(1.0 / lam, lam)


def kappa_lambda(t: float, lam: float) -> float:
    """kappa_lam(t) = sqrt(k_lam(t/lam) - k_lam(t)) (Eq. (14)).

    By Eq. (13) the difference is one integral,
      k_lam(t/lam) - k_lam(t) = int_{t/lam}^{t} s_lam(u)^2/u du / I(1/lam)
    (limits clipped to the support [1/lam, 1]); it is evaluated in that form,
    which avoids the cancellation of two numbers near 1 at the support edges."""
    t = float(t)
    return math.sqrt(_Iab(t / lam, t, lam) / _I(1.0 / lam, lam))


def kappa(j: int, l: int, L: int, lam: float) -> float:
    """kappa^j(l) = kappa_lam(lam^j l / L) (Eq. (15))."""
    return kappa_lambda(lam ** j * l / L, lam)


def phi_l(l: int, L: int, lam: float, J: int) -> float:
    """Phi_l0 = sqrt(k_lam(lam^J l / L)) (Eq. (16))."""
    return math.sqrt(k_lambda(lam ** J * l / L, lam))


def support(j: int, L: int, lam: float):
    """Support of kappa^j quoted in Sec. 2.2: [floor(lam^-(1+j) L), ceil(lam^(1-j) L)]."""
    return math.floor(lam ** (-(1 + j)) * L), math.ceil(lam ** (1 - j) * L)


def s_dir(l: int, n: int, N: int) -> complex:
    """Directionality coefficient s_ln (Eq. (11)):
    eta_N beta_(N,n) sqrt(2^-gamma C(gamma, (gamma-n)/2)), gamma = gamma_(N,l).
    s_0n = 0 (zero-mean condition of Sec. 2.2); the binomial is 0 outside
    0..gamma or for a non-integer lower index."""
    if l == 0:
        return 0.0
    eta = 1.0 if (N - 1) % 2 == 0 else 1j
    beta = (1 - (-1) ** (N + n)) // 2
    gamma = min(N - 1, l - (1 + (-1) ** (N + l)) // 2)
    if beta == 0 or (gamma - n) % 2 != 0:
        return 0.0
    k = (gamma - n) // 2
    if k < 0 or k > gamma:
        return 0.0
    return eta * math.sqrt(2.0 ** (-gamma) * math.comb(gamma, k))


def kernels(L: int, N: int, lam: float, J0: int):
    """Psi^j_ln = kappa^j(l) s_ln (Eq. (7)) for n = n_k, and Phi_l0 (Eq. (16)).

    Returns psi complex [J+1][L][N] and phi real [L]."""
    J = n_scales(L, lam, J0)
    ns = n_orders(N)
    psi = np.zeros((J + 1, L, N), dtype=np.complex128)
    for j in range(J + 1):
        for l in range(L):
            kj = kappa(j, l, L, lam)
            if kj == 0.0:
                continue
            for k, n in enumerate(ns):
                psi[j, l, k] = kj * s_dir(l, int(n), N)
    phi = np.array([phi_l(l, L, lam, J) for l in range(L)])
    return psi, phi


# ---------------------------------------------------------------------------
# Sampling and quadrature (Sec. 3.1)
# ---------------------------------------------------------------------------

def grids(L: int, N: int):
    """alpha_a = 2 pi a/(2L-1) (a < 2L-1), beta_b = pi(2b+1)/(4L) (b < 2L),
    gamma_g = pi g / N (g < N) (Sec. 3.1)."""
    alpha = 2.0 * np.pi * np.arange(2 * L - 1) / (2 * L - 1)
    beta = np.pi * (2 * np.arange(2 * L) + 1) / (4 * L)
    gamma = np.pi * np.arange(N) / N
    return alpha, beta, gamma


def dh_weights(L: int) -> np.ndarray:
    """q(theta_t) = (2/L) sin(theta_t) sum_{k<L} sin((2k+1) theta_t)/(2k+1) (Eq. (18))."""
    _, theta, _ = grids(L, 1)
    k = np.arange(L)
    s = np.sin(np.outer(theta, 2 * k + 1)) / (2 * k + 1)
    return 2.0 / L * np.sin(theta) * s.sum(axis=1)


# ---------------------------------------------------------------------------
# Wigner d-functions (convention of Eq. (24): D = e^{-im alpha} d e^{-in gamma})
# ---------------------------------------------------------------------------

def _d_first_log(beta, m, n):
    """d^{l0}_{mn}(beta) at l0 = max(|m|, |n|), where Wigner's explicit sum has
    a single term:  d^l_{l,n} = (-1)^{l-n} sqrt(C(2l, l+n)) c^{l+n} s^{l-n},
    d^l_{-l,n} = sqrt(C(2l, l-n)) c^{l-n} s^{l+n}, c = cos(beta/2),
    s = sin(beta/2); the case |n| > |m| uses d_mn = (-1)^{m-n} d_nm."""
    beta, m, n = np.broadcast_arrays(np.asarray(beta, np.float64), np.asarray(m), np.asarray(n))
    swap = np.abs(n) > np.abs(m)
    mm = np.where(swap, n, m)
    nn = np.where(swap, m, n)
    sign = np.where(swap & ((m - n) % 2 == 1), -1.0, 1.0)
    l0 = np.abs(mm)
    pos = mm >= 0
    a = np.where(pos, l0 + nn, l0 - nn)           # power of cos(beta/2)
    b = np.where(pos, l0 - nn, l0 + nn)           # power of sin(beta/2)
    sign = sign * np.where(pos & ((l0 - nn) % 2 == 1), -1.0, 1.0)
    logc = np.vectorize(lambda L2, A: math.log(math.comb(int(L2), int(A))), otypes=[float])(2 * l0, a)
    c = np.cos(beta / 2.0)
    s = np.sin(beta / 2.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        tc = np.where(a == 0, 0.0, a * np.log(c))
        ts = np.where(b == 0, 0.0, b * np.log(s))
    return sign, 0.5 * logc + tc + ts     # d = sign * exp(log|d|), log|d| may be -inf


def wigner_d(beta, L: int, m, n) -> np.ndarray:
    """d^l_{mn}(beta) for l = 0..L-1 (zero where l < max(|m|,|n|)).

    beta, m, n broadcast together; the result has shape (L,) + that shape.
    From the first nonzero degree the textbook three-term recurrence in l
    (Varshalovich et al. 1989, Sec. 4.8) is run forward:
      l sqrt(((l+1)^2-m^2)((l+1)^2-n^2)) d^{l+1}
        = (2l+1)(l(l+1) cos(beta) - m n) d^l - (l+1) sqrt((l^2-m^2)(l^2-n^2)) d^{l-1}.
    """
    beta, m, n = np.broadcast_arrays(np.asarray(beta, np.float64), np.asarray(m), np.asarray(n))
    m = m.astype(np.int64)
    n = n.astype(np.int64)
    l0 = np.maximum(np.abs(m), np.abs(n))
    # The first value can lie far below the float64 range (e.g. ~e^-750 at
    # l ~ 1400, beta = pi/2) while later degrees are O(1): the recurrence is
    # linear, so it runs on values scaled by exp(-E) with E tracked per entry.
    sgn, logd = _d_first_log(beta, m, n)
    fin = np.isfinite(logd)
    E = np.where(fin, np.floor(np.where(fin, logd, 0.0)), 0.0)
    first = np.where(fin, sgn * np.exp(np.where(fin, logd, 0.0) - E), 0.0)
    cb = np.cos(beta)
    mf = m.astype(np.float64)
    nf = n.astype(np.float64)
    out = np.zeros((L,) + beta.shape)
    prev2 = np.zeros(beta.shape)
    prev = np.zeros(beta.shape)
    for l in range(L):
        if l == 0:
            cur = np.zeros(beta.shape)
        else:
            lp = l - 1  # recurrence written for degree lp -> lp + 1 = l
            with np.errstate(divide="ignore", invalid="ignore"):
                lhs = lp * np.sqrt(np.maximum((lp + 1) ** 2 - mf ** 2, 0) * np.maximum((lp + 1) ** 2 - nf ** 2, 0))
                t1 = (2 * lp + 1) * (lp * (lp + 1) * cb - mf * nf) * prev
                t2 = (lp + 1) * np.sqrt(np.maximum(lp ** 2 - mf ** 2, 0) * np.maximum(lp ** 2 - nf ** 2, 0)) * prev2
                cur = (t1 - t2) / lhs
            # degree 1 from degree 0 (m = n = 0): d^1_00 = cos(beta)
            if lp == 0:
                cur = np.where(l0 == 0, cb, cur)
            cur = np.where(l > l0, cur, 0.0)
        cur = np.where(l == l0, first, cur)
        with np.errstate(under="ignore", over="ignore"):
            out[l] = cur * np.exp(E)
        prev2, prev = prev, cur
        big = np.abs(prev) > 1e100
        if np.any(big):
            prev = np.where(big, prev * 1e-100, prev)
            prev2 = np.where(big, prev2 * 1e-100, prev2)
            E = np.where(big, E + 100.0 * np.log(10.0), E)
    return out


def delta(L: int, mp, m) -> np.ndarray:
    """Delta^l_{m'm} = d^l_{m'm}(pi/2) (Sec. 3.2, below Eq. (25)) for l < L."""
    return wigner_d(np.pi / 2, L, mp, m)


# ---------------------------------------------------------------------------
# Harmonic-coefficient layout
# ---------------------------------------------------------------------------

def flm_to_grid(flm: np.ndarray, L: int) -> np.ndarray:
    """Flat f[l*l + l + m] -> grid F[l, m + L - 1] (zero for |m| > l)."""
    F = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    for l in range(L):
        F[l, L - 1 - l:L + l] = flm[l * l:l * l + 2 * l + 1]
    return F


def grid_to_flm(F: np.ndarray, L: int) -> np.ndarray:
    out = np.zeros(L * L, dtype=np.complex128)
    for l in range(L):
        out[l * l:l * l + 2 * l + 1] = F[l, L - 1 - l:L + l]
    return out


# ---------------------------------------------------------------------------
# Analysis (Sec. 3.2)
# ---------------------------------------------------------------------------

def analysis_rows(flm, L: int, N: int, lam: float, J0: int, b_list, kern=None, betas=None):
    """Wavelet and scaling coefficients on the rows beta_b, b in b_list.

    W^j(alpha_a, beta_b, gamma_g) = sum_{l<L} sum_{|m|<=l} sum_{n=n_k}
        f_lm Psi^j*_ln e^{i m alpha_a} d^l_mn(beta_b) e^{i n gamma_g}
    is Eq. (20) with D^l*_mn from Eq. (24) on the SO(3) grid of Sec. 3.1.
    W^Phi(theta_t, phi_p) = sum_lm f_lm Phi_l0 e^{i m phi_p} d^l_m0(theta_t)
    is Eq. (3) with (R_omega Phi)_lm = D^l_m0(phi, theta, 0) Phi_l0.

    `betas` replaces the DH beta samples (b_list then indexes into it).
    Returns (W [J+1][N][len(b_list)][2L-1], Wphi [len(b_list)][2L-1],
    max |imag part| seen)."""
    psi, phi = kern if kern is not None else kernels(L, N, lam, J0)
    J1 = psi.shape[0]
    alpha, beta, gamma = grids(L, N)
    if betas is not None:
        beta = np.asarray(betas, np.float64)
    ns = n_orders(N)
    ms = np.arange(-(L - 1), L)
    F = flm_to_grid(np.asarray(flm, np.complex128), L)
    Ea = np.exp(1j * np.outer(ms, alpha))          # [m][a]
    Eg = np.exp(1j * np.outer(ns, gamma))          # [k][g]
    W = np.zeros((J1, N, len(b_list), 2 * L - 1))
    Wphi = np.zeros((len(b_list), 2 * L - 1))
    imag = 0.0
    for ib, b in enumerate(b_list):
        D = wigner_d(beta[b], L, ms[:, None], ns[None, :])        # [l][m][k]
        D0 = wigner_d(beta[b], L, ms, 0)                          # [l][m]
        for j in range(J1):
            T = np.einsum("lm,lk,lmk->mk", F, np.conj(psi[j]), D)
            Wag = Ea.T @ T @ Eg                                    # [a][g]
            imag = max(imag, float(np.abs(Wag.imag).max()))
            W[j, :, ib, :] = Wag.real.T
        Tphi = np.einsum("lm,l,lm->m", F, phi, D0)
        wp = Tphi @ Ea
        imag = max(imag, float(np.abs(wp.imag).max()))
        Wphi[ib] = wp.real
    return W, Wphi, imag


def analysis(flm, L: int, N: int, lam: float, J0: int, kern=None):
    """Full analysis on every beta row (see analysis_rows)."""
    W, Wphi, _ = analysis_rows(flm, L, N, lam, J0, range(2 * L), kern)
    return W, Wphi


def fourier_cube(flm, L: int, N: int, lam: float, J0: int, j: int, kern=None):
    """U_{m m' n} = e^{i(n-m)pi/2} sum_l Delta^l_{m'm} Delta^l_{m'n} f_lm Psi^j*_ln
    (Eq. (27)) for m, m' in (-L, L), n = n_k: array [m][m'][k]."""
    psi, _ = kern if kern is not None else kernels(L, N, lam, J0)
    ns = n_orders(N)
    ms = np.arange(-(L - 1), L)
    F = flm_to_grid(np.asarray(flm, np.complex128), L)
    Dmm = delta(L, ms[:, None], ms[None, :])          # [l][m'][m]
    Dmn = delta(L, ms[:, None], ns[None, :])          # [l][m'][k]
    U = np.einsum("lpm,lpk,lm,lk->mpk", Dmm, Dmn, F, np.conj(psi[j]))
    phase = np.exp(1j * (ns[None, :] - ms[:, None]) * np.pi / 2)   # [m][k]
    return U * phase[:, None, :]


# ---------------------------------------------------------------------------
# Synthesis (Sec. 3.3)
# ---------------------------------------------------------------------------

def _synth_factors(L, N):
    alpha, beta, gamma = grids(L, N)
    q = dh_weights(L)
    return alpha, beta, gamma, q


def synthesis(W, Wphi, L: int, N: int, lam: float, J0: int, kern=None, b_list=None):
    """f_lm from wavelet and scaling coefficients.

    Wavelet part, Eqs. (32)-(33):
      f_lm += sum_j sum_n (2l+1)/(8 pi^2) Psi^j_ln (W^j)^l_mn,
      (W^j)^l_mn = int_SO(3) W^j D^l_mn, evaluated exactly by the quadratures
      of Sec. 3.1: 2pi/(2L-1) sum_a (Eq. (19)), sum_b q(beta_b) (Eq. (17)),
      and 2pi z_n sum_g with z_n = 1/N over gamma_g in [0, pi) (Eq. (39)).
    b_list restricts the beta sum to those rows (a partial sum; default all).
    Scaling part, Eq. (41):
      f_lm += sqrt((2l+1)/4pi) W^Phi_lm Phi_l0, with
      W^Phi_lm = sqrt((2l+1)/4pi) int_S2 W^Phi e^{-im phi} d^l_m0(theta).
    """
    psi, phi = kern if kern is not None else kernels(L, N, lam, J0)
    J1 = psi.shape[0]
    alpha, beta, gamma, q = _synth_factors(L, N)
    ns = n_orders(N)
    ms = np.arange(-(L - 1), L)
    Ea = np.exp(-1j * np.outer(ms, alpha))         # [m][a]
    Eg = np.exp(-1j * np.outer(ns, gamma))         # [k][g]
    wa = 2.0 * np.pi / (2 * L - 1)
    wg = 2.0 * np.pi / N
    Fw = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    Fs = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    for b in (range(2 * L) if b_list is None else b_list):
        D = wigner_d(beta[b], L, ms[:, None], ns[None, :])        # [l][m][k]
        D0 = wigner_d(beta[b], L, ms, 0)                          # [l][m]
        for j in range(J1):
            E = Ea @ W[j][:, b, :].T @ Eg.T                        # [m][k]
            Fw += wa * wg * q[b] * np.einsum("lk,lmk,mk->lm", psi[j], D, E)
        Es = Ea @ Wphi[b]                                          # [m]
        Fs += wa * q[b] * (phi[:, None] * D0 * Es[None, :])
    ell = np.arange(L)[:, None]
    F = (2 * ell + 1) / (8 * np.pi ** 2) * Fw + (2 * ell + 1) / (4 * np.pi) * Fs
    return grid_to_flm(F, L)


def synthesis_modes(W, Wphi, L: int, N: int, lam: float, J0: int, lm_list, kern=None):
    """The synthesis of `synthesis` evaluated only at the (l, m) in lm_list
    (same sums; used for spot checks at large L)."""
    psi, phi = kern if kern is not None else kernels(L, N, lam, J0)
    J1 = psi.shape[0]
    alpha, beta, gamma, q = _synth_factors(L, N)
    ns = n_orders(N)
    wa = 2.0 * np.pi / (2 * L - 1)
    wg = 2.0 * np.pi / N
    Eg = np.exp(-1j * np.outer(ns, gamma))         # [k][g]
    out = {}
    by_m = {}
    for (l, m) in lm_list:
        by_m.setdefault(m, []).append(l)
    for m, ls in by_m.items():
        ea = np.exp(-1j * m * alpha)               # [a]
        lmax = max(ls) + 1
        D = wigner_d(beta[:, None], lmax, m, ns[None, :])          # [l][b][k]
        D0 = wigner_d(beta, lmax, m, 0)                            # [l][b]
        Es = Wphi @ ea                                             # [b]
        for l in ls:
            acc = 0.0 + 0.0j
            for j in range(J1):
                if not np.any(psi[j, l]):
                    continue
                E = np.einsum("gba,a,kg->bk", W[j], ea, Eg)         # [b][k]
                acc += wa * wg * np.sum(q[:, None] * psi[j, l][None, :] * D[l] * E) * (2 * l + 1) / (8 * np.pi ** 2)
            acc += wa * (2 * l + 1) / (4 * np.pi) * phi[l] * np.sum(q * D0[l] * Es)
            out[(l, m)] = acc
    return out


# ---------------------------------------------------------------------------
# Steerability (Sec. 2.2, Eq. (10))
# ---------------------------------------------------------------------------

def steer(W, N: int, gammas):
    """Wavelet coefficients at arbitrary orientations from the N samples:
    W(alpha, beta, gamma) = sum_{g<N} z(gamma - gamma_g) W(alpha, beta, gamma_g)
    (Eq. (10)), gamma_g = pi g / N (Sec. 3.1), with the interpolating function
    z(x) = sum_{n in S_N} z_n e^{i n x}, z_n = 1/N for the orders n_k of the
    even/odd kernels (Eq. (11)).

    W: [J+1][N][2L][2L-1] real; returns [J+1][len(gammas)][2L][2L-1]."""
    W = np.asarray(W, dtype=np.float64)
    ns = n_orders(N)
    gamma_g = np.pi * np.arange(N) / N
    gammas = np.asarray(gammas, dtype=np.float64)
    x = gammas[:, None] - gamma_g[None, :]                       # [t][g]
    z = np.real(np.exp(1j * x[:, :, None] * ns[None, None, :]).sum(axis=2)) / N
    return np.einsum("tg,jgba->jtba", z, W)


# ---------------------------------------------------------------------------
# Spherical harmonic transforms on the DH grid (Sec. 2.1, Sec. 3.1)
# ---------------------------------------------------------------------------

def _ylm_factor(L: int) -> np.ndarray:
    """sqrt((2l+1)/(4 pi)), the normalisation of Y_lm = sqrt((2l+1)/(4 pi))
    D^l*_m0(phi, theta, 0) (Sec. 2.1)."""
    return np.sqrt((2.0 * np.arange(L) + 1.0) / (4.0 * np.pi))


def sht_inverse(flm, L: int) -> np.ndarray:
    """f(theta_t, phi_p) = sum_{l<L} sum_{|m|<=l} f_lm Y_lm(theta_t, phi_p) on the
    DH sphere grid of Sec. 3.1 (theta_t = pi(2t+1)/(4L), t < 2L; phi_p =
    2 pi p/(2L-1)), Y_lm(theta, phi) = sqrt((2l+1)/(4 pi)) e^{i m phi} d^l_m0(theta).
    Returns the complex samples [2L][2L-1] (real for a real signal)."""
    phi, theta, _ = grids(L, 1)
    ms = np.arange(-(L - 1), L)
    F = flm_to_grid(np.asarray(flm, np.complex128), L) * _ylm_factor(L)[:, None]
    E = np.exp(1j * np.outer(ms, phi))                      # [m][p]
    out = np.zeros((2 * L, 2 * L - 1), dtype=np.complex128)
    for t in range(2 * L):
        d = wigner_d(theta[t], L, ms, 0)                    # [l][m]
        out[t] = (F * d).sum(axis=0) @ E
    return out


def sht_forward(fpix, L: int) -> np.ndarray:
    """f_lm = sum_{t, p} q_t (2 pi/(2L-1)) f(theta_t, phi_p) Y*_lm(theta_t, phi_p):
    the integral of f Y*_lm over the sphere by the DH quadrature of Eqs.
    (17)-(18), exact for band-limited f.  Returns the flat f[l*l + l + m]."""
    phi, theta, _ = grids(L, 1)
    q = dh_weights(L)
    ms = np.arange(-(L - 1), L)
    E = np.exp(-1j * np.outer(phi, ms)) * (2.0 * np.pi / (2 * L - 1))  # [p][m]
    F = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    fpix = np.asarray(fpix)
    for t in range(2 * L):
        G = fpix[t] @ E                                     # [m]
        d = wigner_d(theta[t], L, ms, 0)                    # [l][m]
        F += q[t] * d * G[None, :]
    F *= _ylm_factor(L)[:, None]
    # entries with |m| > l are exactly zero in d; keep only the valid ones
    return grid_to_flm(F, L)


# ---------------------------------------------------------------------------
# Multi-resolution sampling (Sec. 3.2 / 3.3 remark: a scale need not be
# transformed at the full band-limit)
# ---------------------------------------------------------------------------

def band_limits(L: int, N: int, lam: float, J0: int, kern=None):
    """Band-limit of every scale and of the scaling part: 1 + the largest l
    with a nonzero kernel (kappa^j(l) > 0, resp. Phi_l > 0); W^j and W^Phi are
    band-limited there, so the DH grid of that band-limit samples them
    exactly (at least 1)."""
    psi, phi = kern if kern is not None else kernels(L, N, lam, J0)
    Ls = []
    for j in range(psi.shape[0]):
        nz = np.nonzero(np.abs(psi[j]).max(axis=1) > 0)[0]
        Ls.append(int(nz[-1]) + 1 if nz.size else 1)
    nz = np.nonzero(phi > 0)[0]
    return Ls, (int(nz[-1]) + 1 if nz.size else 1)


def analysis_multires(flm, L: int, N: int, lam: float, J0: int, kern=None):
    """W^j on the SO(3) grid of its own band-limit L_j and W^Phi on the sphere
    grid of L_Phi: the sums of Eq. (20) / Eq. (3) (analysis_rows) with only the
    l < L_j that carry kernel weight.  Returns ([W^j: [N][2L_j][2L_j-1]],
    W^Phi: [2L_Phi][2L_Phi-1])."""
    psi, phi = kern if kern is not None else kernels(L, N, lam, J0)
    Ls, Lp = band_limits(L, N, lam, J0, (psi, phi))
    flm = np.asarray(flm, np.complex128)
    Ws = []
    for j, Lj in enumerate(Ls):
        W, _, _ = analysis_rows(flm[:Lj * Lj], Lj, N, lam, J0, range(2 * Lj),
                                (psi[j:j + 1, :Lj], np.zeros(Lj)))
        Ws.append(W[0])
    _, Wphi, _ = analysis_rows(flm[:Lp * Lp], Lp, N, lam, J0, range(2 * Lp),
                               (psi[:0, :Lp], phi[:Lp]))
    return Ws, Wphi


def synthesis_multires(Ws, Wphi, L: int, N: int, lam: float, J0: int, kern=None):
    """f_lm from multi-resolution coefficients: the synthesis of Eqs. (32)-(33)
    and (41) with each scale's integrals evaluated by the quadrature of its own
    grid (exact, the integrands being band-limited to L_j)."""
    psi, phi = kern if kern is not None else kernels(L, N, lam, J0)
    Ls, Lp = band_limits(L, N, lam, J0, (psi, phi))
    out = np.zeros(L * L, dtype=np.complex128)
    for j, Lj in enumerate(Ls):
        fj = synthesis(np.asarray(Ws[j])[None], np.zeros((2 * Lj, 2 * Lj - 1)), Lj, N, lam, J0,
                       (psi[j:j + 1, :Lj], np.zeros(Lj)))
        out[:Lj * Lj] += fj
    fs = synthesis(np.zeros((0, N, 2 * Lp, 2 * Lp - 1)), Wphi, Lp, N, lam, J0, (psi[:0, :Lp], phi[:Lp]))
    out[:Lp * Lp] += fs
    return out


# ---------------------------------------------------------------------------
# Sampling with L beta samples (the McEwen-Wiaux grid that Sec. 4
# names as the replacement of the DH grid): beta_b = pi(2b+1)/(2L-1), b < L
# (the last sample is beta = pi), alpha and gamma as in Sec. 3.1.
# ---------------------------------------------------------------------------

def mw_betas(L: int) -> np.ndarray:
    """beta_b = pi (2b+1)/(2L-1), b < L: half of the 2L-1 equispaced points
    of the beta torus [0, 2 pi), the other half being their reflections
    2 pi - beta."""
    return np.pi * (2 * np.arange(L) + 1) / (2 * L - 1)


def analysis_mw(flm, L: int, N: int, lam: float, J0: int, kern=None):
    """Eq. (20) / Eq. (3) sampled at the L beta values of mw_betas (the sums
    of analysis_rows at those beta).  Returns (W [J+1][N][L][2L-1],
    W^Phi [L][2L-1])."""
    W, Wphi, _ = analysis_rows(flm, L, N, lam, J0, range(L), kern, betas=mw_betas(L))
    return W, Wphi


def _mw_beta_to_dh(U, L: int, sigma, band=None):
    """Band-limited resampling in beta of U [..., L samples at mw_betas, ...]
    (axis -2) to the 2L DH samples: U is a trigonometric polynomial of degree
    < band (<= L) in beta with U(2 pi - beta) = sigma U(beta) (sigma
    broadcast over the other axes), so its L samples and their reflections
    are 2L-1 equispaced samples on the torus, whose discrete Fourier
    coefficients |p| < band give it exactly.  The last sample is its own
    reflection (beta = pi): where sigma = -1 a symmetric U vanishes there, and
    the sample is weighted by (1 + sigma)/2 (it is 0 for coefficients of a
    band-limited signal; for arbitrary ones this keeps the extension
    symmetric, i.e. c_{-p} = sigma c_p)."""
    n = 2 * L - 1
    band = L if band is None else band
    bet = np.pi * (2 * np.arange(n) + 1) / n                       # the whole torus
    U = np.array(U, dtype=np.complex128)
    U[..., L - 1, :] *= (1.0 + sigma[..., 0, :] if np.ndim(sigma) >= 2 else 1.0 + sigma) / 2.0
    ext = np.concatenate([U, sigma * U[..., L - 2::-1, :]], axis=-2)  # b >= L: reflection of n-1-b
    p = np.arange(-(band - 1), band)
    c = np.einsum("...bm,pb->...pm", ext, np.exp(-1j * np.outer(p, bet))) / n
    _, bdh, _ = grids(L, 1)
    return np.einsum("...pm,tp->...tm", c, np.exp(1j * np.outer(bdh, p)))


def resample_mw_to_dh(W, Wphi, L: int, N: int, bands=None):
    """Coefficients on the grid of mw_betas -> the same band-limited functions
    on the DH grid of Sec. 3.1 (exact): per (m, n) Fourier component in
    (alpha, gamma) the beta dependence sum_l c_l d^l_mn(beta) is a
    trigonometric polynomial of degree < L_j (the scale's band, l < L_j) with
    U(2 pi - beta) = (-1)^{m-n} U(beta) (d^l_mn(-beta) = (-1)^{m-n}
    d^l_mn(beta)); the scaling part has n = 0.  bands = ([L_j], L_Phi)
    (default: L for every part)."""
    alpha, _, gamma = grids(L, N)
    n = 2 * L - 1
    ms = np.arange(-(L - 1), L)
    ns = n_orders(N)
    Ea = np.exp(-1j * np.outer(alpha, ms)) / n                     # [a][m]: alpha Fourier coefficients
    Eg = np.exp(-1j * np.outer(gamma, ns)) / N                     # [g][k]: gamma coefficients (z_n = 1/N)
    W = np.asarray(W, np.float64)
    out = np.zeros(W.shape[:2] + (2 * L, n))
    sig = (-1.0) ** (ms[None, :] - ns[:, None])                    # [k][m]
    Ls, Lp = bands if bands is not None else ([L] * W.shape[0], L)
    for j in range(W.shape[0]):
        A = np.einsum("gba,am,gk->kbm", W[j], Ea, Eg)                # [k][b][m]
        Ad = _mw_beta_to_dh(A, L, sig[:, None, :], max(1, Ls[j]))   # [k][t][m]
        out[j] = np.einsum("ktm,am,gk->gta", Ad, np.exp(1j * np.outer(alpha, ms)),
                           np.exp(1j * np.outer(gamma, ns))).real
    A0 = np.asarray(Wphi, np.float64) @ Ea                         # [b][m]
    A0d = _mw_beta_to_dh(A0, L, ((-1.0) ** ms)[None, :], max(1, Lp))
    Wphi_dh = (A0d @ np.exp(1j * np.outer(ms, alpha))).real
    return out, Wphi_dh


def synthesis_mw(W, Wphi, L: int, N: int, lam: float, J0: int, kern=None):
    """f_lm from coefficients on the grid of mw_betas: the synthesis of
    Eqs. (32)-(33), (41) (exact on the DH grid) applied to the exact DH
    resampling of the coefficients (resample_mw_to_dh, each part within its
    band L_j; for coefficients that are not band-limited this is the
    projection onto the band)."""
    psi, phi = kern if kern is not None else kernels(L, N, lam, J0)
    Wd, Wpd = resample_mw_to_dh(W, Wphi, L, N, band_limits(L, N, lam, J0, (psi, phi)))
    return synthesis(Wd, Wpd, L, N, lam, J0, (psi, phi))
