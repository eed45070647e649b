"""Pins of the CPU oracle to facts fixed by the paper and by textbook closed
forms (independent of the oracle's own code paths).  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300.inputs import flm_gaussian, flm_uniform

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- closed-form Wigner d (textbook, Varshalovich et al. 1989 Table 4.3) ----

def d_closed(l, m, n, b):
    """d^l_mn(beta) for l <= 2 from the tabulated closed forms; negative
    indices by d_mn = (-1)^(m-n) d_nm = d_{-n,-m}."""
    c, s = math.cos(b), math.sin(b)
    base = {
        (0, 0, 0): 1.0,
        (1, 1, 1): (1 + c) / 2, (1, 1, 0): -s / math.sqrt(2), (1, 1, -1): (1 - c) / 2,
        (1, 0, 0): c,
        (2, 2, 2): ((1 + c) / 2) ** 2, (2, 2, 1): -(1 + c) * s / 2,
        (2, 2, 0): math.sqrt(3.0 / 8.0) * s * s, (2, 2, -1): -(1 - c) * s / 2,
        (2, 2, -2): ((1 - c) / 2) ** 2,
        (2, 1, 1): (1 + c) * (2 * c - 1) / 2, (2, 1, 0): -math.sqrt(1.5) * s * c,
        (2, 1, -1): (1 - c) * (2 * c + 1) / 2, (2, 0, 0): (3 * c * c - 1) / 2,
    }
    for key, sign in (((l, m, n), 1.0), ((l, n, m), (-1.0) ** (m - n)),
                      ((l, -n, -m), 1.0), ((l, -m, -n), (-1.0) ** (m - n))):
        if key in base:
            return sign * base[key]
    raise KeyError((l, m, n))


def D_closed(l, m, n, a, b, g):
    """D^l_mn(alpha, beta, gamma) = e^{-im alpha} d^l_mn(beta) e^{-in gamma} (Eq. (24))."""
    return np.exp(-1j * m * a) * d_closed(l, m, n, b) * np.exp(-1j * n * g)


# --- scales and kernels (Sec. 2.2) -------------------------------------------

def test_jmax_values():
    assert O.j_max(1024, 2.0) == 10
    assert O.j_max(32, 2.0) == 5
    assert O.j_max(128, 2.0) == 7
    assert O.j_max(1000, 3.0) == 7          # 3^6 = 729 < 1000 <= 2187
    assert O.j_max(2, 2.0) == 1


@pytest.mark.parametrize("fname", ["supports_L1024_lam2.txt", "supports_L100_lam3.txt"])
def test_support_golden_and_kernel_zeros(fname):
    """Supports typed by hand from the Sec. 2.2 formulas (fixture headers show
    the arithmetic); kappa^j must vanish at the ends and peak at lam^-j L."""
    lines = open(os.path.join(GOLDEN, fname)).read().splitlines()
    L, lam = [(int(a.split("=")[1]), float(b.split("=")[1]))
              for a, b in (ln[2:].split() for ln in lines if ln.startswith("# L="))][0]
    rows = [ln.split() for ln in lines if ln and not ln.startswith("#")]
    assert rows[0][0] == "Jmax"
    assert O.j_max(L, lam) == int(rows[0][1])
    assert len(rows) - 1 == O.j_max(L, lam) + 1
    for j, lo, hi in ((int(a), int(b), int(c)) for a, b, c in rows[1:]):
        assert O.support(j, L, lam) == (lo, hi)
        # kappa^j vanishes at and outside the support ends, is positive inside
        for l in (lo, min(hi, L - 1) if hi < L else None):
            if l is not None and l < L:
                assert O.kappa(j, l, L, lam) == 0.0
        if lo > 0:
            assert O.kappa(j, lo - 1, L, lam) == 0.0
        mid = lam ** (-j) * L
        if 0 < mid < L and float(mid).is_integer():
            assert abs(O.kappa(j, int(mid), L, lam) - 1.0) < 1e-14     # peak of unity at lam^-j L
        # strictly inside the support kappa^j > 0 (checked a tenth of the way in;
        # right at the ends exp(-1/(1-x^2)) underflows in float64)
        inner = lo + max(1, (min(hi, L - 1) - lo) // 10)
        if inner < min(hi, L):
            assert O.kappa(j, inner, L, lam) > 0.0


def test_scale_counts_orders_and_band_limits():
    """Closed values derived by hand from Sec. 2.2: J = J_max - J0; the orders
    n with beta_(N,n) = 1, |n| < N (Eq. (11)); the band-limit of scale j is the
    upper support end ceil(lam^(1-j) L) clipped at L (kappa^j vanishes there and
    is positive just below), that of Phi the largest l with lam^J l / L < 1,
    plus one."""
    assert O.n_scales(1024, 2.0, 0) == 10 and O.n_scales(1024, 2.0, 3) == 7
    with pytest.raises(ValueError):
        O.n_scales(1024, 2.0, 11)
    assert list(O.n_orders(5)) == [-4, -2, 0, 2, 4]
    assert list(O.n_orders(4)) == [-3, -1, 1, 3]
    assert list(O.n_orders(1)) == [0]
    assert O.band_limits(1024, 5, 2.0, 0) == ([1024, 1024, 512, 256, 128, 64, 32, 16, 8, 4, 2], 1)
    # L = 100, lam = 3: hi = 300, 100, 34, 12, 4, 2 (supports_L100_lam3.txt);
    # Phi: 3^5 l / 100 < 1 -> l = 0 (J0 = 0); 3^4 l / 100 < 1 -> l <= 1 (J0 = 1)
    assert O.band_limits(100, 3, 3.0, 0) == ([100, 100, 34, 12, 4, 2], 1)
    assert O.band_limits(100, 3, 3.0, 1) == ([100, 100, 34, 12, 4], 2)


def test_flm_grid_layout():
    """f_lm sits at flat index l*l + l + m and at grid cell [l, m + L - 1]."""
    L = 5
    f = np.zeros(L * L, complex)
    f[3 * 3 + 3 - 2] = 1.0 + 2.0j                  # (l, m) = (3, -2)
    F = O.flm_to_grid(f, L)
    assert F[3, -2 + L - 1] == 1.0 + 2.0j and np.count_nonzero(F) == 1
    g = flm_gaussian(L, 1)
    assert np.array_equal(O.grid_to_flm(O.flm_to_grid(g, L), L), g)


def test_k_lambda_limits_and_derivative():
    for lam in (2.0, 3.0, 1.5):
        assert O.k_lambda(0.5 / lam, lam) == 1.0
        assert O.k_lambda(1.0 / lam, lam) == 1.0
        assert O.k_lambda(1.0, lam) == 0.0
        assert O.k_lambda(1.3, lam) == 0.0
        # I(1/lam) by an independent rule: composite Simpson on 200001 points
        u = np.linspace(1.0 / lam, 1.0, 200001)
        f = O.s_lambda(u, lam) ** 2 / u
        h = u[1] - u[0]
        I0 = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
        for t in np.linspace(1.0 / lam, 1.0, 9)[1:-1]:
            eps = 1e-5
            dk = (O.k_lambda(t + eps, lam) - O.k_lambda(t - eps, lam)) / (2 * eps)
            expect = -float(O.s_lambda(t, lam)) ** 2 / t / I0
            assert abs(dk - expect) < 1e-7 * max(1.0, abs(expect))
            # monotone decrease
            assert O.k_lambda(t, lam) > O.k_lambda(t + 0.01, lam)


def test_directionality_coefficients():
    for N in range(1, 9):
        ns = O.n_orders(N)
        for l in range(0, 20):
            vals = np.array([O.s_dir(l, int(n), N) for n in range(-l - 2, l + 3)])
            tot = float(np.sum(np.abs(vals) ** 2))
            if l == 0:
                assert tot == 0.0
            else:
                assert abs(tot - 1.0) < 1e-15
            for n in range(-l - 2, l + 3):
                if n not in ns:
                    assert O.s_dir(l, n, N) == 0.0
    # explicit values: N = 3 (eta = 1), l >= 2: gamma = 2
    assert O.s_dir(5, 2, 3) == pytest.approx(0.5, abs=1e-16)
    assert O.s_dir(5, 0, 3) == pytest.approx(math.sqrt(0.5), abs=1e-16)
    # N = 2 (eta = i), l >= 1: gamma = 1, n = +-1: i/sqrt(2)
    assert abs(O.s_dir(4, 1, 2) - 1j / math.sqrt(2)) < 1e-15
    # N = 3 at l = 1: gamma = min(2, 1 - 1) = 0 -> only n = 0, s = 1
    assert O.s_dir(1, 0, 3) == pytest.approx(1.0, abs=1e-16)
    assert O.s_dir(1, 2, 3) == 0.0


@pytest.mark.parametrize("L,N,lam,J0", [(32, 3, 2.0, 0), (64, 5, 2.0, 1), (50, 4, 3.0, 0),
                                        (40, 2, 1.5, 2), (128, 3, 2.0, 2), (1024, 5, 2.0, 0)])
def test_admissibility(L, N, lam, J0):
    psi, phi = O.kernels(L, N, lam, J0)
    total = phi ** 2 + (np.abs(psi) ** 2).sum(axis=(0, 2))
    # Eq. (6) for every l < L, including l = 0 (carried by Phi)
    assert np.abs(total - 1.0).max() < 2e-15


# --- quadrature (Sec. 3.1) ----------------------------------------------------

@pytest.mark.parametrize("L", [2, 5, 16, 33])
def test_dh_weights(L):
    q = O.dh_weights(L)
    _, theta, _ = O.grids(L, 1)
    assert abs(q.sum() - 2.0) < 1e-14
    for k in range(0, 2 * L):
        exact = 0.0 if k == 1 else (1 + math.cos(k * math.pi)) / (1 - k * k)
        assert abs(np.sum(q * np.cos(k * theta)) - exact) < 1e-13
    from scipy.special import eval_legendre
    x = np.cos(theta)
    for l in range(L):
        for lp in range(L):
            got = np.sum(q * eval_legendre(l, x) * eval_legendre(lp, x))
            assert abs(got - (2.0 / (2 * l + 1) if l == lp else 0.0)) < 1e-13


# --- Wigner d -----------------------------------------------------------------

def test_wigner_closed_forms():
    rng = np.random.default_rng(1)
    for b in rng.uniform(0.05, math.pi - 0.05, 7):
        for l in range(3):
            for m in range(-l, l + 1):
                for n in range(-l, l + 1):
                    got = O.wigner_d(b, l + 1, m, n)[l]
                    assert abs(got - d_closed(l, m, n, b)) < 1e-15, (l, m, n)


def test_wigner_explicit_sum_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60

    def wig(l, m, n, beta):
        c = mp.cos(mp.mpf(beta) / 2)
        s = mp.sin(mp.mpf(beta) / 2)
        pref = mp.sqrt(mp.factorial(l + m) * mp.factorial(l - m) * mp.factorial(l + n) * mp.factorial(l - n))
        tot = mp.mpf(0)
        for k in range(0, 2 * l + 1):
            a, cc, d = l + n - k, m - n + k, l - m - k
            if a < 0 or cc < 0 or d < 0:
                continue
            tot += (-1) ** (m - n + k) * c ** (2 * l + n - m - 2 * k) * s ** (m - n + 2 * k) / (
                mp.factorial(a) * mp.factorial(k) * mp.factorial(cc) * mp.factorial(d))
        return float(pref * tot)

    rng = np.random.default_rng(2)
    for _ in range(40):
        l = int(rng.integers(0, 31))
        m = int(rng.integers(-l, l + 1))
        n = int(rng.integers(-l, l + 1))
        b = float(rng.uniform(0.01, math.pi - 0.01))
        got = O.wigner_d(b, l + 1, m, n)[l]
        assert abs(got - wig(l, m, n, b)) < 5e-14, (l, m, n, b)


def test_wigner_orthogonality():
    for b, l in ((0.3, 10), (1.5707963, 77), (2.9, 200), (np.pi / 2, 2047), (0.9, 1500)):
        ms = np.arange(-l, l + 1)
        for k, kp in ((0, 0), (3, 3), (3, -2), (l, l - 1), (-l, -l), (1323, 1323), (1323, 1201)):
            if abs(k) > l or abs(kp) > l:
                continue
            col = O.wigner_d(b, l + 1, ms, k)[l]
            colp = O.wigner_d(b, l + 1, ms, kp)[l]
            assert abs(col @ colp - (1.0 if k == kp else 0.0)) < 1e-12


def test_delta_symmetries_and_fourier_expansion():
    L = 13
    ms = np.arange(-(L - 1), L)
    Dl = O.delta(L, ms[:, None], ms[None, :])          # [l][m'][m]
    for l in range(L):
        sl = slice(L - 1 - l, L + l)
        D = Dl[l][sl, sl]
        mm = np.arange(-l, l + 1)
        sgn_row = (-1.0) ** (l + mm)                  # Delta_{-m',m} = (-1)^(l+m) Delta_{m'm}
        assert np.abs(D[::-1, :] - D * sgn_row[None, :]).max() < 1e-14
        assert np.abs(D[:, ::-1] - D * sgn_row[:, None]).max() < 1e-14
        par = (-1.0) ** (mm[:, None] - mm[None, :])
        assert np.abs(D - D.T * par).max() < 1e-14
    # Eq. (25): d^l_mn(beta) = e^{-i(n-m)pi/2} sum_m' Delta_{m'm} Delta_{m'n} e^{-i m' beta}
    rng = np.random.default_rng(3)
    for b in rng.uniform(0, math.pi, 5):
        for l in range(L):
            sl = slice(L - 1 - l, L + l)
            D = Dl[l][sl, sl]
            mm = np.arange(-l, l + 1)
            for m in range(-l, l + 1):
                for n in range(-l, l + 1):
                    s = np.sum(D[:, m + l] * D[:, n + l] * np.exp(-1j * mm * b))
                    val = np.exp(-1j * (n - m) * math.pi / 2) * s
                    assert abs(val.imag) < 1e-13
                    assert abs(val.real - O.wigner_d(b, l + 1, m, n)[l]) < 1e-13


# --- whole transform ----------------------------------------------------------

def _single_mode_f(L, l0, m0, c):
    f = np.zeros(L * L, dtype=np.complex128)
    f[l0 * l0 + l0 + m0] += c
    if m0 != 0:
        f[l0 * l0 + l0 - m0] += (-1) ** m0 * np.conj(c)
    else:
        f[l0 * l0 + l0] = c.real
    return f


@pytest.mark.parametrize("N,lam,J0", [(3, 2.0, 0), (2, 2.0, 1), (1, 2.0, 2), (4, 1.5, 0)])
def test_single_mode_analysis_closed_form(N, lam, J0):
    L = 6
    psi, phi = O.kernels(L, N, lam, J0)
    alpha, beta, gamma = O.grids(L, N)
    ns = O.n_orders(N)
    for (l0, m0, c) in ((1, 1, 0.3 - 0.7j), (2, 1, 1.1 + 0.2j), (2, 2, -0.4 + 0.9j), (1, 0, 0.8 + 0j), (2, 0, -1.3 + 0j)):
        f = _single_mode_f(L, l0, m0, c)
        W, Wphi = O.analysis(f, L, N, lam, J0)
        for j in range(psi.shape[0]):
            for (g, b, a) in ((0, 1, 2), (N - 1, 7, 10), (N // 2, 11, 0)):
                ref = 0.0
                for k, n in enumerate(ns):
                    if abs(n) > l0:
                        continue
                    for mm, cc in ((m0, f[l0 * l0 + l0 + m0]), (-m0, f[l0 * l0 + l0 - m0])) if m0 else ((0, f[l0 * l0 + l0]),):
                        ref += cc * np.conj(psi[j, l0, k]) * np.conj(D_closed(l0, mm, n, alpha[a], beta[b], gamma[g]))
                assert abs(ref.imag) < 1e-14
                assert abs(W[j, g, b, a] - ref.real) < 1e-14
        # scaling coefficients: sum_m f_lm Phi_l D^l*_m0(phi, theta, 0)
        for (b, a) in ((0, 0), (5, 3)):
            ref = 0.0
            for mm in ((m0, -m0) if m0 else (0,)):
                ref += f[l0 * l0 + l0 + mm] * phi[l0] * np.conj(D_closed(l0, mm, 0, alpha[a], beta[b], 0.0))
            assert abs(Wphi[b, a] - ref.real) < 1e-14


@pytest.mark.parametrize("N", [1, 3, 4])
def test_single_mode_synthesis_closed_form(N):
    """W^j = D^{l0 *}_{m0 n0} on one scale -> f_{l0 m0} = Psi^j_{l0 n0} (Eqs. (32)-(33),
    orthogonality of D); W^Phi = e^{i m0 phi} d^{l0}_{m0 0}(theta) -> f_{l0 m0} = Phi_{l0} (Eq. (41))."""
    L, lam, J0 = 6, 2.0, 1
    psi, phi = O.kernels(L, N, lam, J0)
    alpha, beta, gamma = O.grids(L, N)
    ns = O.n_orders(N)
    J1 = psi.shape[0]
    A, B, G = np.meshgrid(alpha, beta, gamma, indexing="ij")      # [a][b][g]
    for (l0, m0, k0, j) in ((2, 1, 0, 0), (2, -2, N - 1, 1), (1, 0, N // 2, 1)):
        n0 = int(ns[k0])
        if abs(n0) > l0:
            continue
        W = np.zeros((J1, N, 2 * L, 2 * L - 1), dtype=np.complex128)
        vals = np.vectorize(lambda a, b, g: np.conj(D_closed(l0, m0, n0, a, b, g)))(A, B, G)
        W[j] = np.transpose(vals, (2, 1, 0))
        f = O.synthesis(W, np.zeros((2 * L, 2 * L - 1)), L, N, lam, J0)
        expect = np.zeros(L * L, dtype=np.complex128)
        expect[l0 * l0 + l0 + m0] = psi[j, l0, k0]
        assert np.abs(f - expect).max() < 1e-14
    for (l0, m0) in ((2, 1), (0, 0), (1, -1)):
        Wp = np.zeros((2 * L, 2 * L - 1), dtype=np.complex128)
        for b in range(2 * L):
            Wp[b] = np.exp(1j * m0 * alpha) * d_closed(l0, m0, 0, beta[b])
        f = O.synthesis(np.zeros((J1, N, 2 * L, 2 * L - 1)), Wp, L, N, lam, J0)
        expect = np.zeros(L * L, dtype=np.complex128)
        expect[l0 * l0 + l0 + m0] = phi[l0]
        assert np.abs(f - expect).max() < 1e-14


def test_realness_and_steerability():
    L, N, lam, J0 = 8, 3, 2.0, 0
    f = flm_gaussian(L, 7)
    W, Wphi, imag = O.analysis_rows(f, L, N, lam, J0, range(2 * L))
    assert imag < 1e-13
    # Eq. (10): W(gamma) = sum_g z(gamma - gamma_g) W(gamma_g) with z_n = 1/N,
    # z(x) = sum_n z_n e^{i n x}; W at gamma off the grid by the direct sum.
    psi, _ = O.kernels(L, N, lam, J0)
    alpha, beta, gamma = O.grids(L, N)
    ns = O.n_orders(N)
    F = O.flm_to_grid(f, L)
    ms = np.arange(-(L - 1), L)
    gam = 0.7318
    for (j, b, a) in ((0, 3, 4), (1, 10, 1)):
        D = O.wigner_d(beta[b], L, ms[:, None], ns[None, :])
        T = np.einsum("lm,lk,lmk->mk", F, np.conj(psi[j]), D)
        direct = np.sum(T * np.exp(1j * ms[:, None] * alpha[a]) * np.exp(1j * ns[None, :] * gam)).real
        z = lambda x: np.sum(np.exp(1j * ns * x)).real / N
        steered = sum(z(gam - gamma[g]) * W[j, g, b, a] for g in range(N))
        assert abs(direct - steered) < 1e-13
        # the oracle's steer() is the same interpolation
        assert abs(O.steer(W, N, [gam])[j, 0, b, a] - direct) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_steer_reproduces_samples(N):
    """z(gamma_g' - gamma_g) = delta_gg' (Dirichlet kernel of the odd-spaced
    orders at multiples of pi/N), so steering to the sample angles returns W."""
    rng = np.random.default_rng(N)
    W = rng.standard_normal((2, N, 6, 5))
    gamma_g = np.pi * np.arange(N) / N
    assert np.abs(O.steer(W, N, gamma_g) - W).max() < 1e-13
    # period: gamma and gamma + 2 pi give the same coefficients
    g = rng.uniform(0, np.pi, 3)
    assert np.abs(O.steer(W, N, g) - O.steer(W, N, g + 2 * np.pi)).max() < 1e-12


@pytest.mark.parametrize("L,N,lam,J0,kind", [(8, 3, 2.0, 0, "unit"), (16, 5, 2.0, 0, "cl"),
                                              (16, 2, 2.0, 1, "uniform"), (12, 1, 3.0, 0, "unit"),
                                              (16, 4, 2.5, 1, "unit"), (32, 3, 2.0, 0, "unit"),
                                              (10, 8, 2.0, 0, "unit")])
def test_round_trip_exact(L, N, lam, J0, kind):
    f = flm_uniform(L, 11) if kind == "uniform" else flm_gaussian(L, 3, kind)
    W, Wphi = O.analysis(f, L, N, lam, J0)
    fr = O.synthesis(W, Wphi, L, N, lam, J0)
    # Sec. 3.4 metric: eps = max |f_rec - f_orig|
    assert np.abs(fr - f).max() < 1e-12


@pytest.mark.parametrize("L,N,lam,J0", [(8, 3, 2.0, 1), (12, 1, 2.0, 2), (12, 4, 3.0, 1), (10, 2, 2.0, 0)])
def test_synthesis_modes_round_trip_exact(L, N, lam, J0):
    """synthesis_modes (the per-(l, m) form of Eqs. (32)-(33), (41)) must
    return every f_lm exactly, negative m included, from the analysis of a
    real signal, with J0 > 0 so that the scaling term of Eq. (41) carries
    signal (Sec. 3.4 exactness, eps to 1e-12)."""
    f = flm_gaussian(L, 5)
    W, Wphi = O.analysis(f, L, N, lam, J0)
    if J0 > 0:
        assert np.abs(Wphi).max() > 1e-3          # the Phi term is live
    lm = [(l, m) for l in range(L) for m in range(-l, l + 1)]
    got = O.synthesis_modes(W, Wphi, L, N, lam, J0, lm)
    err = max(abs(got[(l, m)] - f[l * l + l + m]) for (l, m) in lm)
    assert err < 1e-12, err


@pytest.mark.parametrize("L,N,lam,J0", [(8, 3, 2.0, 1), (9, 2, 2.0, 1)])
def test_synthesis_modes_equals_synthesis_on_arbitrary_arrays(L, N, lam, J0):
    """On arrays that are not the analysis of any signal (so nothing cancels),
    synthesis_modes must equal the full synthesis at every (l, m)."""
    rng = np.random.default_rng(7)
    J1 = O.n_scales(L, lam, J0) + 1
    W = rng.standard_normal((J1, N, 2 * L, 2 * L - 1))
    Wphi = rng.standard_normal((2 * L, 2 * L - 1))
    full = O.synthesis(W, Wphi, L, N, lam, J0)
    lm = [(l, m) for l in range(L) for m in range(-l, l + 1)]
    got = O.synthesis_modes(W, Wphi, L, N, lam, J0, lm)
    scale = np.abs(full).max()
    err = max(abs(got[(l, m)] - full[l * l + l + m]) for (l, m) in lm)
    assert err < 1e-12 * max(1.0, scale), err


def test_fourier_cube_reproduces_analysis():
    """Eq. (26): W = sum_{m m' n} U_{m m' n} e^{i(m alpha + m' beta + n gamma)}."""
    L, N, lam, J0 = 8, 3, 2.0, 0
    f = flm_gaussian(L, 9)
    W, _ = O.analysis(f, L, N, lam, J0)
    alpha, beta, gamma = O.grids(L, N)
    ns = O.n_orders(N)
    ms = np.arange(-(L - 1), L)
    for j in (0, 2):
        U = O.fourier_cube(f, L, N, lam, J0, j)          # [m][m'][k]
        for (g, b, a) in ((0, 0, 0), (2, 9, 13), (1, 15, 6)):
            val = np.einsum("mpk,m,p,k->", U, np.exp(1j * ms * alpha[a]), np.exp(1j * ms * beta[b]),
                            np.exp(1j * ns * gamma[g]))
            assert abs(val - W[j, g, b, a]) < 1e-13


# ---- spherical harmonic transforms on the DH grid ----

def _ylm_textbook(l, m, theta, phi):
    """Textbook spherical harmonics (Condon-Shortley phase), l <= 2, m >= 0."""
    c, s = np.cos(theta), np.sin(theta)
    table = {
        (0, 0): 0.5 * np.sqrt(1 / np.pi) + 0 * theta,
        (1, 0): np.sqrt(3 / (4 * np.pi)) * c,
        (1, 1): -np.sqrt(3 / (8 * np.pi)) * s,
        (2, 0): np.sqrt(5 / (16 * np.pi)) * (3 * c * c - 1),
        (2, 1): -np.sqrt(15 / (8 * np.pi)) * s * c,
        (2, 2): np.sqrt(15 / (32 * np.pi)) * s * s,
    }
    return table[(l, m)][:, None] * np.exp(1j * m * phi)[None, :]


@pytest.mark.parametrize("l,m", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)])
def test_sht_textbook_harmonics(l, m):
    L = 5
    phi, theta, _ = O.grids(L, 1)
    Y = _ylm_textbook(l, m, theta, phi)
    flm = np.zeros(L * L, dtype=np.complex128)
    flm[l * l + l + m] = 1.0
    assert np.abs(O.sht_inverse(flm, L) - Y).max() < 1e-14
    back = O.sht_forward(Y, L)
    assert np.abs(back - flm).max() < 1e-14


@pytest.mark.parametrize("L", [4, 9, 16])
def test_sht_round_trip_exact(L):
    f = flm_gaussian(L, 13)
    pix = O.sht_inverse(f, L)
    assert np.abs(pix.imag).max() < 1e-13          # real signal -> real samples
    assert np.abs(O.sht_forward(pix.real, L) - f).max() < 1e-13


# ---- multi-resolution sampling ----

@pytest.mark.parametrize("L,N,lam,J0", [(16, 3, 2.0, 0), (24, 2, 2.0, 1), (20, 1, 3.0, 0), (12, 4, 2.0, 0)])
def test_multires_round_trip_exact(L, N, lam, J0):
    f = flm_gaussian(L, 31, "unit")
    Ws, Wphi = O.analysis_multires(f, L, N, lam, J0)
    Ls, Lp = O.band_limits(L, N, lam, J0)
    assert all(W.shape == (N, 2 * Lj, 2 * Lj - 1) for W, Lj in zip(Ws, Ls)) and Wphi.shape == (2 * Lp, 2 * Lp - 1)
    assert np.abs(O.synthesis_multires(Ws, Wphi, L, N, lam, J0) - f).max() < 1e-12


def test_multires_matches_full_resolution_on_shared_samples():
    """alpha = 0 is on every grid; beta_b of band-limit L_j equals beta_{3b+1} of
    band-limit 3 L_j, so a scale with L = 3 L_j shares those samples."""
    L, N, lam, J0 = 24, 3, 2.0, 0
    f = flm_gaussian(L, 41, "cl")
    Ws, Wphi = O.analysis_multires(f, L, N, lam, J0)
    W, Wp = O.analysis(f, L, N, lam, J0)
    Ls, Lp = O.band_limits(L, N, lam, J0)
    checked = 0
    for j, Lj in enumerate(Ls):
        if 3 * Lj == L:
            b = np.arange(2 * Lj)
            assert np.abs(Ws[j][:, b, 0] - W[j][:, 3 * b + 1, 0]).max() < 1e-13
            checked += 1
        if Lj == L:
            assert np.abs(Ws[j] - W[j]).max() < 1e-13
            checked += 1
    assert checked >= 2


# ---- sampling with L beta samples (the grid named in Sec. 4 as the DH replacement) ----

def test_mw_betas_values():
    b = O.mw_betas(5)
    assert b.shape == (5,)
    assert np.allclose(b, np.pi * np.array([1, 3, 5, 7, 9]) / 9)
    assert abs(b[-1] - np.pi) < 1e-15          # the last sample is the pole beta = pi


@pytest.mark.parametrize("N", [1, 3, 4])
def test_mw_single_mode_analysis_closed_form(N):
    """Eq. (20) at the MW beta samples against closed-form D (l <= 2)."""
    L, lam, J0 = 6, 2.0, 1
    psi, phi = O.kernels(L, N, lam, J0)
    alpha, _, gamma = O.grids(L, N)
    beta = O.mw_betas(L)
    ns = O.n_orders(N)
    for (l0, m0, c) in ((1, 1, 0.3 - 0.7j), (2, 2, -0.4 + 0.9j), (2, 0, -1.3 + 0j)):
        f = _single_mode_f(L, l0, m0, c)
        W, Wphi = O.analysis_mw(f, L, N, lam, J0)
        assert W.shape == (psi.shape[0], N, L, 2 * L - 1) and Wphi.shape == (L, 2 * L - 1)
        for j in range(psi.shape[0]):
            for (g, b, a) in ((0, 0, 2), (N - 1, L - 1, 10), (N // 2, 3, 0)):
                ref = 0.0
                for k, n in enumerate(ns):
                    if abs(n) > l0:
                        continue
                    for mm, cc in ((m0, f[l0 * l0 + l0 + m0]), (-m0, f[l0 * l0 + l0 - m0])) if m0 else ((0, f[l0 * l0 + l0]),):
                        ref += cc * np.conj(psi[j, l0, k]) * np.conj(D_closed(l0, mm, n, alpha[a], beta[b], gamma[g]))
                assert abs(W[j, g, b, a] - ref.real) < 1e-14
        for (b, a) in ((0, 0), (L - 1, 3)):
            ref = 0.0
            for mm in ((m0, -m0) if m0 else (0,)):
                ref += f[l0 * l0 + l0 + mm] * phi[l0] * np.conj(D_closed(l0, mm, 0, alpha[a], beta[b], 0.0))
            assert abs(Wphi[b, a] - ref.real) < 1e-14


@pytest.mark.parametrize("L,N,lam,J0", [(8, 3, 2.0, 0), (9, 2, 2.0, 1), (12, 4, 3.0, 0), (7, 1, 2.0, 1)])
def test_mw_resampling_and_round_trip_exact(L, N, lam, J0):
    """The L-sample coefficients hold the same band-limited functions: resampled
    to the DH grid they equal the DH analysis, and the synthesis from them is
    exact (Sec. 3.4 metric)."""
    f = flm_gaussian(L, 13, "unit")
    kern = O.kernels(L, N, lam, J0)
    Wm, Wpm = O.analysis_mw(f, L, N, lam, J0, kern)
    Wd, Wpd = O.analysis(f, L, N, lam, J0, kern)
    Wr, Wpr = O.resample_mw_to_dh(Wm, Wpm, L, N)
    assert np.abs(Wr - Wd).max() < 1e-13 * np.abs(Wd).max()
    assert np.abs(Wpr - Wpd).max() < 1e-13 * max(1.0, np.abs(Wpd).max())
    fr = O.synthesis_mw(Wm, Wpm, L, N, lam, J0, kern)
    assert np.abs(fr - f).max() < 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("m,vanishes", [(1, True), (3, True), (2, False)])
def test_mw_pole_only_component(m, vanishes):
    """The pole sample beta = pi is its own reflection on the beta torus.
    Take coefficients nonzero only there, and constant in gamma, so that for
    the wavelets only the order n = 0 of S_N (N = 3) survives the gamma sum.
    In a Fourier component with sigma = (-1)^{m-n} = -1 (odd m) they
    describe no band-limited function, because such a component vanishes at
    the pole.  Their synthesis (the projection onto band-limited signals)
    is then exactly zero.  With sigma = +1 (even m) it is not."""
    L, N, lam, J0 = 6, 3, 2.0, 1
    kern = O.kernels(L, N, lam, J0)
    alpha, _, _ = O.grids(L, N)
    nj = kern[0].shape[0]
    W = np.zeros((nj, N, L, 2 * L - 1))
    W[:, :, L - 1, :] = np.cos(m * alpha)[None, None, :]
    Wphi = np.zeros((L, 2 * L - 1))
    Wphi[L - 1, :] = np.cos(m * alpha)
    f = O.synthesis_mw(W, Wphi, L, N, lam, J0, kern)
    if vanishes:
        assert np.abs(f).max() < 1e-13
    else:
        assert np.abs(f).max() > 1e-3


def test_parity_table_names_every_public_function():
    """Every public oracle function states how it is pinned."""
    import oracle.s2dw_oracle as OS
    missing = [n for n in OS.__all__ if n != "PARITY" and n not in OS.PARITY]
    assert not missing, missing
