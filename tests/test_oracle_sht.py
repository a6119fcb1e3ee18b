"""Pins of the oracle's grid, Legendre functions and transforms (CPU only).

Each check compares the oracle with something other than itself: numpy's
Gauss-Legendre routine, exact monomial integrals, textbook closed forms of
low-order Y_lm, scipy's spherical harmonics, an explicit-polynomial
evaluation of P_lm in 1600-digit arithmetic, and the addition theorem.
"""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy.special import sph_harm_y

import simgen
from oracle import sht


@pytest.mark.parametrize("n", [1, 2, 3, 8, 33, 64, 501])
def test_gl_nodes_match_numpy(n):
    mu, w = sht.gl_nodes(n)
    x, wx = np.polynomial.legendre.leggauss(n)
    assert np.all(np.diff(mu) < 0)                       # north first
    np.testing.assert_allclose(mu, x[::-1], atol=2e-15)
    # numpy's weights lose ~1e-9 relative near the poles at n ~ 500 (see the
    # high-precision check below); agreement to 2e-9 is what it offers there.
    np.testing.assert_allclose(w, wx[::-1], rtol=2e-9, atol=1e-15)
    assert abs(w.sum() - 2.0) < 1e-13
    np.testing.assert_array_equal(mu, -mu[::-1])         # exact mirror symmetry


def test_gl_pole_weight_high_precision():
    n = 501
    mu, w = sht.gl_nodes(n)
    with mp.workdps(40):
        def p_and_dp(t):
            p0, p1 = mp.mpf(1), t
            for k in range(2, n + 1):
                p0, p1 = p1, ((2 * k - 1) * t * p1 - (k - 1) * p0) / k
            return p1, n * (t * p1 - p0) / (t * t - 1)
        for j in (0, 3, 250):
            t = mp.mpf(mu[j])
            for _ in range(6):
                p, dp = p_and_dp(t)
                t = t - p / dp
            p, dp = p_and_dp(t)
            assert abs(float(t) - mu[j]) < 1e-15
            assert abs(float(2 / ((1 - t * t) * dp * dp)) / w[j] - 1) < 1e-11


@pytest.mark.parametrize("n", [5, 17, 40])
def test_gl_integrates_monomials_exactly(n):
    mu, w = sht.gl_nodes(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * mu ** k) - exact) < 1e-13


def test_lambda_low_order_closed_forms():
    th = np.linspace(0.05, 3.1, 23)
    mu, s = np.cos(th), np.sin(th)
    tab = sht.legendre_table(2, mu)
    idx = lambda l, m: simgen.alm_index(l, m, 2)
    pi = math.pi
    np.testing.assert_allclose(tab[idx(0, 0)], 1 / math.sqrt(4 * pi), rtol=1e-13)
    np.testing.assert_allclose(tab[idx(1, 0)], math.sqrt(3 / (4 * pi)) * mu, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(tab[idx(1, 1)], -math.sqrt(3 / (8 * pi)) * s, rtol=1e-13)
    np.testing.assert_allclose(tab[idx(2, 0)], math.sqrt(5 / (4 * pi)) * (3 * mu * mu - 1) / 2,
                               rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(tab[idx(2, 1)], -math.sqrt(15 / (8 * pi)) * s * mu, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(tab[idx(2, 2)], 0.25 * math.sqrt(15 / (2 * pi)) * s * s, rtol=1e-13)


def test_lambda_matches_scipy():
    L = 40
    th = np.linspace(0.01, 3.13, 37)
    tab = sht.legendre_table(L, np.cos(th))
    lidx, midx = simgen.lm_arrays(L)
    ref = sph_harm_y(lidx[:, None], midx[:, None], th[None, :], 0.0).real
    np.testing.assert_allclose(tab, ref, atol=2e-13)


def _lambda_explicit(l, m, x, dps=1600):
    """sqrt((2l+1)/4pi (l-m)!/(l+m)!) (-1)^m (1-x^2)^{m/2} d^m/dx^m P_l(x), with P_l from
    its explicit power series, in high-precision arithmetic."""
    with mp.workdps(dps):
        x = mp.mpf(x)
        acc = mp.mpf(0)
        for k in range((l - m) // 2 + 1):
            n = l - 2 * k
            c = math.comb(l, k) * math.comb(2 * l - 2 * k, l) * (math.factorial(n) // math.factorial(n - m))
            acc += (-1) ** k * c * x ** (n - m)
        p = (-1) ** m * (1 - x * x) ** (mp.mpf(m) / 2) * acc / mp.mpf(2) ** l
        return float(mp.sqrt(mp.mpf(2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m)) * p)


@pytest.mark.parametrize("m,sin_theta", [(1400, 0.55), (1500, 0.70), (1700, 0.84), (1900, 0.93), (300, 0.2)])
def test_lambda_high_order_near_underflow(m, sin_theta):
    """lambda_mm underflows FP64 for the first cases (0.55^1400 ~ 1e-364): the rescaled
    recurrence must still give lambda_{2000,m} to full precision."""
    L = 2000
    x = math.sqrt(1 - sin_theta ** 2)
    tab = sht.legendre_table(L, np.array([x]))
    for l in (m, m + 1, (m + L) // 2, L):
        got = tab[simgen.alm_index(l, m, L)][0]
        ref = _lambda_explicit(l, m, x)
        assert got == pytest.approx(ref, rel=1e-10, abs=1e-300), (l, m)


def test_addition_theorem_l2000():
    L = 2000
    mu, _ = sht.gl_nodes(L + 1)
    rings = np.array([0, 1, 7, 250, 600, 1000])           # pole-most ring to the equator
    tab = sht.legendre_table(L, mu[rings])
    acc = np.zeros((L + 1, rings.size))
    for m in range(L + 1):
        s = simgen.alm_index(m, m, L)
        acc[m:] += (1.0 if m == 0 else 2.0) * tab[s: s + L - m + 1] ** 2
    l = np.arange(L + 1)
    np.testing.assert_allclose(acc, np.broadcast_to(((2 * l + 1) / (4 * math.pi))[:, None], acc.shape), rtol=1e-10)


def test_synthesis_matches_scipy_ylm():
    L, nphi = 12, 32
    mu, _ = sht.gl_nodes(L + 1)
    a = simgen.white_alm(L, 1, seed=5)[0]
    filt = np.ones((1, L + 1))
    maps = sht.synthesize(a, L, filt, mu, nphi)[0]
    th, ph = np.meshgrid(np.arccos(mu), sht.phi_grid(nphi), indexing="ij")
    ref = np.zeros_like(maps)
    for i, (l, m) in enumerate(zip(*simgen.lm_arrays(L))):
        y = sph_harm_y(l, m, th, ph)
        ref += (1 if m == 0 else 2) * (y * a[i]).real     # the -m partner doubles m > 0
    np.testing.assert_allclose(maps, ref, atol=1e-12)


def test_filtered_synthesis_is_linear_in_basis():
    L, nphi = 10, 32
    mu, _ = sht.gl_nodes(L + 1)
    a = simgen.white_alm(L, 1, seed=6)[0]
    basis = simgen.shifted_legendre_basis(L, 3)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(basis, cl)
    maps = sht.synthesize(a, L, filt, mu, nphi)
    for p in range(3):
        single = sht.synthesize(a * 1.0, L, filt[p:p + 1], mu, nphi)[0]
        np.testing.assert_allclose(maps[p], single, atol=1e-12)
    assert np.all(filt[:, :2] == 0.0)                      # C_0 = C_1 = 0 filtered out


@pytest.mark.parametrize("L,nrings,nphi", [(20, 21, 64), (16, 25, 64), (7, 8, 16)])
def test_analysis_inverts_synthesis(L, nrings, nphi):
    mu, w = sht.gl_nodes(nrings)
    a = simgen.white_alm(L, 1, seed=7)[0]
    maps = sht.synthesize(a, L, np.ones((1, L + 1)), mu, nphi)[0]
    np.testing.assert_allclose(sht.analyze(maps, L, mu, w, nphi), a, atol=1e-12)


def test_batched_transforms_equal_the_per_map_transforms():
    """synthesize_many / analyze_many (the lambda table of a ring block formed once for
    several maps, used by the full-size fixture script) give the per-map results exactly."""
    L, P, R, nphi = 24, 3, 27, 64
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    a = simgen.gaussian_alm(cl, 3, seed=51)
    mu, w = sht.gl_nodes(R)
    many = sht.synthesize_many(a, L, filt, mu, nphi)
    for i in range(3):
        assert np.array_equal(many[i], sht.synthesize(a[i], L, filt, mu, nphi))
    x = simgen.noise_maps(R, nphi, 3, seed=52, sigma0_sq=0.1).astype(np.float64)
    am = sht.analyze_many(x, L, mu, w, nphi)
    for i in range(3):
        ref = sht.analyze(x[i], L, mu, w, nphi)
        assert np.max(np.abs(am[i] - ref)) <= 1e-13 * np.max(np.abs(ref))
