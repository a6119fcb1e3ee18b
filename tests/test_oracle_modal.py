"""Pins of the oracle's modal coefficients, linear term, covariance and solve (CPU only).

Every check compares the oracle with an independent fact: sympy's 3j and Gaunt
values, the harmonic-space Gaunt sum of Eq. bbispect evaluated by brute force,
closed forms of the covariance and of the local-shape mean, Wick identities of
the linear term, finite differences, and exact linear-algebra identities of
Sec. III.B.  The last block plants mistakes in copies of oracle functions and
checks that the pins catch them.
"""
import math

import numpy as np
import pytest

import simgen
from oracle import modal, sht, wigner


def _grid(nrings, nphi, mask=None):
    mu, w = sht.gl_nodes(nrings)
    return mu, w, modal.pixel_weights(w, nphi, mask)


def _exact_cubic_rings(L):
    return (3 * L + 2) // 2 + 1


# ---------------------------------------------------------------- Gaunt / 3j

def test_wigner3j_and_gaunt_match_sympy():
    wig = pytest.importorskip("sympy.physics.wigner")
    g = np.random.default_rng(1)
    for _ in range(60):
        l1, l2 = g.integers(0, 7, size=2)
        l3 = g.integers(abs(l1 - l2), l1 + l2 + 1)
        m1 = g.integers(-l1, l1 + 1)
        m2 = g.integers(-l2, l2 + 1)
        m3 = -m1 - m2
        if abs(m3) > l3:
            continue
        ref = float(wig.wigner_3j(int(l1), int(l2), int(l3), int(m1), int(m2), int(m3)))
        assert wigner.wigner3j(l1, l2, l3, m1, m2, m3) == pytest.approx(ref, abs=1e-14)
        refg = float(wig.gaunt(int(l1), int(l2), int(l3), int(m1), int(m2), int(m3)))
        assert wigner.gaunt(l1, l2, l3, m1, m2, m3) == pytest.approx(refg, abs=1e-14)


@pytest.mark.parametrize("L,P", [(5, 3), (7, 2)])
def test_grid_cubic_equals_gaunt_sum_on_exact_cubic_grid(L, P):
    """Eq. bbispect with R_n = q_p q_r q_s, v_l = 1: the Gaunt sum equals the sphere
    integral of M_p M_r M_s; on a grid exact for degree 3L the quadrature is exact."""
    nrings, nphi = _exact_cubic_rings(L), 32
    mu, w, W = _grid(nrings, nphi)
    cl = simgen.cl_model(L)
    cl[:2] = [0.7, 0.4]                                   # keep l = 0, 1 in play
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    a = simgen.gaussian_alm(cl, 1, seed=11)[0]
    maps = sht.synthesize(a, L, filt, mu, nphi)
    got = modal.cubic_beta(maps, W)
    ref = wigner.gaunt_beta(a, L, filt)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_config_grid_aliases_the_cubic_term():
    """With R = L + 1 rings the grid sum is not the Gaunt sum (degree 3L > 2L + 1): the
    definition of beta adopted here is the grid quadrature, shared by oracle and GPU."""
    L, P, nphi = 6, 2, 32
    mu, w, W = _grid(L + 1, nphi)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    a = simgen.gaussian_alm(cl, 1, seed=12)[0]
    got = modal.cubic_beta(sht.synthesize(a, L, filt, mu, nphi), W)
    ref = wigner.gaunt_beta(a, L, filt)
    assert np.max(np.abs(got - ref)) > 1e-6 * np.max(np.abs(ref))


# ---------------------------------------------------------------- closed forms

def _alpha_bruteforce(filt, cl):
    """Eq. abispect with v = 1, R_n = q q q / sqrt(CCC) folded into filt:
    sum_{l_i} h^2 b f_p f_r f_s, h^2 = (2l1+1)(2l2+1)(2l3+1)/(4pi) (l1 l2 l3; 0 0 0)^2."""
    P, L1 = filt.shape
    out = np.zeros(modal.n_modes(P))
    modes = modal.mode_list(P)
    for l1 in range(L1):
        for l2 in range(L1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, L1 - 1) + 1):
                if (l1 + l2 + l3) % 2:
                    continue
                h2 = (2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4 * math.pi) \
                    * wigner.wigner3j(l1, l2, l3, 0, 0, 0) ** 2
                b = 2.0 * (cl[l1] * cl[l2] + cl[l2] * cl[l3] + cl[l3] * cl[l1])
                for n, (p, r, s) in enumerate(modes):
                    out[n] += h2 * b * filt[p, l1] * filt[r, l2] * filt[s, l3]
    return out


def test_alpha_local_matches_harmonic_bruteforce():
    L, P = 9, 3
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    np.testing.assert_allclose(modal.alpha_local(filt, cl), _alpha_bruteforce(filt, cl), rtol=1e-11)


def _gaussian_betas(L, P, nrings, nphi, N, seed, mask=None, pairmean=None, stream=simgen.STREAM_COV):
    mu, w, W = _grid(nrings, nphi, mask)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    alms = simgen.gaussian_alm(cl, N, seed=seed, stream=stream)
    out = []
    for a in alms:
        maps = sht.synthesize(a, L, filt, mu, nphi)
        out.append((modal.cubic_beta(maps, W), None if pairmean is None else modal.cubic_beta(maps, W, pairmean)))
    return filt, cl, out


def test_zeta_matches_closed_form_covariance():
    """zeta = <beta beta^T>/6 (Eq. linearterm) against the six-pairing closed form."""
    L, P, N = 6, 2, 3000
    filt, cl, res = _gaussian_betas(L, P, _exact_cubic_rings(L), 32, N, seed=21)
    betas = np.array([b for b, _ in res])
    zeta = modal.covariance_zeta(betas)
    ref = modal.zeta_closed_form(filt, cl)
    cov = 6.0 * ref
    se = np.sqrt((np.outer(np.diag(cov), np.diag(cov)) + cov * cov) / N) / 6.0
    assert np.all(np.abs(zeta - ref) < 5.0 * se)
    assert np.all(np.abs(betas.mean(axis=0)) < 5.0 * np.sqrt(np.diag(cov) / N))   # zero mean


def _pairmean_isotropic(filt, cl, nrings, nphi):
    """Ensemble <M_p M_r>_x = sum_l (2l+1)/(4pi) f_p f_r C_l (addition theorem), every pixel."""
    l = np.arange(cl.size)
    vals = [np.sum((2 * l + 1) / (4 * math.pi) * filt[p] * filt[r] * cl) for (p, r) in modal.pair_list(filt.shape[0])]
    return np.array(vals)[:, None, None] * np.ones((1, nrings, nphi))


def test_linear_term_removes_correlation_with_linear_statistics():
    """With the ensemble <M M>, beta - lin is uncorrelated with every linear functional of
    the map (Wick); lin itself is one, so cov(beta - lin, lin) = 0 while cov(beta, lin) > 0.
    A masked sky makes lin non-zero."""
    L, P, nrings, nphi, N = 8, 2, 9, 32, 2500
    mask = simgen.band_mask(nrings, 20.0)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    pm = _pairmean_isotropic(filt, cl, nrings, nphi)
    _, _, res = _gaussian_betas(L, P, nrings, nphi, N, seed=31, mask=mask, pairmean=pm)
    b0 = np.array([b for b, _ in res])
    bl = np.array([b for _, b in res])
    lin = b0 - bl
    for n in range(b0.shape[1]):
        c_corr = np.corrcoef(bl[:, n], lin[:, n])[0, 1]
        c_raw = np.corrcoef(b0[:, n], lin[:, n])[0, 1]
        assert abs(c_corr) < 5.0 / math.sqrt(N), (n, c_corr)
        assert c_raw > 10.0 / math.sqrt(N), (n, c_raw)
    assert np.all(bl.var(axis=0) < b0.var(axis=0))       # the cross terms of Eq. crossterms


def test_local_shape_mean_matches_alpha():
    """T = G + f (G^2 - <G^2>) has E[beta] = f alpha + O(f^3), alpha from Eq. abispect.
    The antithetic difference (beta(f) - beta(-f)) / 2f cancels the Gaussian part exactly
    and leaves alpha + O(f^2)."""
    L, P, N, f = 8, 2, 300, 0.1
    nr, nphi = _exact_cubic_rings(L), 32
    mu, w, W = _grid(nr, nphi)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    raw = np.ones((1, L + 1))
    g2 = np.sum((2 * np.arange(L + 1) + 1) / (4 * math.pi) * cl)
    diffs = []
    for a in simgen.gaussian_alm(cl, N, seed=41, stream=simgen.STREAM_NG):
        G = sht.synthesize(a, L, raw, mu, nphi)[0]
        b = []
        for ff in (f, -f):
            aT = sht.analyze(G + ff * (G * G - g2), L, mu, w, nphi)
            b.append(modal.cubic_beta(sht.synthesize(aT, L, filt, mu, nphi), W))
        diffs.append((b[0] - b[1]) / (2 * f))
    diffs = np.array(diffs)
    alpha = modal.alpha_local(filt, cl)
    se = diffs.std(axis=0, ddof=1) / math.sqrt(N)
    assert np.all(np.abs(diffs.mean(axis=0) - alpha) < 5.0 * se + 0.02 * np.abs(alpha))
    assert np.all(np.abs(alpha) > 5.0 * se)               # the test has power


# ---------------------------------------------------------------- solve

def _spd(n, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def test_solve_matches_direct_formula_and_is_mode_invariant():
    n, B = 10, 4
    g = np.random.default_rng(3)
    zeta, alpha, betas = _spd(n, 4), g.standard_normal(n), g.standard_normal((B, n))
    fnl, sigma = modal.solve_fnl(zeta, alpha, betas)
    zi_a = np.linalg.solve(zeta, alpha)
    np.testing.assert_allclose(fnl, betas @ zi_a / (alpha @ zi_a), rtol=1e-12)
    assert sigma == pytest.approx(math.sqrt(6.0 / (alpha @ zi_a)), rel=1e-12)
    T = simgen.random_modes_matrix(n, seed=5)
    fnl2, sigma2 = modal.solve_fnl(T @ zeta @ T.T, T @ alpha, betas @ T.T)
    np.testing.assert_allclose(fnl2, fnl, rtol=1e-10)
    assert sigma2 == pytest.approx(sigma, rel=1e-10)


def test_bivector_identities():
    g = np.random.default_rng(8)
    bt, alpha = g.standard_normal(7), g.standard_normal(7)
    zeta = np.eye(7) + np.outer(bt, bt)
    np.testing.assert_allclose(modal.bivector_inverse(bt) @ zeta, np.eye(7), atol=1e-13)
    np.testing.assert_allclose(modal.bivector_cholesky(bt), np.linalg.cholesky(zeta), atol=1e-13)
    assert modal.bivector_variance(alpha, bt) == pytest.approx(1.0 / (alpha @ np.linalg.solve(zeta, alpha)), rel=1e-12)


# ---------------------------------------------------------------- adjoint

def test_adjoint_matches_central_differences():
    L, P, nrings, nphi = 5, 2, 6, 16
    mu, w = sht.gl_nodes(nrings)
    mask = simgen.band_mask(nrings, 20.0)
    W = modal.pixel_weights(w, nphi, mask)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    a = simgen.gaussian_alm(cl, 1, seed=51)[0]
    rng = np.random.default_rng(9)
    pm = np.abs(rng.standard_normal((modal.pair_list(P).__len__(), nrings, nphi)))
    g = rng.standard_normal(modal.n_modes(P))
    grad = modal.adjoint_grad(a, g, L, filt, mu, w, nphi, mask, pm)

    def loss(x):
        return float(g @ modal.cubic_beta(sht.synthesize(x, L, filt, mu, nphi), W, pm))

    lidx, midx = simgen.lm_arrays(L)
    for i in range(a.size):
        if cl[lidx[i]] == 0:
            continue
        h = 1e-3 * math.sqrt(cl[lidx[i]])
        d = np.zeros_like(a)
        d[i] = h
        dre = (loss(a + d) - loss(a - d)) / (2 * h)
        assert grad[i].real == pytest.approx(dre, rel=1e-6, abs=1e-9 * np.abs(grad).max())
        if midx[i] > 0:
            dim = (loss(a + 1j * d) - loss(a - 1j * d)) / (2 * h)
            assert grad[i].imag == pytest.approx(dim, rel=1e-6, abs=1e-9 * np.abs(grad).max())
        else:
            assert grad[i].imag == pytest.approx(0.0, abs=1e-12 * np.abs(grad).max())


# ---------------------------------------------------------------- planted mistakes
# Each case copies a piece of the oracle, plants one plausible mistake, and checks that
# the corresponding pin above would fail.  This is how the pins are known to bite.

def _antithetic_setup(P=3, L=8, nrings=9, nphi=32, nsim=6):
    mask = simgen.band_mask(nrings, 30.0)
    mu, w, W = _grid(nrings, nphi, mask)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    M = sht.synthesize(simgen.gaussian_alm(cl, 1, seed=81)[0], L, filt, mu, nphi)
    sims = [sht.synthesize(a, L, filt, mu, nphi)
            for a in simgen.gaussian_alm(cl, nsim, seed=82, stream=simgen.STREAM_LINEAR)]
    return M, sims, W, P


def _shift_average(M, sims, W):
    """(1/2N) sum_i [beta(M + M'_i) + beta(M - M'_i)] with the plain cubic (no linear term)."""
    return np.mean([0.5 * (modal.cubic_beta(M + s, W) + modal.cubic_beta(M - s, W)) for s in sims], axis=0)


def test_linear_term_is_the_antithetic_shift_average():
    """Expanding the cubic, the terms odd in M'_i cancel between +M'_i and -M'_i, so the
    shift average equals beta(M) + sum_x W (<pr> M_s + <ps> M_r + <rs> M_p) with <.> the
    sims' own pair mean: the linear term of Eq. bispectrumest, exactly."""
    M, sims, W, P = _antithetic_setup()
    pm = modal.pair_means(sims)
    b0 = modal.cubic_beta(M, W)
    bl = modal.cubic_beta(M, W, pm)
    np.testing.assert_allclose(2.0 * b0 - bl, _shift_average(M, sims, W), rtol=1e-11,
                               atol=1e-12 * np.abs(b0).max())


def test_planted_linear_term_mistakes_are_caught():
    M, sims, W, P = _antithetic_setup()
    pm = modal.pair_means(sims)
    pidx = {pr: i for i, pr in enumerate(modal.pair_list(P))}
    ref = _shift_average(M, sims, W) - modal.cubic_beta(M, W)     # = lin(M)
    Mf, pmf = M.reshape(P, -1), pm.reshape(pm.shape[0], -1)
    for kind in ("dropped", "wrong_index", "no_pair_symmetry"):
        out = []
        for (p, r, s) in modal.mode_list(P):
            t = [pmf[pidx[(p, r)]] * Mf[s], pmf[pidx[(p, s)]] * Mf[r], pmf[pidx[(r, s)]] * Mf[p]]
            if kind == "dropped":
                t = t[:1]
            elif kind == "wrong_index":
                t[1] = pmf[pidx[(p, s)]] * Mf[s]
            else:
                t = [3.0 * t[0]]
            out.append(np.sum(W.ravel() * sum(t)))
        assert np.max(np.abs(np.array(out) - ref)) > 1e-3 * np.max(np.abs(ref)), kind


def test_planted_synthesis_mistakes_are_caught():
    from scipy.special import sph_harm_y
    L, nphi = 6, 16
    mu, _ = sht.gl_nodes(L + 1)
    a = simgen.white_alm(L, 1, seed=71)[0]
    th, ph = np.meshgrid(np.arccos(mu), sht.phi_grid(nphi), indexing="ij")
    ref = np.zeros((L + 1, nphi))
    for i, (l, m) in enumerate(zip(*simgen.lm_arrays(L))):
        ref += (1 if m == 0 else 2) * (sph_harm_y(l, m, th, ph) * a[i]).real
    D = sht.legendre_sums(a, L, np.ones((1, L + 1)), mu)
    good = sht.fourier_synthesis(D, nphi)[0]
    assert np.max(np.abs(good - ref)) < 1e-12
    # c_m = 1 for every m (the -m partner forgotten)
    ms = np.arange(L + 1)
    bad1 = np.real(D[0].T @ np.exp(1j * np.outer(ms, sht.phi_grid(nphi))))
    assert np.max(np.abs(bad1 - ref)) > 1e-3
    # Condon-Shortley phase dropped
    tab = sht.legendre_table(L, mu)
    _, midx = simgen.lm_arrays(L)
    sign = np.where(midx % 2 == 1, -1.0, 1.0)[:, None]
    bad_tab = tab * sign
    Dbad = np.zeros_like(D)
    for m in range(L + 1):
        s = simgen.alm_index(m, m, L)
        Dbad[0, m] = a[s: s + L - m + 1] @ bad_tab[s: s + L - m + 1]
    assert np.max(np.abs(sht.fourier_synthesis(Dbad, nphi)[0] - ref)) > 1e-3


def test_planted_alpha_mistake_is_caught():
    L, P = 7, 2
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    ref = _alpha_bruteforce(filt, cl)
    x, wx = np.polynomial.legendre.leggauss(L + 6)
    Pl = modal._legendre_table(L, x)
    A = modal._legendre_sum(filt * cl[None, :], Pl)
    D = modal._legendre_sum(filt, Pl)
    bad = np.array([16 * math.pi ** 2 * np.sum(wx * (A[p] * A[r] * D[s] + A[p] * D[r] * A[s]))
                    for (p, r, s) in modal.mode_list(P)])        # one permutation dropped
    assert np.max(np.abs(bad - ref)) > 1e-3 * np.max(np.abs(ref))


def _ring_parseval(D: np.ndarray) -> np.ndarray:
    """Longitude mean of M_a M_b on each ring from the Fourier coefficients alone:
    D_a0 D_b0 + 2 Re sum_{m>=1} D_am conj(D_bm) (Parseval on N_phi > 2 l_max points)."""
    P = D.shape[0]
    out = []
    for (a, b) in modal.pair_list(P):
        v = np.real(D[a, 0]) * np.real(D[b, 0]) + 2.0 * np.real(np.sum(D[a, 1:] * np.conj(D[b, 1:]), axis=0))
        out.append(v)
    return np.stack(out)                                   # [N_pair][R]


def test_ring_pair_means_match_parseval_on_each_ring():
    """The ring-only pair means (pixel means averaged over longitudes) equal the Fourier-
    space form of the same ring average for every ring and pair."""
    L, P, R, nphi = 20, 4, 21, 64
    basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
    filt = sht.filter_table(basis, cl)
    mu, _ = sht.gl_nodes(R)
    sims = simgen.gaussian_alm(cl, 3, seed=17, stream=simgen.STREAM_LINEAR)
    pm = modal.pair_means([sht.synthesize(a, L, filt, mu, nphi) for a in sims])
    ring = modal.ring_pair_means(pm)
    assert ring.shape == pm.shape
    expect = np.mean([_ring_parseval(sht.legendre_sums(a, L, filt, mu)) for a in sims], axis=0)
    np.testing.assert_allclose(ring[:, :, 0], expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())
    assert np.all(ring == ring[:, :, :1])                  # constant along each ring
    # a planted mistake (averaging over rings instead of longitudes) fails the pin
    wrong = np.repeat(pm.mean(axis=1, keepdims=True), R, axis=1)
    assert not np.allclose(wrong[:, :, 0], expect, rtol=1e-6)


def test_ring_pair_means_equal_pixel_means_for_axisymmetric_sims():
    """Simulations with a_lm = 0 for m > 0 are constant along rings, so the ring-only and
    the pixel means coincide, and so do the two linear terms of beta."""
    L, P, R, nphi = 16, 3, 17, 64
    basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
    filt = sht.filter_table(basis, cl)
    mu, w = sht.gl_nodes(R)
    sims = simgen.gaussian_alm(cl, 2, seed=18, stream=simgen.STREAM_LINEAR)
    m_of = np.concatenate([np.full(L - m + 1, m) for m in range(L + 1)])
    sims[:, m_of > 0] = 0.0
    pm = modal.pair_means([sht.synthesize(a, L, filt, mu, nphi) for a in sims])
    np.testing.assert_allclose(modal.ring_pair_means(pm), pm, rtol=1e-12, atol=1e-14 * np.abs(pm).max())
    maps = sht.synthesize(simgen.gaussian_alm(cl, 1, seed=19)[0], L, filt, mu, nphi)
    W = modal.pixel_weights(w, nphi)
    np.testing.assert_allclose(modal.cubic_beta(maps, W, modal.ring_pair_means(pm)), modal.cubic_beta(maps, W, pm),
                               rtol=1e-10, atol=1e-12)


def test_bivector_fit_and_solve_reduce_to_the_full_solve():
    """For a covariance that is exactly L0 (I + b b^T) L0^T the fit returns b, and the
    bivector estimate and sigma equal the general Cholesky solve of Eq. modalest."""
    g = np.random.default_rng(21)
    n = 9
    A = g.standard_normal((n, n))
    zeta0 = A @ A.T + n * np.eye(n)
    b = np.abs(g.standard_normal(n)) + 0.1                # positive sum fixes the sign convention
    L0 = np.linalg.cholesky(zeta0)
    zeta = L0 @ (np.eye(n) + np.outer(b, b)) @ L0.T
    np.testing.assert_allclose(modal.bivector_fit(zeta, zeta0), b, rtol=1e-10, atol=1e-12)
    alpha = g.standard_normal(n)
    betas = g.standard_normal((4, n))
    fnl, sigma = modal.solve_fnl_bivector(zeta0, b, alpha, betas)
    fnl_ref, sigma_ref = modal.solve_fnl(zeta, alpha, betas)
    np.testing.assert_allclose(fnl, fnl_ref, rtol=1e-10, atol=1e-12)
    assert sigma == pytest.approx(sigma_ref, rel=1e-10)
    # a planted mistake (the inverse without the 1 + |b|^2 denominator) fails the pin
    wrong = np.eye(n) - np.outer(b, b)
    a = np.linalg.solve(L0, alpha)
    B = np.linalg.solve(L0, betas.T)
    assert not np.allclose((a @ wrong @ B) / (a @ wrong @ a), fnl_ref, rtol=1e-6)


# ---------------------------------------------------------------- quartic (trispectrum) modes

def test_gaunt4_matches_direct_quadrature():
    """The four-harmonic Gaunt integral against a Gauss-Legendre x uniform-phi quadrature
    of scipy's Y_lm product (exact for these degrees)."""
    from scipy.special import sph_harm_y
    nr, nphi = 12, 32
    mu, w = sht.gl_nodes(nr)
    th = np.arccos(mu)[:, None]
    ph = (2 * np.pi * np.arange(nphi) / nphi)[None, :]
    g = np.random.default_rng(5)
    checked = 0
    while checked < 12:
        ls = g.integers(0, 5, size=4)
        ms = [int(g.integers(-l, l + 1)) for l in ls[:3]]
        ms.append(-sum(ms))
        if abs(ms[3]) > ls[3] or sum(ls) % 2:
            continue
        prod = np.ones((nr, nphi), dtype=complex)
        for l, m in zip(ls, ms):
            prod = prod * sph_harm_y(int(l), int(m), th, ph)
        ref = np.sum(w[:, None] * (2 * np.pi / nphi) * prod)
        assert wigner.gaunt4(*[int(v) for v in ls], *ms) == pytest.approx(ref.real, abs=1e-12)
        assert abs(ref.imag) < 1e-12
        checked += 1


def test_quartic_grid_sum_equals_gaunt_bruteforce():
    """On an exact-quartic grid (R >= 2L + 1 rings, nphi >= 4L + 1) the grid sum of
    M_p M_r M_s M_u equals the four-harmonic Gaunt sum of Sec. IV."""
    L, P = 5, 2
    nr, nphi = 2 * L + 1, 32
    mu, w, W = _grid(nr, nphi)
    cl = simgen.cl_model(L)
    filt = sht.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    a = simgen.gaussian_alm(cl, 1, seed=44)[0]
    got = modal.quartic_tau(sht.synthesize(a, L, filt, mu, nphi), W)
    ref = wigner.gaunt_tau(a, L, filt)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def _quad_multiplicity(q):
    c = np.bincount(np.asarray(q), minlength=4)
    return math.factorial(4) // int(np.prod([math.factorial(int(k)) for k in c]))


def _hermite_check(tau_fn, P=3, seed=6):
    """Constant fields M_a = m_a, <ab> = C_ab: for every direction t the full symmetric
    contraction sum t_p t_r t_s t_u tau equals sum_x W (t'Ct)^2 He4(t.m / sqrt(t'Ct)),
    He4 the probabilists' Hermite polynomial (Isserlis' theorem); the values on all t
    determine the symmetric tensor, so every coefficient and index is checked."""
    from numpy.polynomial import hermite_e
    g = np.random.default_rng(seed)
    nr, nphi = 5, 16
    W = g.uniform(0.5, 1.5, size=(nr, nphi))
    m = g.standard_normal(P)
    A = g.standard_normal((P, P))
    C = A @ A.T + 0.5 * np.eye(P)
    maps = np.broadcast_to(m[:, None, None], (P, nr, nphi)).copy()
    pm = np.stack([np.full((nr, nphi), C[a, b]) for (a, b) in modal.pair_list(P)])
    tau = tau_fn(maps, W, pm)
    worst = 0.0
    for _ in range(8):
        t = g.standard_normal(P)
        lhs = sum(_quad_multiplicity(q) * t[q[0]] * t[q[1]] * t[q[2]] * t[q[3]] * tau[n]
                  for n, q in enumerate(modal.quad_list(P)))
        s = t @ C @ t
        rhs = W.sum() * s * s * hermite_e.hermeval((t @ m) / math.sqrt(s), [0, 0, 0, 0, 1])
        worst = max(worst, abs(lhs - rhs) / max(abs(rhs), 1e-300))
    return worst


def test_quartic_constant_fields_give_the_hermite_polynomial():
    assert _hermite_check(modal.quartic_tau) < 1e-12


def test_quartic_single_pair_term_by_imaginary_shift():
    """Re prod_i (M + i M')_i = M^4 - sum_6 M'M' M M + M'^4, so over the simulations that
    define <ab>:  tau(M) = mean_i Re Q(M + i M'_i) - mean_i Q(M'_i) + tau(0), with Q the
    quartic sum alone and tau(0) = sum_x W sum_3 <ab><cd>."""
    M, sims, W, P = _antithetic_setup(P=3)
    pm = modal.pair_means(sims)
    lhs = modal.quartic_tau(M, W, pm)
    rhs = (np.mean([modal.quartic_tau(M + 1j * s, W).real for s in sims], axis=0)
           - np.mean([modal.quartic_tau(s, W) for s in sims], axis=0)
           + modal.quartic_tau(np.zeros_like(M), W, pm))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-11 * np.abs(lhs).max())


def test_planted_quartic_mistakes_are_caught():
    """Copies of quartic_tau with one mistake each fail the Hermite pin."""
    def variant(kind):
        def fn(maps, W, pairmean):
            P = maps.shape[0]
            pidx = {pr: i for i, pr in enumerate(modal.pair_list(P))}
            Mf, pmf, Wf = maps.reshape(P, -1), pairmean.reshape(pairmean.shape[0], -1), W.ravel()
            mean = lambda a, b: pmf[pidx[(min(a, b), max(a, b))]]
            splits = modal._QUAD_SPLITS[:3] if kind == "three_splits" else modal._QUAD_SPLITS
            match = ((0, 1, 2, 3),) * 3 if kind == "one_matching" else modal._QUAD_MATCHINGS
            sign = -1.0 if kind == "matching_sign" else 1.0
            out = []
            for q in modal.quad_list(P):
                v = np.sum(Wf * Mf[q[0]] * Mf[q[1]] * Mf[q[2]] * Mf[q[3]])
                for (i, j, k, l) in splits:
                    v -= np.sum(Wf * mean(q[i], q[j]) * Mf[q[k]] * Mf[q[l]])
                for (i, j, k, l) in match:
                    v += sign * np.sum(Wf * mean(q[i], q[j]) * mean(q[k], q[l]))
                out.append(v)
            return np.array(out)
        return fn
    for kind in ("three_splits", "one_matching", "matching_sign"):
        assert _hermite_check(variant(kind)) > 1e-3, kind


def test_fnl_weights_are_the_derivative_of_the_estimate():
    """w = d fNL / d beta: fNL(beta) = w . beta for random beta (fNL is linear in beta), the
    identity covariance gives alpha / |alpha|^2, and under a mode transform T (beta -> T beta,
    alpha -> T alpha, zeta -> T zeta T^T) the weights become T^-T w."""
    rng = np.random.default_rng(7)
    n = 20
    X = rng.standard_normal((3 * n, n))
    zeta = X.T @ X / (3 * n) + 0.1 * np.eye(n)
    alpha = rng.standard_normal(n)
    betas = rng.standard_normal((5, n))
    w = modal.fnl_weights(zeta, alpha)
    fnl, _ = modal.solve_fnl(zeta, alpha, betas)
    assert np.allclose(betas @ w, fnl, rtol=1e-12, atol=1e-12)
    assert np.allclose(modal.fnl_weights(np.eye(n), alpha), alpha / (alpha @ alpha), rtol=1e-13)
    T = simgen.random_modes_matrix(n, seed=8)
    wT = modal.fnl_weights(T @ zeta @ T.T, T @ alpha)
    assert np.allclose(wT, np.linalg.solve(T.T, w), rtol=1e-9, atol=1e-12)
