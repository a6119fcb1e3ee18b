"""Oracle: modal coefficients, linear term, covariance, estimator (FP64).

Test infrastructure only (see the package header).

Orderings shared with the library:
  * modes n <-> (p, r, s), p <= r <= s, lexicographic; n_max = C(P+2, 3);
  * pairs (p, r), p <= r, lexicographic; N_pair = P (P + 1) / 2;
  * quartic modes (p, r, s, u), p <= r <= s <= u, lexicographic; C(P+3, 4) of them.

What each function follows:
  cubic_beta       Eq. bbispect: beta_n = sum G (a a a - 3 C a) R_n / sqrt(CCC).
                   With the separable R_n = q_p q_r q_s and v_l = 1 the Gaunt sum is
                   the sphere integral of M_p M_r M_s, taken as the grid quadrature
                   sum_x W_x M_p M_r M_s, W_x = w_j (2 pi / N_phi) mask_x.  The linear
                   term -3 C a of Eq. bispectrumest, symmetrised over the ordered
                   triple, is -sum_x W_x (<M_p M_r>_x M_s + <M_p M_s>_x M_r + <M_r M_s>_x M_p),
                   with <.> the Monte Carlo mean over Gaussian simulations (Sec. II).
  pair_means       the Monte Carlo mean <M_p M_r>_x of Sec. II ("calculated from Monte
                   Carlo simulations of Gaussian maps").
  ring_pair_means  the same mean averaged over the longitudes of each ring: for weights,
                   noise and mask that depend on the ring alone (the anisotropic noise
                   and band mask of App. A) the pixel mean is a function of the ring in
                   expectation, so the ring average estimates it with N_phi times as many
                   samples (a reading, not printed in the paper).
  covariance_zeta  zeta = <beta beta^T> / 6 (Eq. linearterm, Sec. II with p! = 6),
                   read as the unbiased sample covariance divided by 6.
  solve_fnl        Eq. modalest and Eq. modalvariance via the Cholesky rotation
                   (Eq. Cholrot): E = alpha'.beta' / |alpha'|^2, sigma^2 = 6 / |alpha'|^2.
  fnl_weights      d fNL / d beta of Eq. modalest (fNL is linear in beta):
                   zeta^-1 alpha / (alpha^T zeta^-1 alpha).
  alpha_local      Eq. abispect for b = 2 f (C1 C2 + C2 C3 + C3 C1), the first-order
                   bispectrum of T = G + f (G^2 - <G^2>), evaluated through the identity
                   sum h^2 F G H = 8 pi^2 int f g h dmu (h from Sec. III.A).
  zeta_closed_form the full-sky covariance of beta for Gaussian maps (six cross
                   pairings of Eq. linearterm), by the same identity.
  quartic_tau      the trispectrum modes of Sec. IV (the B term of its estimator with the
                   four-harmonic Gaunt integral): sum_x W [M_p M_r M_s M_u - sum over the 6
                   single pairs <ab> M_c M_d + sum over the 3 pair splits <ab><cd>], the
                   "-6 C a a" and "+3 C C" of Sec. IV symmetrised over the ordered quadruple.
  adjoint_grad     derivative of sum_n g_n beta_n with respect to (Re a_lm, Im a_lm),
                   m >= 0 (not in the paper; chain rule through cubic_beta and synthesis).
  bivector_*       Eq. ic_bivector, ic_bivectorinv, bivecvariance and the analytic
                   Cholesky factor of Sec. III.B.
  bivector_fit,    the bivector model with an ideal covariance zeta0 = L0 L0^T (full sky,
  solve_fnl_bivector  homogeneous noise): zeta ~ L0 (I + bt bt^T) L0^T, bt = sqrt(l1) u1 from
                   the largest eigenpair of L0^-1 zeta L0^-T - I (a reading: Sec. III.B says
                   only that bt is estimated from simulations), and the estimate of Eq.
                   modalest with the inverse of Eq. ic_bivectorinv in the whitened basis.

Pins: tests/test_oracle_modal.py (Gaunt brute force on an exact-cubic grid,
closed-form covariance and mean, zero mean, larger variance without the linear
term, invariance under mode transforms, finite differences for the adjoint,
bivector identities; for the quartic modes: the four-harmonic Gaunt brute force on an
exact-quartic grid, the multivariate Hermite polynomial for constant fields, and an
imaginary-shift identity for the single-pair term).
"""
from __future__ import annotations

import math
import numpy as np
from scipy.linalg import solve_triangular

from . import sht


def mode_list(P: int):
    """(p, r, s), p <= r <= s, lexicographic."""
    return [(p, r, s) for p in range(P) for r in range(p, P) for s in range(r, P)]


def pair_list(P: int):
    """(p, r), p <= r, lexicographic."""
    return [(p, r) for p in range(P) for r in range(p, P)]


def n_modes(P: int) -> int:
    return P * (P + 1) * (P + 2) // 6


def pixel_weights(w, nphi: int, mask=None) -> np.ndarray:
    """W_x = w_j (2 pi / nphi) mask_x as [nrings][nphi]."""
    w = np.asarray(w, dtype=float)
    W = np.repeat((w * 2.0 * np.pi / nphi)[:, None], nphi, axis=1)
    if mask is not None:
        mask = np.asarray(mask, dtype=float)
        W = W * (mask[:, None] if mask.ndim == 1 else mask)
    return W


def pair_products(maps: np.ndarray) -> np.ndarray:
    """M_p M_r for all pairs, [N_pair][...]."""
    P = maps.shape[0]
    return np.stack([maps[p] * maps[r] for (p, r) in pair_list(P)])


def pair_means(map_batches) -> np.ndarray:
    """<M_p M_r>_x over an iterable of map sets [P][...]; mean over the simulations."""
    acc = None
    n = 0
    for maps in map_batches:
        pp = pair_products(maps)
        acc = pp if acc is None else acc + pp
        n += 1
    return acc / n


def ring_pair_means(pairmean: np.ndarray) -> np.ndarray:
    """Longitude average of <M_p M_r> on every ring, repeated over the ring's pixels;
    [N_pair][nrings][nphi] -> the same shape."""
    ring = pairmean.mean(axis=-1, keepdims=True)
    return np.repeat(ring, pairmean.shape[-1], axis=-1)


def cubic_beta(maps: np.ndarray, W: np.ndarray, pairmean=None) -> np.ndarray:
    """beta_prs = sum_x W_x [M_p M_r M_s - (<pr> M_s + <ps> M_r + <rs> M_p)]; [n_max].

    maps [P][nrings][nphi]; W [nrings][nphi]; pairmean [N_pair][nrings][nphi] or None
    (None: no linear term).  Direct sum over all pixels.
    """
    P = maps.shape[0]
    pidx = {pr: i for i, pr in enumerate(pair_list(P))}
    out = np.empty(n_modes(P))
    flatW = W.ravel()
    M = maps.reshape(P, -1)
    for n, (p, r, s) in enumerate(mode_list(P)):
        val = np.sum(flatW * M[p] * M[r] * M[s])
        if pairmean is not None:
            pm = pairmean.reshape(pairmean.shape[0], -1)
            val -= np.sum(flatW * (pm[pidx[(p, r)]] * M[s] + pm[pidx[(p, s)]] * M[r]
                                   + pm[pidx[(r, s)]] * M[p]))
        out[n] = val
    return out


def quad_list(P: int):
    """(p, r, s, u), p <= r <= s <= u, lexicographic."""
    return [(p, r, s, u) for p in range(P) for r in range(p, P) for s in range(r, P) for u in range(s, P)]


def n_quads(P: int) -> int:
    return P * (P + 1) * (P + 2) * (P + 3) // 24


# the six ways to pick one pair of the four indices (the rest is the other pair) and the
# three ways to split them into two pairs
_QUAD_SPLITS = ((0, 1, 2, 3), (0, 2, 1, 3), (0, 3, 1, 2), (1, 2, 0, 3), (1, 3, 0, 2), (2, 3, 0, 1))
_QUAD_MATCHINGS = ((0, 1, 2, 3), (0, 2, 1, 3), (0, 3, 1, 2))


def quartic_tau(maps: np.ndarray, W: np.ndarray, pairmean=None) -> np.ndarray:
    """Trispectrum modal coefficients (Sec. IV, the B term of the quartic estimator);
    [n_quads].  With R_n = q_p q_r q_s q_u and v_l = 1 the four-harmonic Gaunt sum is the
    sphere integral of M_p M_r M_s M_u, taken as the grid sum with W_x; the -6 C a a and
    +3 C C terms, symmetrised over the ordered quadruple, become the six single-pair and
    the three two-pair contractions with the Monte Carlo means:
      tau = sum_x W [M_p M_r M_s M_u - sum_6 <ab> M_c M_d + sum_3 <ab> <cd>].
    maps [P][...] (complex allowed); W like one map; pairmean [N_pair][...] or None."""
    P = maps.shape[0]
    pidx = {pr: i for i, pr in enumerate(pair_list(P))}
    M = maps.reshape(P, -1)
    flatW = W.ravel()
    pm = None if pairmean is None else pairmean.reshape(pairmean.shape[0], -1)

    def mean(a, b):
        return pm[pidx[(min(a, b), max(a, b))]]

    out = np.empty(n_quads(P), dtype=np.result_type(M.dtype, np.float64))
    for n, q in enumerate(quad_list(P)):
        val = np.sum(flatW * M[q[0]] * M[q[1]] * M[q[2]] * M[q[3]])
        if pm is not None:
            for (i, j, k, l) in _QUAD_SPLITS:
                val -= np.sum(flatW * mean(q[i], q[j]) * M[q[k]] * M[q[l]])
            for (i, j, k, l) in _QUAD_MATCHINGS:
                val += np.sum(flatW * mean(q[i], q[j]) * mean(q[k], q[l]))
        out[n] = val
    return out


def covariance_zeta(betas: np.ndarray) -> np.ndarray:
    """zeta = sample covariance of beta (mean removed, 1/(N-1)) divided by 6."""
    betas = np.asarray(betas, dtype=float)
    N = betas.shape[0]
    mean = betas.mean(axis=0)
    d = betas - mean[None, :]
    return (d.T @ d) / (N - 1) / 6.0


def solve_fnl(zeta: np.ndarray, alpha: np.ndarray, betas: np.ndarray):
    """(fnl[B], sigma): Cholesky zeta = L L^T, alpha' = L^-1 alpha, beta' = L^-1 beta,
    fnl = alpha'.beta' / |alpha'|^2, sigma = sqrt(6 / |alpha'|^2)."""
    Lc = np.linalg.cholesky(zeta)
    ap = solve_triangular(Lc, alpha, lower=True)
    bp = solve_triangular(Lc, np.atleast_2d(betas).T, lower=True)
    norm = float(ap @ ap)
    return (ap @ bp) / norm, math.sqrt(6.0 / norm)


def fnl_weights(zeta: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """d fNL / d beta of Eq. modalest: fNL = alpha^T zeta^-1 beta / alpha^T zeta^-1 alpha is
    linear in beta, w = zeta^-1 alpha / (alpha^T zeta^-1 alpha), by the Cholesky factor
    zeta = L L^T: alpha' = L^-1 alpha, w = L^-T alpha' / |alpha'|^2."""
    Lc = np.linalg.cholesky(zeta)
    ap = solve_triangular(Lc, alpha, lower=True)
    return solve_triangular(Lc.T, ap, lower=False) / float(ap @ ap)


def _legendre_table(lmax: int, x: np.ndarray) -> np.ndarray:
    """P_l(x) for l = 0..lmax by the Bonnet recurrence; [lmax+1][len(x)]."""
    out = np.empty((lmax + 1, x.size))
    out[0] = 1.0
    if lmax >= 1:
        out[1] = x
    for l in range(2, lmax + 1):
        out[l] = ((2 * l - 1) * x * out[l - 1] - (l - 1) * out[l - 2]) / l
    return out


def _legendre_sum(coef_l: np.ndarray, Pl: np.ndarray) -> np.ndarray:
    """sum_l (2l+1)/(4 pi) coef_l P_l(x) for each row of coef_l [k][lmax+1]."""
    l = np.arange(coef_l.shape[-1])
    return (np.atleast_2d(coef_l) * ((2 * l + 1) / (4.0 * math.pi))[None, :]) @ Pl


def alpha_local(filt: np.ndarray, cl_signal: np.ndarray) -> np.ndarray:
    """alpha_prs per unit f for the local shape b = 2 f (C1 C2 + C2 C3 + C3 C1).

    E[beta_prs] = sum_{l} h^2 b f_p(l1) f_r(l2) f_s(l3) = 16 pi^2 int (A_p A_r D_s
    + A_p D_r A_s + D_p A_r A_s) dmu, with A_p = sum (2l+1)/(4pi) C_l f_p(l) P_l and
    D_p = sum (2l+1)/(4pi) f_p(l) P_l; exact Gauss-Legendre integration in mu.
    """
    filt = np.atleast_2d(filt)
    P, L1 = filt.shape
    lmax = L1 - 1
    x, wx = np.polynomial.legendre.leggauss((3 * lmax) // 2 + 2)
    Pl = _legendre_table(lmax, x)
    A = _legendre_sum(filt * np.asarray(cl_signal)[None, :], Pl)
    D = _legendre_sum(filt, Pl)
    out = np.empty(n_modes(P))
    for n, (p, r, s) in enumerate(mode_list(P)):
        out[n] = 16.0 * math.pi ** 2 * np.sum(wx * (A[p] * A[r] * D[s] + A[p] * D[r] * A[s]
                                                      + D[p] * A[r] * A[s]))
    return out


def zeta_closed_form(filt: np.ndarray, cl_total: np.ndarray) -> np.ndarray:
    """zeta for Gaussian full-sky maps with power C_l (no mask, isotropic noise in C_l).

    cov(beta_prs, beta_p'r's') = 8 pi^2 sum over the 6 permutations sigma of (p', r', s')
    of int xi_{p sigma1} xi_{r sigma2} xi_{s sigma3} dmu,
    xi_pq = sum_l (2l+1)/(4pi) f_p(l) f_q(l) C_l P_l(mu);  zeta = cov / 6.
    Exact for the Gaunt-sum beta (an exact-cubic grid) with the exact linear term.
    """
    filt = np.atleast_2d(filt)
    P, L1 = filt.shape
    lmax = L1 - 1
    x, wx = np.polynomial.legendre.leggauss((3 * lmax) // 2 + 2)
    Pl = _legendre_table(lmax, x)
    xi = np.empty((P, P, x.size))
    for p in range(P):
        for q in range(P):
            xi[p, q] = _legendre_sum((filt[p] * filt[q] * cl_total)[None, :], Pl)[0]
    modes = mode_list(P)
    n = len(modes)
    cov = np.empty((n, n))
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    for i, (p, r, s) in enumerate(modes):
        for j, t in enumerate(modes):
            acc = 0.0
            for (a, b, c) in perms:
                acc += np.sum(wx * xi[p, t[a]] * xi[r, t[b]] * xi[s, t[c]])
            cov[i, j] = 8.0 * math.pi ** 2 * acc
    return cov / 6.0


def symmetric_g(g: np.ndarray, P: int) -> np.ndarray:
    """h_abc = g_{sort(a,b,c)} / (number of distinct orderings), so that
    sum_n g_n beta_n = sum_x W sum_{a,b,c} h_abc (M_a M_b M_c - 3 <ab> M_c)."""
    h = np.zeros((P, P, P))
    for n, (p, r, s) in enumerate(mode_list(P)):
        perms = {(p, r, s), (p, s, r), (r, p, s), (r, s, p), (s, p, r), (s, r, p)}
        for (a, b, c) in perms:
            h[a, b, c] = g[n] / len(perms)
    return h


def adjoint_grad(alm, g, lmax, filt, mu, w, nphi, mask=None, pairmean=None) -> np.ndarray:
    """d(sum_n g_n beta_n)/d(Re a_lm) + i d(...)/d(Im a_lm) for stored m >= 0; complex [n_alm].

    U_t(x) = 3 W_x sum_ab h_tab (M_a M_b - <ab>_x)   (derivative w.r.t. M_t(x)),
    U~_tm(theta_j) = sum_k U_t(j,k) e^{-i m phi_k},
    grad_lm = c_m sum_t f_t(l) sum_j lambda_lm(theta_j) U~_tm(theta_j), c_0 = 1, c_m>0 = 2.
    """
    filt = np.atleast_2d(filt)
    P = filt.shape[0]
    maps = sht.synthesize(alm, lmax, filt, mu, nphi)
    W = pixel_weights(w, nphi, mask)
    h = symmetric_g(np.asarray(g, dtype=float), P)
    pidx = {pr: i for i, pr in enumerate(pair_list(P))}
    U = np.zeros_like(maps)
    for t in range(P):
        acc = np.zeros(maps.shape[1:])
        for a in range(P):
            for b in range(P):
                if h[t, a, b] == 0.0:
                    continue
                y = maps[a] * maps[b]
                if pairmean is not None:
                    y = y - pairmean[pidx[(min(a, b), max(a, b))]]
                acc += h[t, a, b] * y
        U[t] = 3.0 * W * acc
    out = np.zeros((lmax + 1) * (lmax + 2) // 2, dtype=np.complex128)
    for t in range(P):
        Ut = sht.fourier_analysis(U[t], lmax, nphi)                # [ring][m]
        cm = np.where(np.arange(lmax + 1) == 0, 1.0, 2.0)
        a_t = sht.legendre_analysis(Ut * cm[None, :], lmax, mu, np.ones(len(np.atleast_1d(mu))))
        lidx = np.concatenate([np.arange(mm, lmax + 1) for mm in range(lmax + 1)])
        out += filt[t][lidx] * a_t
    return out


def bivector_inverse(bt: np.ndarray) -> np.ndarray:
    """Eq. ic_bivectorinv: (I + b b^T)^-1 = I - b b^T / (1 + |b|^2)."""
    return np.eye(bt.size) - np.outer(bt, bt) / (1.0 + bt @ bt)


def bivector_cholesky(bt: np.ndarray) -> np.ndarray:
    """Analytic lower Cholesky factor of I + b b^T (Sec. III.B):
    diagonal sqrt(S_n / S_{n-1}), below it b_n b_k / sqrt(S_{k-1} S_k), S_n = 1 + sum_{i<=n} b_i^2."""
    n = bt.size
    S = 1.0 + np.concatenate([[0.0], np.cumsum(bt * bt)])       # S[k] = 1 + sum_{i<k} b_i^2
    Lc = np.zeros((n, n))
    for i in range(n):
        Lc[i, i] = math.sqrt(S[i + 1] / S[i])
        for k in range(i):
            Lc[i, k] = bt[i] * bt[k] / math.sqrt(S[k] * S[k + 1])
    return Lc


def bivector_variance(alpha: np.ndarray, bt: np.ndarray) -> float:
    """Eq. bivecvariance: (1/|a|^2) (1 + (a.b)^2 / (|a|^2 (1+|b|^2) - (a.b)^2))."""
    a2 = alpha @ alpha
    ab = alpha @ bt
    return (1.0 / a2) * (1.0 + ab * ab / (a2 * (1.0 + bt @ bt) - ab * ab))


def bivector_fit(zeta: np.ndarray, zeta0: np.ndarray) -> np.ndarray:
    """bt with zeta ~ L0 (I + bt bt^T) L0^T: largest eigenpair (l1, u1) of the whitened
    L0^-1 zeta L0^-T - I, bt = sqrt(max(l1, 0)) u1, sign fixed by a non-negative sum."""
    L0 = np.linalg.cholesky(zeta0)
    Y = solve_triangular(L0, zeta, lower=True)
    Zw = solve_triangular(L0, Y.T, lower=True)
    Zw = 0.5 * (Zw + Zw.T) - np.eye(zeta.shape[0])
    lam, vec = np.linalg.eigh(Zw)
    u = vec[:, -1]
    if u.sum() < 0:
        u = -u
    return math.sqrt(max(lam[-1], 0.0)) * u


def solve_fnl_bivector(zeta0: np.ndarray, bt: np.ndarray, alpha: np.ndarray, betas: np.ndarray):
    """Eq. modalest with zeta = L0 (I + bt bt^T) L0^T: alpha' = L0^-1 alpha, beta' = L0^-1 beta,
    the inverse of Eq. ic_bivectorinv, E = alpha'^T Z^-1 beta' / alpha'^T Z^-1 alpha', and
    sigma^2 = 6 x the variance of Eq. bivecvariance (zeta = <beta beta^T> / 6)."""
    L0 = np.linalg.cholesky(zeta0)
    a = solve_triangular(L0, alpha, lower=True)
    B = solve_triangular(L0, np.atleast_2d(betas).T, lower=True)          # [n][B]
    Zinv = bivector_inverse(bt)
    norm = a @ Zinv @ a
    fnl = (a @ Zinv @ B) / norm
    return fnl, math.sqrt(6.0 * bivector_variance(a, bt))

