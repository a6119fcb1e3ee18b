"""Oracle: grid, Legendre functions, direct synthesis and analysis (FP64).

Test infrastructure only (see the package header).

The maps the estimator cubes are the filtered maps
    M_p(x) = sum_{l,m} q_p(l) a_lm / sqrt(C_l) Y_lm(x)
of the separable modal basis (Sec. III.A, the isotropic basis Eq. isobasisbi
with v_l = 1 and the Gaunt integral of Sec. II).  Y_lm carries the
Condon-Shortley phase; a_lm obeys the real-field convention
a_{l,-m} = (-1)^m conj(a_lm).  Sums over the sphere are Gauss-Legendre
quadratures on rings of constant theta.

Pins (tests/test_oracle_sht.py): Gauss-Legendre nodes against numpy's
routine and exact monomial integrals; lambda_lm against explicit low-l
formulas, scipy's spherical harmonics and high-precision mpmath values near
the poles at l, m ~ 2000; the addition theorem; synthesis against scipy's
Y_lm at random points; analysis(synthesis(a)) = a.
"""
from __future__ import annotations

import math
import numpy as np


def gl_nodes(n: int):
    """Gauss-Legendre nodes mu_j = cos(theta_j), north first, and weights w_j.

    Roots of P_n by Newton's method from the asymptotic guess
    cos(pi (j + 3/4) / (n + 1/2)); w_j = 2 / ((1 - mu_j^2) P_n'(mu_j)^2).
    The southern half is the mirror image of the northern half, so
    mu_{n-1-j} = -mu_j exactly and an odd n has a ring at mu = 0.
    """
    half = (n + 1) // 2
    j = np.arange(half, dtype=float)
    x = np.cos(np.pi * (j + 0.75) / (n + 0.5))
    for _ in range(100):
        p_prev = np.ones_like(x)
        p = x.copy()
        for k in range(2, n + 1):
            p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
        if n == 1:
            p_prev, p = np.ones_like(x), x.copy()
        dp = n * (x * p - p_prev) / (x * x - 1.0)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p_prev = np.ones_like(x)
    p = x.copy()
    for k in range(2, n + 1):
        p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
    dp = n * (x * p - p_prev) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    if n % 2 == 1:
        x[-1] = 0.0
    mu = np.concatenate([x, -x[: n // 2][::-1]])
    wt = np.concatenate([w, w[: n // 2][::-1]])
    return mu, wt


def legendre_table(lmax: int, mu) -> np.ndarray:
    """lambda_lm(theta) for all 0 <= m <= l <= lmax at mu = cos(theta); [n_alm][len(mu)],
    rows in the packed m-major order idx(l, m) = m (2 lmax + 3 - m) / 2 + (l - m).

    lambda_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_lm(mu), Condon-Shortley
    phase, so that Y_lm = lambda_lm e^{i m phi}.  Start
        lambda_mm = (-1)^m sqrt((2m+1)/(4 pi) prod_{k=1..m} (2k-1)/(2k)) sin^m theta,
        lambda_{m+1,m} = mu sqrt(2m+3) lambda_mm,
    then the three-term recurrence
        lambda_lm = a_lm (mu lambda_{l-1,m} - lambda_{l-2,m} / a_{l-1,m}),
        a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)).
    The recurrence runs on a mantissa v with a separate power-of-two exponent
    e per (m, ring), lambda = v 2^e: lambda_mm underflows FP64 near the poles
    for large m while later lambda_lm need not.  v is renormalised by 2^-200
    whenever it exceeds 2^200; values below the FP64 range come out as zero.
    All m advance together: step d computes l = m + d for every m <= lmax - d.
    """
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    R = mu.size
    L1 = lmax + 1
    out = np.zeros(((L1 * (L1 + 1)) // 2, R))
    m = np.arange(L1, dtype=float)
    starts = (np.arange(L1) * (2 * lmax + 3 - np.arange(L1))) // 2
    s2 = 1.0 - mu * mu
    k = np.arange(1, L1, dtype=float)
    logprod = np.concatenate([[0.0], np.cumsum(np.log2((2 * k - 1) / (2 * k)))])
    log2c = 0.5 * (np.log2((2 * m + 1) / (4.0 * math.pi)) + logprod)          # [m]
    with np.errstate(divide="ignore", invalid="ignore"):
        log2s = np.where(m[:, None] > 0, 0.5 * m[:, None] * np.log2(s2)[None, :], 0.0)
    l2 = log2c[:, None] + log2s                                                  # [m][ring]
    ok = np.isfinite(l2)
    e = np.floor(np.where(ok, l2, -1e6)).astype(np.int64)
    sign = np.where(np.arange(L1) % 2 == 1, -1.0, 1.0)
    v_prev = np.where(ok, sign[:, None] * np.exp2(np.where(ok, l2 - e, 0.0)), 0.0)  # d = 0

    def emit(v, ex):
        return np.ldexp(v, np.clip(ex, -4000, 4000).astype(np.int32))

    out[starts] = emit(v_prev, e)
    if lmax == 0:
        return out
    # d = 1 (exists for m <= lmax - 1)
    n1 = lmax
    v_cur = mu[None, :] * np.sqrt(2 * m[:n1] + 3)[:, None] * v_prev[:n1]
    out[starts[:n1] + 1] = emit(v_cur, e[:n1])
    v_prev = v_prev[:n1]
    e = e[:n1]
    big = 2.0 ** 200
    for d in range(2, L1):
        n = L1 - d                                   # m = 0..n-1
        mm = m[:n]
        l = mm + d
        a = np.sqrt((4.0 * l * l - 1.0) / (l * l - mm * mm))
        b = np.sqrt(((l - 1.0) ** 2 - mm * mm) / (4.0 * (l - 1.0) ** 2 - 1.0))
        v_new = a[:, None] * (mu[None, :] * v_cur[:n] - b[:, None] * v_prev[:n])
        v_prev, v_cur, e = v_cur[:n], v_new, e[:n]
        over = np.abs(v_cur) > big
        if over.any():
            v_prev = np.where(over, v_prev / big, v_prev)
            v_cur = np.where(over, v_cur / big, v_cur)
            e = np.where(over, e + 200, e)
        out[starts[:n] + d] = emit(v_cur, e)
    return out


def legendre_lambda(lmax: int, m: int, mu) -> np.ndarray:
    """lambda_lm for l = m..lmax at mu; [lmax-m+1][len(mu)] (a slice of legendre_table)."""
    start = m * (2 * lmax + 3 - m) // 2
    return legendre_table(lmax, mu)[start: start + lmax - m + 1]


def filter_table(basis: np.ndarray, cl: np.ndarray) -> np.ndarray:
    """f_p(l) = q_p(l) / sqrt(C_l), zero where C_l = 0 (the whitening of Eq. legoestimator)."""
    cl = np.asarray(cl, dtype=float)
    inv = np.zeros_like(cl)
    pos = cl > 0
    inv[pos] = 1.0 / np.sqrt(cl[pos])
    return np.asarray(basis, dtype=float) * inv[None, :]


def _alm_m(alm: np.ndarray, lmax: int, m: int) -> np.ndarray:
    start = m * (2 * lmax + 3 - m) // 2
    return alm[start: start + lmax - m + 1]


def phi_grid(nphi: int) -> np.ndarray:
    return 2.0 * np.pi * np.arange(nphi) / nphi


RING_BLOCK = 32


def ring_blocks(nrings: int):
    for r0 in range(0, nrings, RING_BLOCK):
        yield slice(r0, min(nrings, r0 + RING_BLOCK))


def legendre_sums(alm: np.ndarray, lmax: int, filt: np.ndarray, mu) -> np.ndarray:
    """D_pm(theta_j) = sum_{l >= m} lambda_lm(theta_j) f_p(l) a_lm; complex [P][lmax+1][len(mu)]."""
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    filt = np.atleast_2d(filt)
    P = filt.shape[0]
    D = np.zeros((P, lmax + 1, mu.size), dtype=np.complex128)
    for blk in ring_blocks(mu.size):
        lam = legendre_table(lmax, mu[blk])                       # [idx(l,m)][ring]
        for m in range(lmax + 1):
            start = m * (2 * lmax + 3 - m) // 2
            coef = filt[:, m:] * _alm_m(alm, lmax, m)[None, :]    # [p][l]
            D[:, m, blk] = coef @ lam[start: start + lmax - m + 1]
    return D


def fourier_synthesis(D: np.ndarray, nphi: int) -> np.ndarray:
    """M(theta, phi_k) = D_0 + 2 Re sum_{m>=1} D_m e^{i m phi_k}; D [P][lmax+1][R] -> [P][R][nphi]."""
    P, L1, R = D.shape
    ms = np.arange(L1)
    phase = np.exp(1j * np.outer(ms, phi_grid(nphi)))             # [m][k]
    cm = np.where(ms == 0, 1.0, 2.0)
    maps = np.empty((P, R, nphi))
    for p in range(P):
        maps[p] = np.real(D[p].T @ (cm[:, None] * phase))
    return maps


def synthesize(alm: np.ndarray, lmax: int, filt: np.ndarray, mu, nphi: int) -> np.ndarray:
    """Filtered maps M_p on rings mu x nphi longitudes; [P][len(mu)][nphi].

    Direct Legendre sum per (ring, m):  D_pm(theta) = sum_l lambda_lm f_p(l) a_lm,
    then the direct Fourier sum over m:
        M_p(theta, phi_k) = D_p0 + 2 Re sum_{m=1..lmax} D_pm e^{i m phi_k},
    which is the sum over all m of the real field.
    """
    return fourier_synthesis(legendre_sums(alm, lmax, filt, mu), nphi)


def fourier_analysis(maps: np.ndarray, lmax: int, nphi: int) -> np.ndarray:
    """T~_m(theta_j) = sum_k T(j, k) e^{-i m phi_k}, m = 0..lmax; [...][R][lmax+1]."""
    ms = np.arange(lmax + 1)
    phase = np.exp(-1j * np.outer(phi_grid(nphi), ms))            # [k][m]
    return np.asarray(maps) @ phase


def legendre_analysis(Tm: np.ndarray, lmax: int, mu, wring) -> np.ndarray:
    """a_lm = sum_j wring_j lambda_lm(theta_j) T~_m(theta_j); Tm [R][lmax+1] -> complex [n_alm]."""
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    out = np.zeros((lmax + 1) * (lmax + 2) // 2, dtype=np.complex128)
    for blk in ring_blocks(mu.size):
        lam = legendre_table(lmax, mu[blk])
        wt = (np.asarray(wring)[blk])[:, None] * Tm[blk]           # [ring][m]
        for m in range(lmax + 1):
            start = m * (2 * lmax + 3 - m) // 2
            out[start: start + lmax - m + 1] += lam[start: start + lmax - m + 1] @ wt[:, m]
    return out


def analyze(maps: np.ndarray, lmax: int, mu, w, nphi: int) -> np.ndarray:
    """Quadrature analysis a_lm = sum_x Omega_x T(x) conj(Y_lm(x)), Omega_x = w_j 2 pi / nphi.

    maps: [nrings][nphi] (one map).  Direct Fourier sum over longitudes, then the
    direct Legendre sum over rings.  Exact inverse of synthesis for band-limited
    maps when the grid integrates degree 2 lmax exactly.
    """
    Tm = (2.0 * np.pi / nphi) * fourier_analysis(maps, lmax, nphi)
    return legendre_analysis(Tm, lmax, mu, w)


def legendre_sums_many(alms: np.ndarray, lmax: int, filt: np.ndarray, mu) -> np.ndarray:
    """legendre_sums for several maps, the lambda table of each ring block formed once:
    complex [nmaps][P][lmax+1][len(mu)]."""
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    filt = np.atleast_2d(filt)
    alms = np.atleast_2d(alms)
    D = np.zeros((alms.shape[0], filt.shape[0], lmax + 1, mu.size), dtype=np.complex128)
    for blk in ring_blocks(mu.size):
        lam = legendre_table(lmax, mu[blk])
        for m in range(lmax + 1):
            start = m * (2 * lmax + 3 - m) // 2
            lam_m = lam[start: start + lmax - m + 1]
            for i in range(alms.shape[0]):
                coef = filt[:, m:] * _alm_m(alms[i], lmax, m)[None, :]
                D[i, :, m, blk] = coef @ lam_m
    return D


def synthesize_many(alms: np.ndarray, lmax: int, filt: np.ndarray, mu, nphi: int) -> np.ndarray:
    """synthesize for several maps: [nmaps][P][len(mu)][nphi]."""
    D = legendre_sums_many(alms, lmax, filt, mu)
    return np.stack([fourier_synthesis(D[i], nphi) for i in range(D.shape[0])])


def analyze_many(maps: np.ndarray, lmax: int, mu, w, nphi: int) -> np.ndarray:
    """analyze for several maps [nmaps][nrings][nphi], the lambda table of each ring block
    formed once: complex [nmaps][n_alm]."""
    maps = np.asarray(maps)
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    Tm = (2.0 * np.pi / nphi) * fourier_analysis(maps, lmax, nphi)       # [map][ring][m]
    out = np.zeros((maps.shape[0], (lmax + 1) * (lmax + 2) // 2), dtype=np.complex128)
    for blk in ring_blocks(mu.size):
        lam = legendre_table(lmax, mu[blk])
        wt = (np.asarray(w)[blk])[None, :, None] * Tm[:, blk]         # [map][ring][m]
        for m in range(lmax + 1):
            start = m * (2 * lmax + 3 - m) // 2
            out[:, start: start + lmax - m + 1] += (lam[start: start + lmax - m + 1] @ wt[:, :, m].T).T
    return out
