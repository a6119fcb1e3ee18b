"""Oracle: Wigner 3j symbols (Racah formula) and the brute-force Gaunt sum.

Test infrastructure only (see the package header).

The Gaunt integral of Sec. II,
    G^{l1 l2 l3}_{m1 m2 m3} = int Y_l1m1 Y_l2m2 Y_l3m3 dOmega
        = sqrt((2l1+1)(2l2+1)(2l3+1)/(4 pi)) (l1 l2 l3; 0 0 0)(l1 l2 l3; m1 m2 m3),
and the harmonic-space form of Eq. bbispect (v_l = 1, R_n = q_p q_r q_s):
    beta_prs = sum_{l_i m_i} G F_p(l1 m1) F_r(l2 m2) F_s(l3 m3),   F_p(l m) = f_p(l) a_lm,
summed over all m_i in [-l_i, l_i] with a_{l,-m} = (-1)^m conj(a_lm).
Pins: tests/test_oracle_modal.py compares the 3j values with sympy's and the
brute-force sum with the grid cubic sum on an exact-cubic grid.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def wigner3j(j1: int, j2: int, j3: int, m1: int, m2: int, m3: int) -> float:
    """(j1 j2 j3; m1 m2 m3) for integer arguments by the Racah formula."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    f = math.factorial
    tri = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pref = f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (f(k) * f(j1 + j2 - j3 - k) * f(j1 - m1 - k) * f(j2 + m2 - k)
               * f(j3 - j2 + m1 + k) * f(j3 - j1 - m2 + k))
        s += Fraction((-1) ** k, den)
    sign = -1.0 if (j1 - j2 - m3) % 2 else 1.0
    return sign * math.sqrt(float(tri * pref)) * float(s)


def gaunt(l1, l2, l3, m1, m2, m3) -> float:
    if (l1 + l2 + l3) % 2:
        return 0.0
    return (math.sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4.0 * math.pi))
            * wigner3j(l1, l2, l3, 0, 0, 0) * wigner3j(l1, l2, l3, m1, m2, m3))


def full_m_coefficients(alm: np.ndarray, lmax: int, filt: np.ndarray):
    """F_p(l, m) for m in [-l, l] from the packed m >= 0 a_lm; returns (list of (l,m), [P][n])."""
    filt = np.atleast_2d(filt)
    lm, vals = [], []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            mm = abs(m)
            a = alm[mm * (2 * lmax + 3 - mm) // 2 + (l - mm)]
            if m < 0:
                a = (-1) ** mm * np.conj(a)
            lm.append((l, m))
            vals.append(a)
    vals = np.array(vals)
    return lm, filt[:, [l for (l, _) in lm]] * vals[None, :]


def gaunt_beta(alm: np.ndarray, lmax: int, filt: np.ndarray) -> np.ndarray:
    """beta_prs by the brute-force Gaunt sum (no linear term); [n_max], p <= r <= s lexicographic."""
    filt = np.atleast_2d(filt)
    P = filt.shape[0]
    lm, F = full_m_coefficients(alm, lmax, filt)
    index = {key: i for i, key in enumerate(lm)}
    T = np.zeros((P, P, P), dtype=np.complex128)
    for i1, (l1, m1) in enumerate(lm):
        for i2, (l2, m2) in enumerate(lm):
            m3 = -m1 - m2
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                if abs(m3) > l3 or (l1 + l2 + l3) % 2:
                    continue
                gv = gaunt(l1, l2, l3, m1, m2, m3)
                if gv == 0.0:
                    continue
                i3 = index[(l3, m3)]
                T += gv * np.einsum("a,b,c->abc", F[:, i1], F[:, i2], F[:, i3])
    out = [T[p, r, s].real for p in range(P) for r in range(p, P) for s in range(r, P)]
    return np.array(out)


def gaunt4(l1, l2, l3, l4, m1, m2, m3, m4) -> float:
    """int Y_l1m1 Y_l2m2 Y_l3m3 Y_l4m4 dOmega (Sec. IV): expand Y_l1m1 Y_l2m2 in Y_LM,
    whose coefficient is int Y_l1m1 Y_l2m2 conj(Y_LM) = (-1)^M G^{l1 l2 L}_{m1 m2 -M}, and
    integrate each term against Y_l3m3 Y_l4m4 (M = m1 + m2)."""
    if m1 + m2 + m3 + m4 != 0:
        return 0.0
    M = m1 + m2
    s = 0.0
    for L in range(max(abs(l1 - l2), abs(l3 - l4), abs(M)), min(l1 + l2, l3 + l4) + 1):
        s += (-1) ** (M % 2) * gaunt(l1, l2, L, m1, m2, -M) * gaunt(L, l3, l4, M, m3, m4)
    return s


def gaunt_tau(alm: np.ndarray, lmax: int, filt: np.ndarray) -> np.ndarray:
    """Quartic modes by the brute-force four-harmonic Gaunt sum (no Monte Carlo terms):
    sum_{l_i m_i} G4 F_p F_r F_s F_u; [C(P+3, 4)], p <= r <= s <= u lexicographic."""
    filt = np.atleast_2d(filt)
    P = filt.shape[0]
    lm, F = full_m_coefficients(alm, lmax, filt)
    live = [i for i, (l, _) in enumerate(lm) if np.any(filt[:, l] != 0.0)]
    index = {key: i for i, key in enumerate(lm)}
    T = np.zeros((P, P, P, P), dtype=np.complex128)
    for i1 in live:
        l1, m1 = lm[i1]
        for i2 in live:
            l2, m2 = lm[i2]
            for i3 in live:
                l3, m3 = lm[i3]
                m4 = -m1 - m2 - m3
                for l4 in range(abs(m4), lmax + 1):
                    i4 = index[(l4, m4)]
                    if i4 not in live or (l1 + l2 + l3 + l4) % 2:
                        continue
                    gv = gaunt4(l1, l2, l3, l4, m1, m2, m3, m4)
                    if gv != 0.0:
                        T += gv * np.einsum("a,b,c,d->abcd", F[:, i1], F[:, i2], F[:, i3], F[:, i4])
    out = [T[p, r, s, u].real for p in range(P) for r in range(p, P) for s in range(r, P) for u in range(s, P)]
    return np.array(out)
