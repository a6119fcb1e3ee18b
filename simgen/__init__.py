"""Seeded synthetic inputs for the modal bispectrum estimator.

This module draws random numbers and builds the fixed input tables (basis,
power spectrum, mask, noise profile).  It holds none of the estimator's
arithmetic: no spherical-harmonic transform, no cubic sum, no covariance.
Both the FP64 oracle and the CUDA path receive exactly the arrays made here.

Random numbers come from Philox4x32-10 (Salmon et al., SC'11), numpy's
``Philox`` bit generator, keyed by (seed, stream) so that the data maps,
the linear-term sims and the covariance sims use disjoint streams.

Conventions shared with the library:
  * a_lm are stored for m >= 0 only, m-major:
        idx(l, m) = m (2 lmax + 3 - m) / 2 + (l - m)
  * real-field convention a_{l,-m} = (-1)^m conj(a_lm), a_l0 real, so for a
    unit-variance field a_l0 ~ N(0, 1) and Re, Im a_lm ~ N(0, 1/2) for m > 0.
"""
from __future__ import annotations

import math
import numpy as np

# Disjoint RNG streams (the second half of the Philox key).
STREAM_DATA = 0
STREAM_LINEAR = 1
STREAM_COV = 2
STREAM_NOISE = 3
STREAM_NG = 4
STREAM_MISC = 5


def n_alm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(l, m, lmax: int):
    """m-major packed index of (l, m), m >= 0."""
    return m * (2 * lmax + 3 - m) // 2 + (l - m)


def lm_arrays(lmax: int):
    """Arrays (l, m) over the packed m-major layout."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def shifted_legendre_basis(lmax: int, P: int) -> np.ndarray:
    """q_p(l) = P_p(2 l / lmax - 1), p = 0..P-1 (unnormalised), as [P][lmax+1] float64."""
    x = 2.0 * np.arange(lmax + 1) / max(lmax, 1) - 1.0
    out = np.empty((P, lmax + 1))
    for p in range(P):
        c = np.zeros(p + 1)
        c[p] = 1.0
        out[p] = np.polynomial.legendre.legval(x, c)
    return out


def cl_model(lmax: int, amplitude: float = 1.0) -> np.ndarray:
    """C_l = A / (l (l + 1)) for l >= 2, zero for l < 2."""
    cl = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1, dtype=float)
    cl[2:] = amplitude / (l * (l + 1.0))
    return cl


def white_alm(lmax: int, nmaps: int, seed: int, stream: int = STREAM_DATA,
              first_map: int = 0) -> np.ndarray:
    """Unit-variance real-field a_lm, complex128 [nmaps][n_alm].

    Map i uses its own Philox key (seed, stream, first_map + i) so a batch can
    be regenerated map by map.
    """
    l, m = lm_arrays(lmax)
    out = np.empty((nmaps, l.size), dtype=np.complex128)
    m0 = (m == 0)
    for i in range(nmaps):
        g = _rng(seed * 1_000_003 + first_map + i, stream)
        z = g.standard_normal((2, l.size))
        re = np.where(m0, z[0], z[0] * math.sqrt(0.5))
        im = np.where(m0, 0.0, z[1] * math.sqrt(0.5))
        out[i] = re + 1j * im
    return out


def gaussian_alm(cl: np.ndarray, nmaps: int, seed: int, stream: int = STREAM_DATA,
                 first_map: int = 0) -> np.ndarray:
    """Gaussian a_lm with power spectrum C_l (real-field convention)."""
    lmax = cl.size - 1
    l, _ = lm_arrays(lmax)
    return white_alm(lmax, nmaps, seed, stream, first_map) * np.sqrt(cl)[l]


def pixel_normals(nrings: int, nphi: int, nmaps: int, seed: int,
                  stream: int = STREAM_NOISE, first_map: int = 0) -> np.ndarray:
    """Standard normal pixel draws xi_x, float64 [nmaps][nrings][nphi]."""
    out = np.empty((nmaps, nrings, nphi))
    for i in range(nmaps):
        out[i] = _rng(seed * 1_000_003 + first_map + i, stream).standard_normal((nrings, nphi))
    return out


def ring_cos_theta(nrings: int) -> np.ndarray:
    """Ring latitudes as cos(theta), north first, from numpy's Gauss-Legendre routine.

    Used only to place the band mask and the noise profile on the rings.
    """
    x, _ = np.polynomial.legendre.leggauss(nrings)
    return x[::-1].copy()


def band_mask(nrings: int, cut_deg: float = 20.0) -> np.ndarray:
    """Ring mask: 0 where |latitude| < cut_deg, 1 elsewhere, float64 [nrings]."""
    mu = ring_cos_theta(nrings)
    return np.where(np.abs(mu) < math.sin(math.radians(cut_deg)), 0.0, 1.0)


def noise_sigma_rings(nrings: int, sigma0_sq: float) -> np.ndarray:
    """Per-ring white-noise level sigma(theta) with sigma^2 = sigma0^2 (1 + 3 cos^2 theta)."""
    mu = ring_cos_theta(nrings)
    return np.sqrt(sigma0_sq * (1.0 + 3.0 * mu * mu))


def random_subset(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct sorted indices from range(n)."""
    g = _rng(seed, STREAM_MISC)
    return np.sort(g.choice(n, size=min(k, n), replace=False))


def random_modes_matrix(n: int, seed: int) -> np.ndarray:
    """A well-conditioned random invertible n x n matrix (identity + small noise)."""
    g = _rng(seed, STREAM_MISC)
    return np.eye(n) + 0.3 * g.standard_normal((n, n)) / math.sqrt(n)


def config(name: str) -> dict:
    """Named workload presets (sizes of the paper's WMAP-resolution and high-l runs)."""
    presets = {
        # l_max = 32, 6 shifted-Legendre modes (n_max = 56); 128 longitudes so that
        # every m <= l_max survives the phi sampling.
        "tiny": dict(lmax=32, nrings=33, nphi=128, P=6, seed=0, mask=False, noise=False),
        # WMAP resolution: l_max = 500, 501 x 1024 grid, 10 modes (n_max = 220),
        # anisotropic noise and a 20-degree band mask.
        "wmap": dict(lmax=500, nrings=501, nphi=1024, P=10, seed=1, mask=True, noise=True,
                     n_lin=256, n_cov=1024),
        # High resolution: l_max = 2000, 2001 x 4096 grid, 16 modes (n_max = 816).
        "l2000": dict(lmax=2000, nrings=2001, nphi=4096, P=16, seed=3, mask=False, noise=False),
        "l1000": dict(lmax=1000, nrings=1001, nphi=2048, P=12, seed=4, mask=True, noise=True),
    }
    return dict(presets[name])


def ring_weights(nrings: int) -> np.ndarray:
    """Gauss-Legendre weights, north first, from numpy's routine (float64 [nrings]).

    Used only to scale the pixel noise draws (noise_maps)."""
    _, w = np.polynomial.legendre.leggauss(nrings)
    return w[::-1].copy()


def noise_maps(nrings: int, nphi: int, nmaps: int, seed: int, sigma0_sq: float,
               stream: int = STREAM_NOISE, first_map: int = 0) -> np.ndarray:
    """White pixel noise n(x) = sigma(theta_j) xi_x / sqrt(Omega_j), Omega_j = w_j 2 pi / nphi,
    sigma^2 = sigma0^2 (1 + 3 cos^2 theta), xi ~ N(0, 1); rounded to float32
    [nmaps][nrings][nphi] so that every consumer reads the same values."""
    sig = noise_sigma_rings(nrings, sigma0_sq)
    omega = ring_weights(nrings) * 2.0 * math.pi / nphi
    xi = pixel_normals(nrings, nphi, nmaps, seed, stream, first_map)
    return ((sig / np.sqrt(omega))[None, :, None] * xi).astype(np.float32)


def standard_normals(shape, seed: int, stream: int = STREAM_MISC) -> np.ndarray:
    """Standard normal draws of the given shape, float64."""
    return _rng(seed, stream).standard_normal(shape)


def field_variance(cl: np.ndarray) -> float:
    """<G^2> = sum_l (2l+1) C_l / (4 pi) of a Gaussian field with power C_l (the constant
    subtracted in the non-Gaussian maps T = G + f (G^2 - <G^2>))."""
    l = np.arange(np.asarray(cl).size)
    return float(np.sum((2 * l + 1) * np.asarray(cl)) / (4.0 * math.pi))
