"""Writes the full-size oracle fixtures: the FP64 oracle's results at the workload sizes the
GPU path is measured on, too slow to recompute inside a GPU test (tens of minutes on a
few host cores).  Every value here comes from oracle/ and simgen/ alone.

Targets (python tests/golden/make_fullsize.py <target> [--small]):

  beta_l2000   the l_max = 2000 workload on its full 2001 x 4096 Gauss-Legendre grid,
               16 modes (n_max = 816), C_l = 1/(l(l+1)), no mask: beta_n (Eq. bbispect)
               with and without the linear term of Eq. bispectrumest, the Monte Carlo
               pair means taken over 2 Gaussian simulations, for a Gaussian map G and for
               T = G + 50 (G^2 - <G^2>) (G synthesised on an exact-cubic 3001 x 8192 grid,
               T analysed back to l_max = 2000).  Sampled a_lm of T are stored so that a
               consumer building T with its own transforms can check its input first.
  grad_l1000   the adjoint workload: l_max = 1000 on 1001 x 2048, 12 modes (n_max = 364),
               signal plus anisotropic white noise sigma^2 = sigma0^2 (1 + 3 cos^2 theta),
               sigma0^2 = 0.1 C_1000, 20-degree band mask, filter with C_l + N_l; the
               gradient of sum_n g_n beta_n (linear term from 2 noisy simulations) with
               respect to (Re a_lm, Im a_lm) on the full grid, sampled at 4096 coefficients
               and projected on 4 seeded random directions, and beta_n itself.
  wmap_chain   the WMAP-resolution workload (l_max = 500, 501 x 1024, 10 modes, n_max = 220,
               noise and mask as above with sigma0^2 = 0.1 C_500): pair means over
               N_lin = 256 noisy simulations, beta_n with the linear term of N_cov = 1024
               noisy simulations, zeta = their covariance / 6 (Eq. linearterm), the local
               alpha (Eq. abispect), fNL and sigma (Eq. modalest, Eq. modalvariance) of 4
               data maps (2 Gaussian, 2 with f = 0.01 local non-Gaussianity), all sums on 8
               unmasked rings (a ring mask selects them on the GPU).
  chain_l2000  the same chain at 816 modes: l_max = 2000, 2001 x 4096, 16 modes, no mask,
               N_lin = 16, N_cov = 1024, 4 Gaussian data maps, sums on 8 rings.

--small shrinks every target (l_max / 10) to check the script itself quickly.
Run from the repository root.
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import simgen  # noqa: E402
from oracle import modal as om, sht as osh  # noqa: E402

FILES = {
    "beta_l2000": "fullsize_beta_l2000_p16.json",
    "grad_l1000": "fullsize_grad_l1000_p12.json",
    "wmap_chain": "chain_wmap_l500_p10.json",
    "chain_l2000": "chain_l2000_p16.json",
}
F_NG_L2000 = 50.0        # T = G + 50 (G^2 - <G^2>) (the precision-sweep maps)
F_NG_CHAIN = 0.01        # weakly non-Gaussian data maps of the WMAP chain


def _log(msg):
    print("[%s] %s" % (time.strftime("%H:%M:%S"), msg), flush=True)


def _cplx(a):
    a = np.asarray(a)
    return [[float(x) for x in a.real], [float(x) for x in a.imag]]


def exact_cubic_grid(L):
    """Rings and longitudes on which the sphere integral of a degree-3L product is exact."""
    R = (3 * L + 2 + 1) // 2
    nphi = 1 << int(math.ceil(math.log2(3 * L + 1)))
    return R, nphi


def nongaussian_alm(aG, cl, f):
    """a_lm of T = G + f (G^2 - <G^2>) with G synthesised and T analysed on an exact-cubic grid."""
    L = cl.size - 1
    R, nphi = exact_cubic_grid(L)
    mu, w = osh.gl_nodes(R)
    one = osh.filter_table(np.sqrt(cl)[None, :], cl)
    G = osh.synthesize_many(np.atleast_2d(aG), L, one, mu, nphi)[:, 0]
    T = G + f * (G * G - simgen.field_variance(cl))
    return osh.analyze_many(T, L, mu, w, nphi)


def noisy_alm(cl, n, seed, stream, sigma0_sq, R, nphi, mu, w, batch=64):
    """Signal a_lm (seeded Philox) plus the quadrature analysis of seeded pixel noise."""
    L = cl.size - 1
    out = simgen.gaussian_alm(cl, n, seed=seed, stream=stream)
    for b0 in range(0, n, batch):
        nb = min(batch, n - b0)
        nm = simgen.noise_maps(R, nphi, nb, seed=seed, sigma0_sq=sigma0_sq, first_map=b0).astype(np.float64)
        out[b0:b0 + nb] += osh.analyze_many(nm, L, mu, w, nphi)
    return out


def sample_rings(mask_rings, nsel):
    """nsel rings spread over the unmasked ones, north pole to equator."""
    ok = np.nonzero(np.asarray(mask_rings) > 0)[0]
    half = ok[ok <= (len(mask_rings) - 1) // 2]
    pick = np.unique(np.round(np.linspace(0, len(half) - 1, nsel)).astype(int))
    return half[pick]


# ---------------------------------------------------------------------------- targets
def beta_l2000(small=False):
    L, R, nphi, P = (200, 201, 512, 16) if small else (2000, 2001, 4096, 16)
    cl = simgen.cl_model(L)
    basis = simgen.shifted_legendre_basis(L, P)
    filt = osh.filter_table(basis, cl)
    mu, w = osh.gl_nodes(R)
    aG = simgen.gaussian_alm(cl, 1, seed=3)[0]
    sims = simgen.gaussian_alm(cl, 2, seed=4, stream=simgen.STREAM_LINEAR)
    _log("beta_l2000: T = G + f (G^2 - <G^2>) on the exact-cubic grid %s" % (exact_cubic_grid(L),))
    aT = nongaussian_alm(aG, cl, F_NG_L2000)[0]
    _log("beta_l2000: maps of G, T and the 2 simulations")
    maps = osh.synthesize_many(np.stack([aG, aT, sims[0], sims[1]]), L, filt, mu, nphi)
    W = om.pixel_weights(w, nphi)
    _log("beta_l2000: pair means")
    pm = om.pair_means([maps[2], maps[3]])
    out = {}
    for name, i in (("G", 0), ("T", 1)):
        _log("beta_l2000: beta of %s" % name)
        out["beta_%s" % name] = [float(x) for x in om.cubic_beta(maps[i], W)]
        out["beta_lin_%s" % name] = [float(x) for x in om.cubic_beta(maps[i], W, pm)]
    idx = simgen.random_subset(aT.size, 512, seed=2001)
    return dict(
        what="beta_n of G and T = G + %g (G^2 - <G^2>) with and without the linear term, full grid" % F_NG_L2000,
        lmax=L, nrings=R, nphi=nphi, P=P, n_max=om.n_modes(P), cl="1/(l(l+1)), l >= 2",
        data="simgen.gaussian_alm(cl, 1, seed=3)[0]", sims="simgen.gaussian_alm(cl, 2, seed=4, STREAM_LINEAR)",
        f_ng=F_NG_L2000, ng_grid=list(exact_cubic_grid(L)),
        aT_index=[int(i) for i in idx], aT_sample=_cplx(aT[idx]), aT_norm=float(np.linalg.norm(aT)),
        **out)


def grad_l1000(small=False):
    L, R, nphi, P = (100, 101, 256, 12) if small else (1000, 1001, 2048, 12)
    cl = simgen.cl_model(L)
    s0 = 0.1 * cl[L]
    cl_tot = cl + np.where(np.arange(L + 1) >= 2, 2.0 * s0, 0.0)
    basis = simgen.shifted_legendre_basis(L, P)
    filt = osh.filter_table(basis, cl_tot)
    mask = simgen.band_mask(R, 20.0)
    mu, w = osh.gl_nodes(R)
    _log("grad_l1000: noisy data map and 2 noisy simulations")
    a = noisy_alm(cl, 1, 102, simgen.STREAM_DATA, s0, R, nphi, mu, w)[0]
    sims = noisy_alm(cl, 2, 101, simgen.STREAM_LINEAR, s0, R, nphi, mu, w)
    smaps = osh.synthesize_many(sims, L, filt, mu, nphi)
    pm = om.pair_means([smaps[0], smaps[1]])
    del smaps
    n_max = om.n_modes(P)
    g = simgen.standard_normals(n_max, seed=103)
    _log("grad_l1000: beta and the adjoint gradient")
    maps = osh.synthesize(a, L, filt, mu, nphi)
    beta = om.cubic_beta(maps, om.pixel_weights(w, nphi, mask), pm)
    grad = om.adjoint_grad(a, g, L, filt, mu, w, nphi, mask=mask, pairmean=pm)
    idx = simgen.random_subset(grad.size, 4096, seed=104)
    r = simgen.standard_normals((4, grad.size, 2), seed=105)
    proj = [float(np.sum(grad.real * r[k, :, 0] + grad.imag * r[k, :, 1])) for k in range(4)]
    return dict(
        what="d(sum_n g_n beta_n)/d(Re a_lm, Im a_lm) on the full grid, noisy band-masked sky, linear term",
        lmax=L, nrings=R, nphi=nphi, P=P, n_max=n_max, sigma0_sq=s0, mask_deg=20.0,
        data="gaussian_alm(cl, 1, seed=102) + analysis of noise_maps(seed=102)",
        sims="gaussian_alm(cl, 2, seed=101, STREAM_LINEAR) + analysis of noise_maps(seed=101)",
        g="standard_normals(n_max, seed=103)", beta_lin=[float(x) for x in beta],
        grad_index=[int(i) for i in idx], grad_sample=_cplx(grad[idx]), grad_norm=float(np.linalg.norm(grad)),
        proj_seed=105, grad_proj=proj)


def _chain(L, R, nphi, P, s0, masked, n_lin, n_cov, data_ng, seeds, nrings_sel=8, batch=32):
    """pair means, covariance sims, zeta, alpha, data maps' beta, fNL and sigma on the
    selected rings (the oracle sums over them only)."""
    cl = simgen.cl_model(L)
    noise = s0 > 0
    cl_tot = cl + (np.where(np.arange(L + 1) >= 2, 2.0 * s0, 0.0) if noise else 0.0)
    basis = simgen.shifted_legendre_basis(L, P)
    filt = osh.filter_table(basis, cl_tot)
    mask = simgen.band_mask(R, 20.0) if masked else np.ones(R)
    mu, w = osh.gl_nodes(R)
    rings = sample_rings(mask, nrings_sel)
    W = om.pixel_weights(w[rings], nphi)

    def ring_maps(a):
        return osh.synthesize_many(a, L, filt, mu[rings], nphi)

    _log("chain lmax=%d: %d linear-term simulations" % (L, n_lin))
    lin_all = noisy_alm(cl, n_lin, seeds[0], simgen.STREAM_LINEAR, s0, R, nphi, mu, w) if noise else None
    acc, n = None, 0
    for b0 in range(0, n_lin, batch):
        nb = min(batch, n_lin - b0)
        a = lin_all[b0:b0 + nb] if noise else simgen.gaussian_alm(cl, nb, seed=seeds[0],
                                                                   stream=simgen.STREAM_LINEAR, first_map=b0)
        for mp in ring_maps(a):
            pp = om.pair_products(mp)
            acc = pp if acc is None else acc + pp
            n += 1
    pm = acc / n
    _log("chain lmax=%d: %d covariance simulations" % (L, n_cov))
    betas = []
    cov_all = noisy_alm(cl, n_cov, seeds[1], simgen.STREAM_COV, s0, R, nphi, mu, w) if noise else None
    for b0 in range(0, n_cov, batch):
        nb = min(batch, n_cov - b0)
        a = cov_all[b0:b0 + nb] if noise else simgen.gaussian_alm(cl, nb, seed=seeds[1], stream=simgen.STREAM_COV,
                                                                   first_map=b0)
        for mp in ring_maps(a):
            betas.append(om.cubic_beta(mp, W, pm))
    betas = np.array(betas)
    zeta = om.covariance_zeta(betas)
    alpha = om.alpha_local(filt, cl)
    _log("chain lmax=%d: data maps" % L)
    nd = 4
    if noise:
        data = noisy_alm(cl, nd, seeds[2], simgen.STREAM_DATA, s0, R, nphi, mu, w)
    else:
        data = simgen.gaussian_alm(cl, nd, seed=seeds[2], stream=simgen.STREAM_DATA)
    if data_ng:      # maps 2 and 3: signal S -> T = S + f (S^2 - <S^2>), noise unchanged
        aS = simgen.gaussian_alm(cl, nd, seed=seeds[2], stream=simgen.STREAM_DATA)[2:]
        data[2:] += nongaussian_alm(aS, cl, data_ng) - aS
    bd = np.array([om.cubic_beta(mp, W, pm) for mp in ring_maps(data)])
    fnl, sigma = om.solve_fnl(zeta, alpha, bd)
    iu = simgen.random_subset(zeta.size, 256, seed=seeds[0] + 7)
    return dict(lmax=L, nrings=R, nphi=nphi, P=P, n_max=om.n_modes(P), sigma0_sq=s0, masked=bool(masked),
                rings=[int(r) for r in rings], n_lin=n_lin, n_cov=n_cov, seeds=list(seeds), f_ng=data_ng,
                zeta_diag=[float(x) for x in np.diag(zeta)], zeta_fro=float(np.linalg.norm(zeta)),
                zeta_index=[int(i) for i in iu], zeta_sample=[float(x) for x in zeta.ravel()[iu]],
                alpha=[float(x) for x in alpha], beta_data=[[float(x) for x in b] for b in bd],
                beta_cov_mean=[float(x) for x in betas.mean(axis=0)],
                fnl=[float(x) for x in np.ravel(fnl)], sigma=float(sigma))


def wmap_chain(small=False):
    L, R, nphi, P = (50, 51, 128, 10) if small else (500, 501, 1024, 10)
    cl = simgen.cl_model(L)
    out = _chain(L, R, nphi, P, 0.1 * cl[L], True, 256, 1024, F_NG_CHAIN, (11, 12, 13))
    out["what"] = ("WMAP-resolution chain: pair means (256 noisy sims), zeta (1024 noisy sims), "
                   "alpha, fNL and sigma of 2 Gaussian and 2 f=%g maps, sums on the selected rings" % F_NG_CHAIN)
    return out


def chain_l2000(small=False):
    L, R, nphi, P = (200, 201, 512, 16) if small else (2000, 2001, 4096, 16)
    out = _chain(L, R, nphi, P, 0.0, False, 16, 1024, 0.0, (21, 22, 23))
    out["what"] = ("816-mode chain at l_max=2000: pair means (16 sims), zeta (1024 sims), alpha, fNL and "
                   "sigma of 4 Gaussian maps, sums on the selected rings")
    return out


TARGETS = {"beta_l2000": beta_l2000, "grad_l1000": grad_l1000, "wmap_chain": wmap_chain,
           "chain_l2000": chain_l2000}


def path(target, small=False):
    name = FILES[target]
    return os.path.join(HERE, name.replace(".json", "_small.json") if small else name)


def load(target, small=False):
    with open(path(target, small)) as f:
        return json.load(f)


if __name__ == "__main__":
    small = "--small" in sys.argv
    names = [a for a in sys.argv[1:] if not a.startswith("--")] or list(TARGETS)
    for nm in names:
        t0 = time.time()
        res = TARGETS[nm](small)
        res["written_by"] = "tests/golden/make_fullsize.py %s%s (oracle/ and simgen/ only)" % (
            nm, " --small" if small else "")
        res["seconds"] = round(time.time() - t0, 1)
        with open(path(nm, small), "w") as f:
            json.dump(res, f)
        _log("%s written in %.0f s" % (path(nm, small), time.time() - t0))
