"""Writes tiny_l32_p6_seed0.txt: the small workload's result as the FP64 oracle gives it.

Workload: l_max = 32, Gauss-Legendre grid 33 x 128, P = 6 shifted-Legendre modes
(n_max = 56), C_l = 1/(l(l+1)) for l >= 2, one map of Gaussian a_lm from seed 0, no mask,
no noise.  Stored: beta_n of the map (Eq. bbispect on the grid, no linear term), alpha_n
of the local shape, and the local-shape estimate fNL with its sigma (Eq. modalest,
Eq. modalvariance), taking zeta from the full-sky closed form (one map cannot estimate it).

This calls only oracle/ and simgen/; the file is a regression fixture for the oracle (a
change to its arithmetic shows up here), not an independent pin: the pins are in
tests/test_oracle_*.py.  Run from the repository root:  python tests/golden/make_tiny.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import simgen  # noqa: E402
from oracle import modal as om, sht as osh  # noqa: E402

NAME = "tiny_l32_p6_seed0.txt"


def compute():
    cfg = simgen.config("tiny")
    L, R, nphi, P = cfg["lmax"], cfg["nrings"], cfg["nphi"], cfg["P"]
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    filt = osh.filter_table(basis, cl)
    alm = simgen.gaussian_alm(cl, 1, seed=cfg["seed"])[0]
    mu, w = osh.gl_nodes(R)
    maps = osh.synthesize(alm, L, filt, mu, nphi)
    beta = om.cubic_beta(maps, om.pixel_weights(w, nphi))
    alpha = om.alpha_local(filt, cl)
    zeta = om.zeta_closed_form(filt, cl)
    fnl, sigma = om.solve_fnl(zeta, alpha, beta[None, :])
    return beta, alpha, float(np.ravel(fnl)[0]), float(sigma)


def write(path):
    beta, alpha, fnl, sigma = compute()
    P = simgen.config("tiny")["P"]
    with open(path, "w") as f:
        f.write("# l_max=32 grid 33x128 P=6 C_l=1/(l(l+1)) seed=0; written by tests/golden/make_tiny.py (oracle)\n")
        f.write("# fnl sigma\n%.17e %.17e\n" % (fnl, sigma))
        f.write("# n p r s beta_n alpha_n\n")
        for n, (p, r, s) in enumerate(om.mode_list(P)):
            f.write("%d %d %d %d %.17e %.17e\n" % (n, p, r, s, beta[n], alpha[n]))


def read(path):
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    fnl, sigma = float(rows[0][0]), float(rows[0][1])
    body = np.array([[float(x) for x in r] for r in rows[1:]])
    return body[:, 4], body[:, 5], fnl, sigma, body[:, 1:4].astype(int)


if __name__ == "__main__":
    write(os.path.join(HERE, NAME))
