"""GPU trispectrum modes (Sec. IV) through the C ABI against the oracle's quartic_tau.

Tolerance: ||tau_gpu - tau_oracle||_2 / ||tau_oracle||_2 <= 1e-5 per map, the same
metric as beta (FP32 products, FP64 sums).  Each side synthesises its own maps from the
same a_lm; the Monte Carlo means come from the same simulation a_lm on both sides.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import simgen
from oracle import modal as om, sht as osh

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "fp16x3"]


def _cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    return M


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


CASES = [
    # (lmax, P, nrings, nphi, nmaps, chunk)
    (24, 3, 25, 64, 2, None),        # 15 modes, 4-mode template
    (40, 6, 41, 128, 2, None),       # 126 modes, 8-mode template
    (36, 9, 40, 128, 3, 2),          # 16-mode template with padding pairs, chunk boundary, no equator
    (40, 16, 41, 128, 2, None),      # 3876 modes, every register tile
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L,P,R,nphi,nb,chunk", CASES)
def test_quartic_parity(prec, L, P, R, nphi, nb, chunk):
    M = _cuda_or_skip()
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    alm = simgen.gaussian_alm(cl, nb, seed=300 + L + P).astype(np.complex64)
    plan = M.Plan(L, P, basis, cl, R, nphi, prec=prec)
    if chunk:
        plan.set_chunk(chunk)
    assert plan.n_quad == om.n_quads(P)
    tau = plan.quartic(torch.from_numpy(alm).cuda()).cpu().numpy()
    plan.sync()
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    W = om.pixel_weights(w, nphi)
    for b in range(nb):
        ref = om.quartic_tau(osh.synthesize(alm[b].astype(np.complex128), L, filt, mu, nphi), W)
        err = _rel(tau[b], ref)
        print("quartic lmax=%d P=%d %s map %d: rel err %.3g" % (L, P, prec, b, err))
        assert err <= 1e-5
    plan.close()


@pytest.mark.parametrize("mode", ["pixel", "ring"])
@pytest.mark.parametrize("P", [4, 16])
def test_quartic_with_monte_carlo_terms(mode, P):
    """Band-masked sky: the single-pair and two-pair terms with the plan's own means (per
    pixel, or per ring) against the oracle with the means of the same simulations."""
    M = _cuda_or_skip()
    L, R, nphi, n_lin, nb = 30, 31, 64, 12, 2
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    mask = simgen.band_mask(R, 20.0)
    plan = M.Plan(L, P, basis, cl, R, nphi, prec="fp32", ring_mask=mask)
    if mode == "ring":
        plan.set_linear_mode("ring")
    sims = simgen.gaussian_alm(cl, n_lin, seed=31, stream=simgen.STREAM_LINEAR).astype(np.complex64)
    plan.linear_term(torch.from_numpy(sims[:5]).cuda())
    plan.linear_term(torch.from_numpy(sims[5:]).cuda(), finalize=True)
    alm = simgen.gaussian_alm(cl, nb, seed=32).astype(np.complex64)
    a = torch.from_numpy(alm).cuda()
    tau = plan.quartic(a, use_linear=True).cpu().numpy()
    tau0 = plan.quartic(a).cpu().numpy()
    plan.sync()
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    W = om.pixel_weights(w, nphi, mask)
    pm = om.pair_means([osh.synthesize(s.astype(np.complex128), L, filt, mu, nphi) for s in sims])
    if mode == "ring":
        pm = om.ring_pair_means(pm)
    for b in range(nb):
        maps = osh.synthesize(alm[b].astype(np.complex128), L, filt, mu, nphi)
        ref = om.quartic_tau(maps, W, pm)
        ref0 = om.quartic_tau(maps, W)
        err, err0 = _rel(tau[b], ref), _rel(tau0[b], ref0)
        print("quartic MC terms %s P=%d map %d: rel err %.3g (quartic sum alone %.3g)" % (mode, P, b, err, err0))
        assert err <= 1e-5 and err0 <= 1e-5
    plan.close()


def test_quartic_errors_and_empty_batch():
    M = _cuda_or_skip()
    L, P = 20, 2
    plan = M.Plan(L, P, simgen.shifted_legendre_basis(L, P), simgen.cl_model(L), 21, 64)
    a = torch.zeros((1, plan.n_alm), dtype=torch.complex64, device="cuda")
    with pytest.raises(M.ModalError) as ei:
        plan.quartic(a, use_linear=True)
    assert ei.value.status == M.MODAL_ESTATE
    out = plan.quartic(a[:0])
    assert out.shape == (0, plan.n_quad)
    np.testing.assert_array_equal(plan.quartic(a).cpu().numpy(), 0.0)
    plan.close()


def test_quartic_full_size_l2000_sampled_rings():
    """l_max = 2000, 2001 x 4096, 16 modes (3876 quartic modes), per-ring means from four
    simulations: the ring mask restricts every pixel sum to five rings from the pole to
    the equator, where the oracle can synthesise the maps."""
    M = _cuda_or_skip()
    L, P, R, nphi = 2000, 16, 2001, 4096
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    rings = np.array([0, 3, 517, 1000, 1998])
    mask = np.zeros(R)
    mask[rings] = 1.0
    plan = M.Plan(L, P, basis, cl, R, nphi, prec="fp16x3", ring_mask=mask)
    plan.set_linear_mode("ring")
    sims = simgen.gaussian_alm(cl, 4, seed=2001, stream=simgen.STREAM_LINEAR).astype(np.complex64)
    plan.linear_term(torch.from_numpy(sims).cuda(), finalize=True)
    alm = simgen.gaussian_alm(cl, 1, seed=2002).astype(np.complex64)
    tau = plan.quartic(torch.from_numpy(alm).cuda(), use_linear=True).cpu().numpy()
    plan.sync()
    plan.close()
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    W = om.pixel_weights(w[rings], nphi)
    pm = om.ring_pair_means(om.pair_means([osh.synthesize(s.astype(np.complex128), L, filt, mu[rings], nphi)
                                           for s in sims]))
    ref = om.quartic_tau(osh.synthesize(alm[0].astype(np.complex128), L, filt, mu[rings], nphi), W, pm)
    err = _rel(tau[0], ref)
    print("quartic lmax=2000 sampled rings: rel err %.3g" % err)
    assert err <= 1e-5
