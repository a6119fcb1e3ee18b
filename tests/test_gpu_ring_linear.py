"""Ring-only linear term (modal_set_linear_mode "ring"): beta, gradient and pair means
against the oracle with the longitude-averaged Monte Carlo means, on an axisymmetric
(band-masked) sky."""
import os

import numpy as np
import pytest
import torch

import simgen
from oracle import modal as om, sht as osh

pytestmark = pytest.mark.gpu

PRECS = [p for p in os.environ.get("MODAL_TEST_PRECS", "fp32,fp16x3,3xtf32").split(",") if p]


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _plan(M, L, P, basis, cl, R, nphi, prec, **kw):
    try:
        return M.Plan(L, P, basis, cl, R, nphi, prec=prec, **kw)
    except M.ModalError as e:
        if prec != "fp32" and "not supported" in str(e):
            pytest.skip("precision %s not built" % prec)
        raise


@pytest.mark.parametrize("prec", PRECS)
def test_ring_linear_term_beta_gradient_and_means(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    L, P, R, nphi = 40, 16, 41, 128
    basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
    mask = simgen.band_mask(R, 20.0)
    plan = _plan(M, L, P, basis, cl, R, nphi, prec, ring_mask=mask)
    plan.set_linear_mode("ring")
    sims = simgen.gaussian_alm(cl, 6, seed=61, stream=simgen.STREAM_LINEAR).astype(np.complex64)
    plan.linear_term(torch.from_numpy(sims[:4]).cuda())
    plan.linear_term(torch.from_numpy(sims[4:]).cuda(), finalize=True)
    alm = simgen.gaussian_alm(cl, 3, seed=62).astype(np.complex64)
    a = torch.from_numpy(alm).cuda()
    beta = plan.cubic(a, use_linear=True).cpu().numpy()
    g = np.random.default_rng(63).standard_normal((3, plan.n_max))
    grad = plan.backward(a, torch.from_numpy(g).cuda(), use_linear=True).cpu().numpy()
    pm_gpu = plan.pair_mean().cpu().numpy()
    plan.sync()
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    W = om.pixel_weights(w, nphi, mask)
    ring = om.ring_pair_means(om.pair_means([osh.synthesize(s.astype(np.complex128), L, filt, mu, nphi)
                                             for s in sims]))
    assert pm_gpu.shape == (plan.n_pair, R)
    assert _rel(pm_gpu, ring[:, :, 0]) <= 1e-5
    for b in range(3):
        maps = osh.synthesize(alm[b].astype(np.complex128), L, filt, mu, nphi)
        eb = _rel(beta[b], om.cubic_beta(maps, W, ring))
        eg = _rel(grad[b], om.adjoint_grad(alm[b].astype(np.complex128), g[b], L, filt, mu, w, nphi, mask, ring))
        print("ring linear term lmax=%d P=%d %s map %d: beta %.3g grad %.3g" % (L, P, prec, b, eb, eg))
        assert eb <= 1e-5 and eg <= 1e-5
    plan.close()


def test_ring_mode_needs_axisymmetric_weights_and_checkpoints():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    L, P, R, nphi = 16, 3, 17, 64
    basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
    pix = np.ones(R * nphi)
    pix[5] = 0.0
    plan = M.Plan(L, P, basis, cl, R, nphi, pix_mask=pix)
    with pytest.raises(M.ModalError, match="EINVAL"):
        plan.set_linear_mode("ring")
    plan.close()
    plan = M.Plan(L, P, basis, cl, R, nphi)
    plan.set_linear_mode("ring")
    sims = torch.from_numpy(simgen.gaussian_alm(cl, 3, seed=64, stream=simgen.STREAM_LINEAR).astype(np.complex64)).cuda()
    plan.linear_term(sims, finalize=True)
    a = torch.from_numpy(simgen.gaussian_alm(cl, 2, seed=65).astype(np.complex64)).cuda()
    before = plan.cubic(a, use_linear=True).cpu()
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "state.bin")
        M.modal_save_state(plan.h, path)
        other = M.Plan(L, P, basis, cl, R, nphi)
        with pytest.raises(M.ModalError, match="EINVAL"):     # pixel-mode plan refuses ring sums
            M.modal_load_state(other.h, path)
        other.set_linear_mode("ring")
        M.modal_load_state(other.h, path)
        assert torch.equal(other.cubic(a, use_linear=True).cpu(), before)
        other.close()
    plan.close()
