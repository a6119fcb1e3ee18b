"""d fNL / d a_lm (Eq. modalest through the adjoint of Eq. bbispect): modal_fnl_weights and the
ModalFnl autograd Function against the FP64 oracle and central differences.

fNL = alpha^T zeta^-1 beta / alpha^T zeta^-1 alpha is linear in beta, so d fNL / d a_lm is the
adjoint of sum_n w_n beta_n with w = zeta^-1 alpha / (alpha^T zeta^-1 alpha).

  weights   each side forms zeta from its own beta of the same simulations and then w; w
            depends on zeta through zeta^-1, so its relative error is bounded by perturbation
            theory: ||dw|| / ||w|| <= 2 kappa(zeta) ||d zeta|| / ||zeta|| (first order; the
            factor 2 covers the normalisation), with ||d zeta|| / ||zeta|| <= 1e-5.  Checked
            at 10 modes, where kappa(zeta) ~ 6e3 (the unnormalised shifted-Legendre modes make
            kappa ~ 1e10 at 56 modes, beyond any FP32 beta).
  adjoint   the library's gradient for the oracle's w of the full-sky covariance at
            l_max = 64, 10 modes, linear term on: ||d grad|| / ||grad|| <= 1e-5.  (At 56
            modes w has entries of both signs up to kappa times larger than the result, so
            the gradient is a difference of large FP32 sums; the same holds for the central
            differences below, which therefore also run at 10 modes.)
  chain     ModalFnl's backward against central differences of its forward in 32 random
            coefficients (step 10 sigma_lm; fNL is cubic in a_lm through beta):
            max |grad - cd| <= 1e-3 max |cd|; and equal to modal_backward with g = w.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import simgen
from oracle import modal as om, sht as osh

pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    return M


def _plan(M, L, P, basis, cl, R, nphi, prec):
    try:
        return M.Plan(L, P, basis, cl, R, nphi, prec=prec)
    except M.ModalError as e:
        if prec != "fp32" and "not supported" in str(e):
            pytest.skip("precision %s not built" % prec)
        raise


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_fnl_weights_against_oracle(prec):
    M = _lib()
    L, P, R, nphi, n_lin, n_cov = 48, 3, 49, 128, 8, 200
    cl = simgen.cl_model(L)
    basis = simgen.shifted_legendre_basis(L, P)
    sims = simgen.gaussian_alm(cl, n_lin, seed=61, stream=simgen.STREAM_LINEAR)
    cov = simgen.gaussian_alm(cl, n_cov, seed=62, stream=simgen.STREAM_COV)
    plan = _plan(M, L, P, basis, cl, R, nphi, prec)
    plan.linear_term(torch.from_numpy(sims.astype(np.complex64)).cuda(), finalize=True)
    plan.cov_accumulate(plan.cubic(torch.from_numpy(cov.astype(np.complex64)).cuda(), use_linear=True))
    alpha = plan.alpha_local()
    w_gpu, sigma_gpu = plan.fnl_weights(alpha)
    w_gpu = w_gpu.cpu().numpy()
    zeta_gpu = plan.zeta()
    plan.sync()
    plan.close()
    filt = osh.filter_table(basis, cl)
    mu, w = osh.gl_nodes(R)
    W = om.pixel_weights(w, nphi)
    pm = om.pair_means(list(osh.synthesize_many(sims, L, filt, mu, nphi)))
    betas = np.array([om.cubic_beta(m, W, pm) for m in osh.synthesize_many(cov, L, filt, mu, nphi)])
    zeta = om.covariance_zeta(betas)
    alpha_o = om.alpha_local(filt, cl)
    w_orc = om.fnl_weights(zeta, alpha_o)
    _, sigma_orc = om.solve_fnl(zeta, alpha_o, betas[:1])
    e_zeta = np.linalg.norm(zeta_gpu - zeta) / np.linalg.norm(zeta)
    kappa = np.linalg.cond(zeta)
    e_w = _rel(w_gpu, w_orc)
    print("fnl weights %s: zeta %.3g, kappa %.3g, w %.3g (bound %.3g), sigma %.3g"
          % (prec, e_zeta, kappa, e_w, 2 * kappa * e_zeta, abs(sigma_gpu - sigma_orc) / sigma_orc))
    assert e_zeta <= 1e-5
    assert e_w <= 2 * kappa * e_zeta + 1e-12
    assert abs(sigma_gpu - sigma_orc) <= 1e-5 * sigma_orc


@pytest.mark.parametrize("prec", ["fp32", "fp16x3", "3xtf32"])
def test_fnl_gradient_adjoint_against_oracle(prec):
    """The adjoint with the oracle's w of the full-sky covariance (the ideal-covariance
    estimator's d fNL / d beta) as g, linear term on."""
    M = _lib()
    L, P, R, nphi = 64, 3, 65, 256
    cl = simgen.cl_model(L)
    basis = simgen.shifted_legendre_basis(L, P)
    filt = osh.filter_table(basis, cl)
    g = om.fnl_weights(om.zeta_closed_form(filt, cl), om.alpha_local(filt, cl))
    sims = simgen.gaussian_alm(cl, 4, seed=63, stream=simgen.STREAM_LINEAR)
    a = simgen.gaussian_alm(cl, 2, seed=64)
    plan = _plan(M, L, P, basis, cl, R, nphi, prec)
    plan.linear_term(torch.from_numpy(sims.astype(np.complex64)).cuda(), finalize=True)
    grad = plan.backward(torch.from_numpy(a.astype(np.complex64)).cuda(),
                         torch.from_numpy(np.tile(g, (2, 1))).cuda(), use_linear=True).cpu().numpy()
    plan.sync()
    plan.close()
    mu, w = osh.gl_nodes(R)
    pm = om.pair_means(list(osh.synthesize_many(sims.astype(np.complex64).astype(np.complex128), L, filt, mu, nphi)))
    for b in range(2):
        ref = om.adjoint_grad(a[b].astype(np.complex64).astype(np.complex128), g, L, filt, mu, w, nphi, pairmean=pm)
        err = _rel(grad[b], ref)
        print("d fNL / d a_lm %s map %d: rel err %.3g" % (prec, b, err))
        assert err <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_fnl_autograd_against_central_differences(prec):
    M = _lib()
    L, P, R, nphi = 64, 3, 65, 256
    cl = simgen.cl_model(L)
    plan = _plan(M, L, P, simgen.shifted_legendre_basis(L, P), cl, R, nphi, prec)
    plan.linear_term(torch.from_numpy(simgen.gaussian_alm(cl, 8, seed=65, stream=simgen.STREAM_LINEAR)
                                      .astype(np.complex64)).cuda(), finalize=True)
    cov = torch.from_numpy(simgen.gaussian_alm(cl, 400, seed=66, stream=simgen.STREAM_COV).astype(np.complex64)).cuda()
    plan.cov_accumulate(plan.cubic(cov, use_linear=True))
    alpha = plan.alpha_local()
    a = torch.from_numpy(simgen.gaussian_alm(cl, 2, seed=67).astype(np.complex64)).cuda().requires_grad_(True)
    fnl = M.modal_fnl(a, plan, alpha)
    fnl.sum().backward()
    grad = a.grad.detach()
    # the same as the adjoint with g = w
    w, _ = plan.fnl_weights(alpha)
    direct = plan.backward(a.detach().contiguous(), torch.stack([w, w]).contiguous(), use_linear=True)
    assert torch.equal(grad, direct)
    # central differences of fNL of map 0 in 32 real parts (l >= 2)
    l_of, m_of = simgen.lm_arrays(L)
    cand = np.nonzero(l_of >= 2)[0]
    idx = cand[simgen.random_subset(len(cand), 32, seed=68)]
    h = 10.0 * np.sqrt(cl[l_of[idx]] / np.where(m_of[idx] > 0, 2.0, 1.0))
    pert = a.detach()[0:1].repeat(2 * len(idx), 1).clone()
    ii = torch.from_numpy(np.concatenate([idx, idx])).cuda()
    hh = torch.from_numpy(np.concatenate([h, -h]).astype(np.float32)).cuda().to(torch.complex64)
    pert[torch.arange(2 * len(idx), device="cuda"), ii] += hh
    f, _ = plan.solve(alpha, plan.cubic(pert.contiguous(), use_linear=True))
    cd = (f[:len(idx)] - f[len(idx):]) / (2.0 * h)
    gsel = grad[0, torch.from_numpy(idx).cuda()].real.double().cpu().numpy()
    plan.sync()
    plan.close()
    err = np.max(np.abs(gsel - cd)) / np.max(np.abs(cd))
    print("ModalFnl %s: max |grad - central difference| / max |cd| = %.3g" % (prec, err))
    assert err <= 1e-3
