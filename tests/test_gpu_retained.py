"""The adjoint and the coefficients from the maps kept by a preceding call
(modal_backward_retained, modal_cubic_retained).

They run the same kernels on the same maps as modal_backward and modal_cubic, so the
results must agree bit for bit; they are also checked against the oracle's adjoint_grad (<= 1e-5 relative,
as for modal_backward).  The state checks cover every call that reuses the map workspace.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import simgen
from oracle import modal as om, sht as osh

pytestmark = pytest.mark.gpu


def _cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    return M


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec", ["fp32", "fp16x3", "3xtf32"])
@pytest.mark.parametrize("mode", ["pixel", "ring"])
def test_backward_retained_matches_backward_and_oracle(prec, mode):
    M = _cuda_or_skip()
    L, P, R, nphi, nb = 24, 6, 25, 64, 3
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    mask = simgen.band_mask(R, 20.0)
    try:
        plan = M.Plan(L, P, basis, cl, R, nphi, prec=prec, ring_mask=mask)
    except M.ModalError as e:
        if "not supported" in str(e):
            pytest.skip("precision %s not built" % prec)
        raise
    if mode == "ring":
        plan.set_linear_mode("ring")
    plan.set_retain_maps(True)
    sims = simgen.gaussian_alm(cl, 6, seed=61, stream=simgen.STREAM_LINEAR).astype(np.complex64)
    plan.linear_term(torch.from_numpy(sims).cuda(), finalize=True)
    alm = simgen.gaussian_alm(cl, nb, seed=62).astype(np.complex64)
    a = torch.from_numpy(alm).cuda()
    g = torch.from_numpy(np.random.default_rng(63).standard_normal((nb, plan.n_max))).cuda()
    plan.cubic(a, use_linear=True)
    kept = plan.backward_retained(a, g, use_linear=True)
    again = plan.backward(a, g, use_linear=True)
    plan.sync()
    assert torch.equal(kept, again)
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    pm = om.pair_means([osh.synthesize(s.astype(np.complex128), L, filt, mu, nphi) for s in sims])
    if mode == "ring":
        pm = om.ring_pair_means(pm)
    got = kept.cpu().numpy()
    gn = g.cpu().numpy()
    for b in range(nb):
        ref = om.adjoint_grad(alm[b].astype(np.complex128), gn[b], L, filt, mu, w, nphi, mask, pm)
        err = _rel(got[b], ref)
        print("retained adjoint %s %s map %d: rel err %.3g" % (prec, mode, b, err))
        assert err <= 1e-5
    plan.close()


def test_backward_retained_needs_the_cubic_calls_maps():
    M = _cuda_or_skip()
    L, P, R, nphi = 16, 3, 17, 64
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    plan = M.Plan(L, P, basis, cl, R, nphi, prec="fp32")
    a = torch.from_numpy(simgen.gaussian_alm(cl, 2, seed=71).astype(np.complex64)).cuda()
    g = torch.ones((2, plan.n_max), dtype=torch.float64, device="cuda")

    def refused(x, gg):
        with pytest.raises(M.ModalError) as ei:
            plan.backward_retained(x, gg)
        assert ei.value.status == M.MODAL_ESTATE

    plan.cubic(a)
    refused(a, g)                                    # retention off
    plan.set_retain_maps(True)
    plan.cubic(a)
    refused(a[:1], g[:1])                            # another batch size
    refused(a.clone(), g)                            # another a_lm buffer
    plan.linear_term(a.clone())                      # linear-term synthesis of another buffer
    refused(a, g)
    plan.cubic(a)
    plan.quartic(a)                                  # so does the trispectrum
    refused(a, g)
    plan.cubic(a)
    plan.backward(a, g)                              # and the adjoint
    refused(a, g)
    plan.cubic(a)
    plan.set_chunk(2)                                # new workspace
    refused(a, g)
    plan.cubic(a)
    plan.set_retain_maps(False)
    refused(a, g)
    plan.set_retain_maps(True)
    plan.set_chunk(1)
    plan.cubic(a)                                    # two maps in two chunks: nothing kept
    refused(a, g)
    plan.set_chunk(4)
    plan.cubic(a)
    ref = plan.backward(a, g)
    plan.cubic(a)
    plan.cubic(a[:0])                                # an empty batch leaves the kept maps alone
    assert plan.backward_retained(a[:0], g[:0]).shape == (0, plan.n_alm)
    got = plan.backward_retained(a, g)
    assert torch.equal(got, ref)
    refused(a, g)                                    # the adjoint consumed the kept maps
    plan.sync()
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
@pytest.mark.parametrize("mode", ["pixel", "ring"])
def test_cubic_retained_from_the_linear_term_maps(prec, mode):
    """A batch that is both a linear-term sample and a coefficient input: linear_term(a) keeps
    its maps, cubic_retained(a) gives cubic(a) bit for bit (and, in ring mode, reads the m = 0
    Legendre sums left beside them), and backward_retained after it gives backward."""
    M = _cuda_or_skip()
    L, P, R, nphi, nb = 24, 6, 25, 64, 3
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    plan = M.Plan(L, P, basis, cl, R, nphi, prec=prec, ring_mask=simgen.band_mask(R, 20.0))
    if mode == "ring":
        plan.set_linear_mode("ring")
    plan.set_retain_maps(True)
    sims = simgen.gaussian_alm(cl, 6, seed=81, stream=simgen.STREAM_LINEAR).astype(np.complex64)
    plan.linear_term(torch.from_numpy(sims).cuda(), finalize=True)
    a = torch.from_numpy(simgen.gaussian_alm(cl, nb, seed=82).astype(np.complex64)).cuda()
    g = torch.from_numpy(np.random.default_rng(83).standard_normal((nb, plan.n_max))).cuda()
    plan.linear_term(a)                              # accumulate only: the mean in use is unchanged
    kept = plan.cubic_retained(a, use_linear=True)
    kept_plain = plan.cubic_retained(a)              # the maps stay kept
    grad_kept = plan.backward_retained(a, g, use_linear=True)
    again = plan.cubic(a, use_linear=True)
    assert torch.equal(kept, again)
    assert torch.equal(kept_plain, plan.cubic(a))
    assert torch.equal(grad_kept, plan.backward(a, g, use_linear=True))
    plan.sync()
    plan.close()


def test_cubic_retained_needs_kept_maps():
    M = _cuda_or_skip()
    L, P, R, nphi = 16, 3, 17, 64
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    plan = M.Plan(L, P, basis, cl, R, nphi, prec="fp32")
    a = torch.from_numpy(simgen.gaussian_alm(cl, 2, seed=91).astype(np.complex64)).cuda()

    def refused(x):
        with pytest.raises(M.ModalError) as ei:
            plan.cubic_retained(x)
        assert ei.value.status == M.MODAL_ESTATE

    plan.linear_term(a)
    refused(a)                                       # retention off
    plan.set_retain_maps(True)
    plan.linear_term(a)
    refused(a[:1])                                   # another batch size
    refused(a.clone())                               # another a_lm buffer
    ref = plan.cubic(a)
    assert torch.equal(plan.cubic_retained(a), ref)  # kept by the cubic call itself
    plan.backward(a, torch.ones((2, plan.n_max), dtype=torch.float64, device="cuda"))
    refused(a)                                       # the adjoint overwrote the maps
    plan.linear_term(a)
    plan.set_chunk(1)                                # two maps in two chunks: nothing kept
    plan.linear_term(a)
    refused(a)
    assert plan.cubic_retained(a[:0]).shape == (0, plan.n_max)
    plan.sync()
    plan.close()
