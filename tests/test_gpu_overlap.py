"""The one overlap the library allows on a plan: the FP64 solve on a second stream beside
the adjoint of the same plan (the order the timed step uses).

The solve reads only the covariance sums and writes only its own workspace and error
word, so the overlapped results must equal the serial ones bit for bit, and a device
error of the data path (a bounded wait that gives up) must stay with the data path: the
solve beside it succeeds, and modal_sync on the data path's stream reports the timeout.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import simgen

pytestmark = pytest.mark.gpu


def _setup(M, prec):
    L, P, R, nphi, nb = 64, 6, 65, 256, 4
    cl = simgen.cl_model(L)
    plan = M.Plan(L, P, simgen.shifted_legendre_basis(L, P), cl, R, nphi, prec=prec)
    sims = torch.from_numpy(simgen.gaussian_alm(cl, 8, seed=301).astype(np.complex64)).cuda()
    plan.linear_term(sims, finalize=True)
    a = torch.from_numpy(simgen.gaussian_alm(cl, nb, seed=302).astype(np.complex64)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(7)
    plan.cov_accumulate(torch.randn((2 * plan.n_max, plan.n_max), generator=gen, device="cuda",
                                    dtype=torch.float64))
    alpha = plan.alpha_local()
    beta = plan.cubic(a, use_linear=True)
    g = torch.randn((nb, plan.n_max), generator=gen, device="cuda", dtype=torch.float64)
    torch.cuda.synchronize()
    return plan, a, alpha, beta, g


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_solve_beside_backward_equals_serial(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    plan, a, alpha, beta, g = _setup(M, prec)
    fnl_s, sig_s = plan.solve(alpha, beta)
    grad_s = plan.backward(a, g, use_linear=True)
    plan.sync()
    side = torch.cuda.Stream()
    for _ in range(3):
        grad = torch.empty_like(grad_s)
        ready = torch.cuda.Event()
        ready.record(torch.cuda.current_stream())
        plan.backward(a, g, use_linear=True, out=grad)
        side.wait_event(ready)
        fnl, sig = M.modal_solve(plan.h, alpha, beta, beta.shape[0], stream=side)
        plan.sync()
        assert np.array_equal(fnl, fnl_s) and sig == sig_s
        assert torch.equal(grad, grad_s)
    plan.close()


def test_data_path_error_stays_with_the_data_path():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    plan, a, alpha, beta, g = _setup(M, "fp16x3")
    fnl_s, sig_s = plan.solve(alpha, beta)
    side = torch.cuda.Stream()
    ready = torch.cuda.Event()
    ready.record(torch.cuda.current_stream())
    M.modal_selftest_wait(plan.h, 1000)              # sets the data path's timeout word
    side.wait_event(ready)
    fnl, sig = M.modal_solve(plan.h, alpha, beta, beta.shape[0], stream=side)
    assert np.array_equal(fnl, fnl_s) and sig == sig_s
    with pytest.raises(M.ModalError) as ei:
        plan.sync()
    assert ei.value.status == M.MODAL_ETIMEOUT
    plan.sync()
    # and a solve error stays with the solve: a rank-deficient covariance
    plan.reset()
    plan.cov_accumulate(beta[:1])
    plan.cov_accumulate(beta[:1])
    with pytest.raises(M.ModalError) as ei:
        plan.solve(alpha, beta)
    assert ei.value.status == M.MODAL_ENOTPD
    plan.sync()
    plan.close()
