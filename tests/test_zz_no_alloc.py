"""modal_cubic_static, the allocation-free cubic reduction, against modal_cubic.

Callers that cannot call cudaMalloc (their device memory belongs to another allocator,
or an allocation's implicit synchronisation is not allowed in their loop) use
modal_cubic_static, which keeps its scratch in a static device array.  These tests call
it through the C ABI on maps made by modal_synthesize and compare with modal_cubic
(no linear term): two identical calls in a row, then calls of different sizes one after
the other (a 16-mode call over several blocks with a partial last block, then a 6-mode
call with fewer maps and blocks), so that scratch contents left by an earlier call
cannot leak into a later one.  They live in a file of their own, collected last.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import simgen

pytestmark = pytest.mark.gpu


def _weights(plan, nphi):
    mu, w = plan.rings()
    return torch.from_numpy(np.repeat((w * 2 * math.pi / nphi)[:, None], nphi, axis=1).astype(np.float32)).cuda()


def _case(M, L, P, R, nphi, nb, seed):
    basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
    alm = torch.from_numpy(simgen.gaussian_alm(cl, nb, seed=seed).astype(np.complex64)).cuda()
    plan = M.Plan(L, P, basis, cl, R, nphi, prec="fp32")
    ref = plan.cubic(alm).cpu().numpy()
    maps = plan.synthesize(alm)
    return plan, ref, maps, _weights(plan, nphi)


def _check(M, maps, W, npix, P, nb, n_max, ref, what):
    beta = torch.full((nb, n_max), float("nan"), dtype=torch.float64, device="cuda")
    M.modal_cubic_static(maps, W, npix, P, nb, beta)
    torch.cuda.synchronize()
    got = beta.cpu().numpy()
    for b in range(nb):
        err = np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b])
        assert err <= 1e-5, (what, b, err)
    return beta


def test_static_cubic_matches_modal_cubic_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    L, P, R, nphi, nb = 70, 16, 71, 256, 3
    plan, ref, maps, W = _case(M, L, P, R, nphi, nb, 901)
    for call in range(2):
        beta = _check(M, maps, W, R * nphi, P, nb, plan.n_max, ref, "call %d" % call)
    # beyond the static scratch (B * n_max > 4 Mi doubles) the library refuses before any
    # launch; called on the C ABI directly, since the Python wrapper would already refuse
    # these undersized tensors
    lib = M.binding.load_library()
    st = lib.modal_cubic_static(maps.data_ptr(), W.data_ptr(), R * nphi, P, 6000, beta.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == M.MODAL_EINVAL
    plan.close()


def test_static_cubic_several_blocks_then_a_smaller_call():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    # 203 x 512 pixels: six blocks of 17344 pixels, the last one partial
    big, ref16, maps16, W16 = _case(M, 200, 16, 203, 512, 3, 902)
    small, ref6, maps6, W6 = _case(M, 40, 6, 41, 128, 2, 903)
    _check(M, maps16, W16, 203 * 512, 16, 3, big.n_max, ref16, "P=16, 6 blocks")
    _check(M, maps6, W6, 41 * 128, 6, 2, small.n_max, ref6, "P=6 after P=16")
    _check(M, maps16, W16, 203 * 512, 16, 3, big.n_max, ref16, "P=16 again")
    # the wrapper refuses tensors the call would overrun or misread
    with pytest.raises(ValueError):
        M.modal_cubic_static(maps6.double(), W6, 41 * 128, 6, 2, torch.empty((2, 56), dtype=torch.float64,
                                                                           device="cuda"))
    with pytest.raises(ValueError):
        M.modal_cubic_static(maps6, W6[:-1], 41 * 128, 6, 2, torch.empty((2, 56), dtype=torch.float64,
                                                                       device="cuda"))
    with pytest.raises(ValueError):
        M.modal_cubic_static(maps6, W6, 41 * 128, 6, 2, torch.empty((1, 56), dtype=torch.float64, device="cuda"))
    big.close()
    small.close()
