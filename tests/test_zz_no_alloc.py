"""modal_cubic_static, the allocation-free cubic reduction, against modal_cubic.

Callers that cannot call cudaMalloc (their device memory belongs to another allocator,
or an allocation's implicit synchronisation is not allowed in their loop) use
modal_cubic_static, which keeps its scratch in a static device array.  This test calls
it through the C ABI on maps made by modal_synthesize and compares with modal_cubic
(no linear term) on two calls in a row, which also checks that leftover scratch
contents from the first call do not leak into the second.  It lives in its own file,
collected last.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import simgen

pytestmark = pytest.mark.gpu


def test_static_cubic_matches_modal_cubic_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    L, P, R, nphi, nb = 70, 16, 71, 256, 3
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    alm = torch.from_numpy(simgen.gaussian_alm(cl, nb, seed=901).astype(np.complex64)).cuda()
    plan = M.Plan(L, P, basis, cl, R, nphi, prec="fp32")
    ref = plan.cubic(alm).cpu().numpy()
    maps = plan.synthesize(alm)
    mu, w = plan.rings()
    W = torch.from_numpy(np.repeat((w * 2 * math.pi / nphi)[:, None], nphi, axis=1).astype(np.float32)).cuda()
    for call in range(2):
        beta = torch.full((nb, plan.n_max), float("nan"), dtype=torch.float64, device="cuda")
        M.modal_cubic_static(maps, W, R * nphi, P, nb, beta)
        torch.cuda.synchronize()
        got = beta.cpu().numpy()
        for b in range(nb):
            err = np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b])
            assert err <= 1e-5, (call, b, err)
    with pytest.raises(M.ModalError) as ei:
        M.modal_cubic_static(maps, W, R * nphi, P, 6000, beta)
    assert ei.value.status == M.MODAL_EINVAL
    plan.close()
