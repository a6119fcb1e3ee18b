"""Allocation failure without a fault: a workspace request the device cannot meet.

modal_set_chunk(4096) at l_max = 1000 with 16 modes asks for 4096 x 131 MB of Legendre
sums alone (over 500 GB, beyond the device), so cudaMalloc fails.  The call must return
MODAL_ENOMEM and leave the plan on its previous chunk, giving the same results as before.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import simgen

pytestmark = pytest.mark.gpu


def test_failed_set_chunk_keeps_the_previous_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    L, P, R, nphi = 1000, 16, 1001, 2048
    cl = simgen.cl_model(L)
    plan = M.Plan(L, P, simgen.shifted_legendre_basis(L, P), cl, R, nphi, prec="fp32")
    a = torch.from_numpy(simgen.gaussian_alm(cl, 2, seed=81).astype(np.complex64)).cuda()
    plan.set_chunk(2)
    before = plan.cubic(a)
    with pytest.raises(M.ModalError) as ei:
        plan.set_chunk(4096)
    assert ei.value.status == M.MODAL_ENOMEM
    assert "previous chunk is kept" in str(ei.value)
    assert plan.info().chunk == 2
    after = plan.cubic(a)
    plan.sync()
    assert torch.equal(before, after)
    plan.close()
