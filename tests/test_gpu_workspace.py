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


def test_init_refuses_tables_that_do_not_fit_before_allocating():
    """modal_init checks the resident tables and a one-map workspace against the free
    device memory before its first allocation.  A blocker tensor leaves 8 GB free; a plan at
    l_max = 2000 (about 25 GB of FP16X3 tables) must be refused with MODAL_ENOMEM, the free
    memory must be what it was, and a plan that fits must still build afterwards."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    L, P = 2000, 16
    cl = simgen.cl_model(L)
    basis = simgen.shifted_legendre_basis(L, P)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    leave = 8 << 30
    if free0 < leave + (1 << 30):
        pytest.skip("not enough free device memory to set the case up")
    blocker = torch.empty(free0 - leave, dtype=torch.uint8, device="cuda")
    try:
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        with pytest.raises(M.ModalError) as ei:
            M.Plan(L, P, basis, cl, L + 1, 4096, prec="fp16x3")
        assert ei.value.status == M.MODAL_ENOMEM
        msg = str(ei.value)
        assert "plan needs" in msg and "GB free" in msg
        need = float(msg.split("plan needs ")[1].split(" GB")[0])
        assert 24.0 < need < 40.0, msg
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        assert abs(free2 - free1) < (64 << 20)
        small = M.Plan(64, 6, simgen.shifted_legendre_basis(64, 6), simgen.cl_model(64), 65, 256, prec="fp16x3")
        small.close()
    finally:
        del blocker
        torch.cuda.empty_cache()
