"""Mixed-l_max batches (modal_batch_*): plans of different l_max run as one coefficient
pass, directly and as a captured CUDA graph, and give the same beta as the plans alone."""
import os

import numpy as np
import pytest
import torch

import simgen
from oracle import modal as om, sht as osh

pytestmark = pytest.mark.gpu

PRECS = [p for p in os.environ.get("MODAL_TEST_PRECS", "fp32,fp16x3,3xtf32").split(",") if p]
# (lmax, P, nrings, nphi, maps)
CONFIGS = [(32, 6, 33, 128, 3), (48, 6, 49, 128, 2), (64, 6, 65, 256, 4)]


def _setup(M, prec):
    plans, alms, sims = [], [], []
    for i, (L, P, R, nphi, nb) in enumerate(CONFIGS):
        basis = simgen.shifted_legendre_basis(L, P)
        cl = simgen.cl_model(L)
        try:
            plan = M.Plan(L, P, basis, cl, R, nphi, prec=prec)
        except M.ModalError as e:
            if prec != "fp32" and "not supported" in str(e):
                pytest.skip("precision %s not built" % prec)
            raise
        s = simgen.gaussian_alm(cl, 6, seed=90 + i, stream=simgen.STREAM_LINEAR).astype(np.complex64)
        plan.linear_term(torch.from_numpy(s).cuda(), finalize=True)
        plans.append(plan)
        sims.append(s)
        alms.append(torch.from_numpy(simgen.gaussian_alm(cl, nb, seed=80 + i).astype(np.complex64)).cuda())
    return plans, alms, sims


SCHEDULES = ["streams", "shared_cubic"]


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("prec", PRECS)
def test_mixed_lmax_batch_matches_single_plans(prec, schedule):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    plans, alms, sims = _setup(M, prec)
    batch = M.Batch(plans, schedule=schedule)
    for graph in (False, True, True):                  # direct, capture, replay
        out = [o.clone() for o in batch.cubic(alms, use_linear=True, graph=graph)]
        for plan, a, o in zip(plans, alms, out):
            assert torch.equal(o, plan.cubic(a, use_linear=True)), (prec, graph, plan.lmax)
    # new contents in the same buffers: the replayed graph reads them
    for i, (a, (L, P, R, nphi, nb)) in enumerate(zip(alms, CONFIGS)):
        a.copy_(torch.from_numpy(simgen.gaussian_alm(simgen.cl_model(L), nb, seed=70 + i).astype(np.complex64)))
    out = [o.clone() for o in batch.cubic(alms, use_linear=True, graph=True)]
    for plan, a, o in zip(plans, alms, out):
        assert torch.equal(o, plan.cubic(a, use_linear=True))
    # and the batch result against the oracle for the l_max = 64 plan
    L, P, R, nphi, nb = CONFIGS[2]
    basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    W = om.pixel_weights(w, nphi)
    pm = om.pair_means([osh.synthesize(s.astype(np.complex128), L, filt, mu, nphi) for s in sims[2]])
    alm_host = alms[2].cpu().numpy()
    for b in range(nb):
        ref = om.cubic_beta(osh.synthesize(alm_host[b].astype(np.complex128), L, filt, mu, nphi), W, pm)
        err = float(np.linalg.norm(out[2][b].cpu().numpy() - ref) / np.linalg.norm(ref))
        assert err <= 1e-5, (prec, b, err)
    for p in plans:
        p.sync()
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_graph_is_recaptured_after_a_plan_changes(schedule):
    """A captured batch graph holds the workspace pointers and chunk loop of its plans at
    capture time: after modal_set_chunk (which frees and reallocates the workspace),
    modal_set_retain_maps or modal_reset the next graph call must capture again, never
    replay launches on freed or stale buffers; so must a change of schedule."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    plans, alms, sims = _setup(M, "fp32")
    batch = M.Batch(plans, schedule=schedule)

    def check():
        out = [o.clone() for o in batch.cubic(alms, use_linear=True, graph=True)]
        for plan, a, o in zip(plans, alms, out):
            assert torch.equal(o, plan.cubic(a, use_linear=True)), plan.lmax

    check()                                             # capture
    check()                                             # replay
    plans[2].set_chunk(1)                               # new workspace, four chunk passes
    check()
    plans[1].set_chunk(2)
    plans[0].set_retain_maps(True)
    check()
    # reset then a new finalised mean (same buffers, new contents)
    plans[2].reset(1)
    with pytest.raises(M.ModalError):
        batch.cubic(alms, use_linear=True, graph=True)  # no finalised mean: refused, not replayed
    plans[2].linear_term(torch.from_numpy(sims[2][:3]).cuda(), finalize=True)
    check()
    batch.set_schedule(SCHEDULES[1 - SCHEDULES.index(schedule)])
    check()
    with pytest.raises(M.ModalError) as ei:
        batch.set_schedule(7)
    assert ei.value.status == M.MODAL_EINVAL
    check()
    for p in plans:
        p.sync()
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_mixed_lmax_batch_at_size_against_oracle(schedule):
    """The batched Monte Carlo configuration's plans, l_max = 500, 1000 and 2000 on their
    (l_max + 1) x next-pow2 grids with 16 modes (816 coefficients), band mask and linear term,
    maps in the ratio 2:1:1, captured as one graph and replayed, against the oracle summed
    over 3 sampled unmasked rings of each plan (a ring mask selects them on the GPU)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    P = 16
    plans, alms, sims, setups = [], [], [], []
    for i, (L, nb) in enumerate([(500, 4), (1000, 2), (2000, 2)]):
        R, nphi = L + 1, 1 << int(np.ceil(np.log2(2 * L + 2)))
        band = simgen.band_mask(R, 20.0)
        ok = np.nonzero(band[: (R + 1) // 2] > 0)[0]
        rings = ok[[0, len(ok) // 2, len(ok) - 1]]
        sel = np.zeros(R)
        sel[rings] = 1.0
        basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
        plan = M.Plan(L, P, basis, cl, R, nphi, prec="fp16x3", ring_mask=sel)
        s = simgen.gaussian_alm(cl, 4, seed=110 + i, stream=simgen.STREAM_LINEAR).astype(np.complex64)
        plan.linear_term(torch.from_numpy(s).cuda(), finalize=True)
        a = simgen.gaussian_alm(cl, nb, seed=120 + i).astype(np.complex64)
        plans.append(plan)
        sims.append(s)
        alms.append(torch.from_numpy(a).cuda())
        setups.append((L, R, nphi, basis, cl, rings, a))
    batch = M.Batch(plans, schedule=schedule)
    batch.cubic(alms, use_linear=True, graph=True)                      # capture
    out = [o.clone().cpu().numpy() for o in batch.cubic(alms, use_linear=True, graph=True)]   # replay
    for p, a, o in zip(plans, alms, out):                               # bit for bit as the plans alone
        assert np.array_equal(p.cubic(a, use_linear=True).cpu().numpy(), o), p.lmax
    for p in plans:
        p.sync()
    batch.close()
    for p in plans:
        p.close()
    for (L, R, nphi, basis, cl, rings, a), s, beta in zip(setups, sims, out):
        mu, w = osh.gl_nodes(R)
        filt = osh.filter_table(basis, cl)
        W = om.pixel_weights(w[rings], nphi)
        pm = om.pair_means(list(osh.synthesize_many(s.astype(np.complex128), L, filt, mu[rings], nphi)))
        maps = osh.synthesize_many(a.astype(np.complex128), L, filt, mu[rings], nphi)
        for b in range(a.shape[0]):
            err = float(np.linalg.norm(beta[b] - om.cubic_beta(maps[b], W, pm)) /
                        np.linalg.norm(om.cubic_beta(maps[b], W, pm)))
            print("mixed batch l_max=%d map %d: beta rel err %.3g" % (L, b, err))
            assert err <= 1e-5


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("other_P", [6, 10])
def test_shared_cubic_members_of_other_shapes_and_no_maps(other_P, graph):
    """Under the shared-cubic schedule members of one P share a cubic launch (one work queue
    over their maps and pixel ranges; a call with a member of another P runs each plan's own
    launches): members with other chunks and pixel ranges and a member without maps in the
    call must all still give each plan's own beta bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1105_2791_gb300 as M
    specs = [(40, 6, 5), (24, 6, 0), (56, 6, 7), (32, other_P, 3), (48, 6, 2)]     # (l_max, P, maps)
    plans, alms = [], []
    for i, (L, P, nb) in enumerate(specs):
        R, nphi = L + 1, 128
        cl = simgen.cl_model(L)
        plan = M.Plan(L, P, simgen.shifted_legendre_basis(L, P), cl, R, nphi, prec="fp16x3")
        s = simgen.gaussian_alm(cl, 4, seed=130 + i, stream=simgen.STREAM_LINEAR).astype(np.complex64)
        plan.linear_term(torch.from_numpy(s).cuda(), finalize=True)
        plans.append(plan)
        alms.append(torch.from_numpy(simgen.gaussian_alm(cl, max(nb, 1), seed=140 + i).astype(np.complex64))
                    .cuda()[:nb])
    plans[0].set_tuning({"chunk": 2, "cubic_ctas": 3})
    plans[2].set_tuning({"chunk": 3, "cubic_ctas": 11})
    plans[4].set_tuning({"cubic_ctas": 1})
    batch = M.Batch(plans, schedule="shared_cubic")
    for rep in range(2):
        out = [o.clone() for o in batch.cubic(alms, use_linear=True, graph=graph)]
        for plan, a, o in zip(plans, alms, out):
            assert o.shape == (a.shape[0], plan.n_max)
            assert torch.equal(o, plan.cubic(a, use_linear=True)), (plan.lmax, rep)
    # one P alone in the batch (every other member empty) takes the plan's own launches
    only = [a if i == 3 else a[:0] for i, a in enumerate(alms)]
    out = batch.cubic(only, use_linear=True, graph=graph)
    assert torch.equal(out[3], plans[3].cubic(alms[3], use_linear=True))
    for p in plans:
        p.sync()
    batch.close()
    for p in plans:
        p.close()
