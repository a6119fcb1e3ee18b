"""Launch shapes (modal_get_tuning / modal_set_tuning) and the autotuner (modal_autotune).

Every legal setting must give the method's result: beta with the linear term against the
default shapes (||d beta|| / ||beta|| <= 5e-6: only the order of the FP32 partial sums over
pixels changes, which moves beta by about 1e-6 at l_max = 200; half the metric's 1e-5) and
against the FP64 oracle (<= 1e-5) at a non-default Legendre tile and after autotuning;
illegal settings are refused without changing the plan; the trispectrum's partial sums
follow a change of cubic_ctas; a captured batch graph is captured again after a member's
tuning changes; the autotuner leaves the plan on a legal setting with the same results
and its JSON cache returns the tuned setting without timing.
"""
import json

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


def _rel(a, b):
    a, b = a.detach().cpu().numpy(), b.detach().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup(M, L, P, prec, nb, seed):
    R, nphi = L + 1, max(16, 1 << int(np.ceil(np.log2(2 * L + 2))))
    cl = simgen.cl_model(L)
    basis = simgen.shifted_legendre_basis(L, P)
    plan = M.Plan(L, P, basis, cl, R, nphi, prec=prec)
    sims = simgen.gaussian_alm(cl, 4, seed=seed, stream=simgen.STREAM_LINEAR).astype(np.complex64)
    plan.linear_term(torch.from_numpy(sims).cuda(), finalize=True)
    a = torch.from_numpy(simgen.gaussian_alm(cl, nb, seed=seed + 1).astype(np.complex64)).cuda()
    return plan, a, sims, basis, cl, R, nphi


@pytest.mark.parametrize("P", [6, 10, 16])
def test_every_legendre_tile_and_split_gives_the_same_beta(P):
    M = _lib()
    L, nb = 64, 12
    plan, a, sims, basis, cl, R, nphi = _setup(M, L, P, "fp16x3", nb, seed=400 + P)
    base = plan.tuning()
    assert base["legendre_maps"] == 8 and base["cubic_ctas"] >= 1
    ref = plan.cubic(a, use_linear=True)
    gs = [g for g in range(1, 33) if (2 * P * g) % 16 == 0 and 2 * P * g <= 256]
    for g in gs:
        plan.set_tuning({"legendre_maps": g})
        assert plan.tuning()["legendre_maps"] == g
        assert _rel(plan.cubic(a, use_linear=True), ref) <= 5e-6, (P, g)
    for ctas, chunk in [(1, 5), (7, 12), (64, 3), (plan.npix // 128, 8)]:
        plan.set_tuning({"legendre_maps": gs[-1], "cubic_ctas": ctas, "chunk": chunk})
        assert _rel(plan.cubic(a, use_linear=True), ref) <= 5e-6, (P, ctas, chunk)
    # the largest Legendre tile against the FP64 oracle
    beta = plan.cubic(a, use_linear=True).cpu().numpy()
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    W = om.pixel_weights(w, nphi)
    pm = om.pair_means([osh.synthesize(s.astype(np.complex128), L, filt, mu, nphi) for s in sims])
    alm_host = a.cpu().numpy()
    for b in (0, nb - 1):
        oref = om.cubic_beta(osh.synthesize(alm_host[b].astype(np.complex128), L, filt, mu, nphi), W, pm)
        assert np.linalg.norm(beta[b] - oref) / np.linalg.norm(oref) <= 1e-5
    plan.sync()
    plan.close()


def test_illegal_settings_are_refused_and_change_nothing():
    M = _lib()
    plan, a, *_ = _setup(M, 48, 10, "fp16x3", 3, seed=420)
    before = plan.tuning()
    bad = [{"legendre_maps": 6},                  # 2 P G = 120: not a multiple of 16
           {"legendre_maps": 16},                 # 320 columns > 256
           {"legendre_maps": 0}, {"cubic_ctas": 0}, {"cubic_ctas": plan.npix // 128 + 1},
           {"chunk": 0}, {"chunk": 5000}]
    for t in bad:
        with pytest.raises(M.ModalError) as ei:
            plan.set_tuning(t)
        assert ei.value.status == M.MODAL_EINVAL, t
        assert plan.tuning() == before
    plan.close()


def test_quartic_follows_a_change_of_cubic_ctas():
    M = _lib()
    plan, a, *_ = _setup(M, 40, 6, "fp32", 3, seed=430)
    tau0 = plan.quartic(a, use_linear=True)
    for ctas in (1, 13, plan.npix // 128):
        plan.set_tuning({"cubic_ctas": ctas})
        assert _rel(plan.quartic(a, use_linear=True), tau0) <= 5e-6, ctas
    plan.sync()
    plan.close()


def test_batch_graph_is_recaptured_after_a_tuning_change():
    M = _lib()
    p1, a1, *_ = _setup(M, 32, 6, "fp16x3", 3, seed=440)
    p2, a2, *_ = _setup(M, 64, 6, "fp16x3", 4, seed=450)
    batch = M.Batch([p1, p2])
    batch.cubic([a1, a2], use_linear=True, graph=True)
    p2.set_tuning({"legendre_maps": 20, "chunk": 2, "cubic_ctas": 9})
    out = [o.clone() for o in batch.cubic([a1, a2], use_linear=True, graph=True)]
    assert torch.equal(out[0], p1.cubic(a1, use_linear=True))
    assert torch.equal(out[1], p2.cubic(a2, use_linear=True))
    batch.close()
    p1.close()
    p2.close()


def test_autotune_keeps_results_and_caches(tmp_path):
    M = _lib()
    plan, a, sims, basis, cl, R, nphi = _setup(M, 200, 16, "fp16x3", 16, seed=460)
    ref = plan.cubic(a, use_linear=True)
    chunk0 = plan.tuning()["chunk"]
    cache = str(tmp_path / "tiles.json")
    best, how = plan.autotune(a, use_linear=True, cache=cache)
    assert how == "measured" and best["ms"] > 0
    cur = plan.tuning()
    for k in ("chunk", "legendre_maps", "cubic_ctas"):
        assert cur[k] == best[k]
    assert best["chunk"] in (8, 16, chunk0) and 1 <= best["legendre_maps"] <= 8
    tuned = plan.cubic(a, use_linear=True)
    assert _rel(tuned, ref) <= 5e-6
    mu, w = osh.gl_nodes(R)
    filt = osh.filter_table(basis, cl)
    pm = om.pair_means([osh.synthesize(s.astype(np.complex128), 200, filt, mu, nphi) for s in sims])
    oref = om.cubic_beta(osh.synthesize(a[3].cpu().numpy().astype(np.complex128), 200, filt, mu, nphi),
                         om.pixel_weights(w, nphi), pm)
    assert np.linalg.norm(tuned[3].cpu().numpy() - oref) / np.linalg.norm(oref) <= 1e-5
    data = json.load(open(cache))
    assert len(data) == 1 and list(data.values())[0]["legendre_maps"] == best["legendre_maps"]
    # a second plan of the same configuration takes the cached shapes without timing
    plan2, a2, *_ = _setup(M, 200, 16, "fp16x3", 16, seed=460)
    best2, how2 = plan2.autotune(a2, use_linear=True, cache=cache)
    assert how2 == "cache"
    for k in ("chunk", "legendre_maps", "cubic_ctas"):
        assert best2[k] == best[k] and plan2.tuning()[k] == best[k]
    assert torch.equal(plan2.cubic(a2, use_linear=True), plan.cubic(a, use_linear=True))
    plan.sync()
    plan2.sync()
    plan.close()
    plan2.close()
