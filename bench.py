#!/usr/bin/env python
"""Throughput of the modal bispectrum hot path on GB300: maps/s at l_max = 2000, 16 modes.

One step = one batch of B maps through every stage of the per-map path:
  linear-term pass   synthesis (filter + Legendre sums + ring FFT) and the pair sums
  coefficient pass   synthesis, cubic term with the linear term, covariance sums
  solve              FP64 Cholesky of zeta and the fNL estimate of every map
  adjoint            d fNL / d a_lm (the adjoint with g = d fNL / d beta) with maps recomputed
The workload is l_max = 2000 on 2001 Gauss-Legendre rings x 4096 longitudes, 16
shifted-Legendre modes (n_max = 816), C_l = 1/(l(l+1)), synthetic Gaussian a_lm
(seeded Philox).  All buffers are far larger than L2 (129 MB), so no flush is needed.

`value` is device-timed maps/s with inputs resident; `e2e` times the same step through
the public API with a_lm copied from pinned host memory every step (on a copy stream,
double-buffered, so that the next step's copy overlaps this step's kernels) and the fNL
values returned to the host.  `cpu_baseline` times the FP64 CPU oracle on a bounded sample of
the workload, and `parity` compares the GPU's beta on that sample with the oracle's.
`--impl reference` times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "maps/s at lmax=2000, 816 modes: batched/split-prec vs plain GPU path, err<=1e-5"
WORKLOAD = dict(lmax=2000, nrings=2001, nphi=4096, P=16)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--batch", type=int, default=32, help="maps per step per GPU")
    ap.add_argument("--prec", default="auto", help="fp32 | 3xtf32 | fp16x3 | bf16x3 | bf16 | auto")
    ap.add_argument("--no-baseline", action="store_true",
                    help="skip the plain FP32 comparison, the CPU baseline and the mixed-workload key")
    ap.add_argument("--no-tune", action="store_true",
                    help="mixed workload: time the default launch shapes only (no modal_autotune)")
    ap.add_argument("--cpu-rings", type=int, default=8, help="rings in the CPU-baseline sample")
    ap.add_argument("--lmax", type=int, default=2000, help="smaller l_max for profiler captures only")
    ap.add_argument("--chunk", type=int, default=32, help="maps per internal pass of the library")
    ap.add_argument("--linear", choices=["pixel", "ring"], default="pixel",
                    help="Monte Carlo pair means per pixel (default) or per ring (axisymmetric weights)")
    ap.add_argument("--adjoint", choices=["recompute", "kept"], default="recompute",
                    help="adjoint maps: synthesised again (default) or kept from the step's cubic call")
    ap.add_argument("--workload", choices=["l2000", "mixed", "trispectrum"], default="l2000",
                    help="l2000: the headline step; mixed: the batched Monte Carlo coefficient pass over "
                         "l_max 500 / 1000 / 2000 maps (2:1:1, 512 per step) as one captured graph; "
                         "trispectrum: the quartic modal coefficients (3876 modes) with per-ring Monte Carlo "
                         "terms on a band-masked sky")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- multi-rank timing
def max_over_ranks(ms, device=None):
    """Slowest rank's timed-region length (ms); identity on one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(maps_per_rank_per_step, steps, world, ms_max):
    """Whole-job maps/s: every rank's maps over the slowest rank's time (weak scaling)."""
    return maps_per_rank_per_step * steps * world / (ms_max / 1e3)


# ---------------------------------------------------------------- GPU arm
def legendre_flops(P, lmax, nrings):
    """Algorithmic flops of the Legendre sums per map: each (l, m, ring pair) contributes
    one multiply-add to 2P real outputs (re/im x P) of one parity."""
    n_alm = (lmax + 1) * (lmax + 2) // 2
    return 4.0 * P * n_alm * ((nrings + 1) // 2)


# DRAM traffic per launch (GB, dram__bytes_read + dram__bytes_write) of each stage's main
# kernel, from one-pass ncu captures (dram__bytes_*, gpu__time_duration) of one bench step at
# this workload; adjoint_pixel is the tensor-core map part (k_adjoint_v) and linear_term the
# harmonic sums (k_linh_s).  Keyed by (precision, lmax, nphi, P, maps per launch); an entry is
# removed whenever its kernel changes until it is captured again.
STAGE_TRAFFIC_GB = {
    ("fp16x3", 2000, 4096, 16, 32): {
        "legendre": 17.02 + 16.39, "pair_means": 25.87 + 8.88, "ring_c2r": 16.52 + 16.74,
        "ring_r2c": 17.78 + 17.17, "legendre_adjoint": 27.06 + 0.57, "legendre_adjoint_prep": 16.56 + 16.73,
        "legendre_prep": 0.515 + 8.394, "cubic": 17.84 + 0.03, "adjoint_pixel": 16.82 + 16.72,
        "linear_term": 2.75 + 0.035 + 0.03,
    },
}


def stage_rooflines(prec, L, R, nphi, P, n_max, n_pair, chunk, B, prof, n_steps, peaks, nsynth=3, probe=None):
    """Roofline of every timed stage: algorithmic work per step (flops or bytes) over the
    stage's live CUDA-event time, against its peak; sorted by time, largest first.
    nsynth: syntheses per chunk per step (3: linear term, coefficient pass and adjoint each
    synthesise; 2: the coefficient pass reads the linear-term pass's maps; 1: the adjoint
    does too)."""
    R_half, L1, npix = (R + 1) // 2, L + 1, R * nphi
    n_alm = (L + 1) * (L + 2) // 2
    probe = probe or {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", 1710.9)
    # FP32 SIMT and tf32 tensor rates: the library's probes in this run where available
    # (modal_peak_probe), else derived (lanes x clock) and the bf16 rate / 2 by nominal ratio
    fp32 = probe.get("fp32_simt") or 152 * 128 * 2 * 2.07e9 / 1e12
    fp32_src = ("measured in this run: packed f32x2 FMA probe" if probe.get("fp32_simt")
                else "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz")
    tf32 = probe.get("tf32_tensor") or bf16 / 2.0
    tf32_src = ("measured in this run: tcgen05 kind::tf32 probe (M128 N256) / 3 products" if probe.get("tf32_tensor")
                else "measured bf16 sustained / 2 (tf32) / 3 products")
    split = {"fp16x3": 3.0, "bf16x3": 3.0, "3xtf32": 6.0, "bf16": 1.0}
    tensor_peak = bf16 / split[prec] if prec in split else None
    if prec == "3xtf32" and probe.get("tf32_tensor"):
        tensor_peak = tf32 / 3.0
    launches = B // chunk
    delta_bytes = chunk * P * R_half * L1 * 16.0                  # E and O rows, complex64
    map_bytes = chunk * P * npix * 4.0
    # stage: (bound, work per launch, launches per step, peak, unit)
    work = {
        "legendre": ("tensor" if tensor_peak else "alu", legendre_flops(P, L, R) * chunk, nsynth * launches),
        "legendre_adjoint": ("tensor" if tensor_peak else "alu", legendre_flops(P, L, R) * chunk, launches),
        "ring_c2r": ("hbm", delta_bytes + map_bytes, nsynth * launches),
        "ring_r2c": ("hbm", delta_bytes + map_bytes, launches),
        "adjoint_pixel": ("tensor" if tensor_peak else "alu", 2.0 * P * n_pair * npix * chunk, launches),
        "cubic": ("alu", 2.0 * n_max * npix * chunk, launches),
        # linear term: split plans sum conj(F_c) a_lm in harmonic space (the pair-mean table of
        # n_pair x n_alm complex64 read once per launch, the a_lm once); the FP32 plan runs the
        # pixel-space product (one multiply-add per pair, basis function and pixel)
        "linear_term": (("hbm", (n_pair + chunk) * n_alm * 8.0, launches) if tensor_peak
                        else ("alu", 2.0 * n_pair * P * npix * chunk, launches)),
        "pair_means": ("hbm", map_bytes + 2.0 * n_pair * npix * 8, launches),
        "legendre_prep": ("hbm", chunk * n_alm * 8.0 + chunk * P * 2 * n_alm * 2 * 2.0, nsynth * launches),
        "legendre_adjoint_prep": ("hbm", 2.0 * delta_bytes, launches),
    }
    traffic = STAGE_TRAFFIC_GB.get((prec, L, nphi, P, chunk), {})
    out = []
    for stage, (bound, per_launch, nl) in work.items():
        if stage not in prof or not prof[stage][1]:
            continue
        ms = prof[stage][0] / n_steps
        total = per_launch * nl
        if bound == "hbm":
            peak, unit, achieved = hbm, "GB/s", total / (ms / 1e3) / 1e9
            src = "measured HBM copy"
        elif bound == "tensor":
            tf32x3 = stage == "adjoint_pixel" or prec == "3xtf32"   # these run 3xTF32
            tp = tf32 / 3.0 if tf32x3 else tensor_peak
            peak, unit, achieved = tp, "TFLOP/s", total / (ms / 1e3) / 1e12
            src = tf32_src if tf32x3 else "measured bf16 sustained / %g products per useful MAC" % split[prec]
        else:
            peak, unit, achieved = fp32, "TFLOP/s", total / (ms / 1e3) / 1e12
            src = fp32_src
        t = traffic.get(stage)
        extra = {}
        if achieved > peak:
            # the peaks are a torch copy kernel and cuBLAS, not hard ceilings: a kernel that
            # streams well can exceed them slightly; flagged, not capped
            src += "; achieved above this measured rate (not a hard ceiling)"
        out.append({"stage": stage, "bound": bound, "achieved": round(achieved, 2), "peak": round(peak, 1),
                    "unit": unit, "frac": round(achieved / peak, 4), "peak_source": src,
                    "traffic": round(t, 2) if t is not None else None,
                    "ms_per_step": round(ms, 3), "launches_per_step": nl,
                    "per_launch": "%.4g %s" % (per_launch / (1e9 if bound == "hbm" else 1.0),
                                               "GB" if bound == "hbm" else "flop"), **extra})
    out.sort(key=lambda r: -r["ms_per_step"])
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import simgen
    import paper_1105_2791_gb300 as M

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    L, R, nphi, P = WORKLOAD["lmax"], WORKLOAD["nrings"], WORKLOAD["nphi"], WORKLOAD["P"]
    if args.lmax != L:
        L, R = args.lmax, args.lmax + 1
        nphi = 1 << int(math.ceil(math.log2(2 * L + 2)))
    B = args.batch
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    alm_host = simgen.gaussian_alm(cl, B, seed=3 + 1000 * rank).astype(np.complex64)
    alm_pinned = torch.from_numpy(alm_host).pin_memory()
    alm = alm_pinned.to(dev)
    lin_sims = torch.from_numpy(simgen.gaussian_alm(cl, 2, seed=4 + 1000 * rank,
                                                    stream=simgen.STREAM_LINEAR).astype(np.complex64)).to(dev)

    # The step's batch is a linear-term sample and the coefficient pass's input: its maps are
    # synthesised once for both (modal_linear_term keeps them, modal_cubic_retained reads
    # them; the batch must fit one chunk).  The adjoint differentiates the coefficient pass
    # and synthesises the maps again (recomputation, not storage).  --adjoint kept reuses the
    # kept maps for the adjoint too (modal_backward_retained); the default run times that
    # variant as well, in a short extra pass reported beside.
    kept_ok = B <= args.chunk
    if args.adjoint == "kept" and not kept_ok:
        raise SystemExit("--adjoint kept needs --batch <= --chunk")
    retain = args.adjoint == "kept"

    def make_plan(prec):
        try:
            plan = M.Plan(L, P, basis, cl, R, nphi, prec=prec)
        except M.ModalError as e:
            if "not supported" in str(e):
                return None
            raise
        plan.set_chunk(min(args.chunk, B))
        plan.set_retain_maps(kept_ok)
        plan.reuse_maps = kept_ok                      # coefficient pass on the linear-term pass's maps
        if args.linear == "ring":
            plan.set_linear_mode("ring")
        plan.linear_term(lin_sims, finalize=True)      # a mean to subtract from the first step on
        return plan

    if args.prec == "auto":
        plan, prec = None, None
        for cand in ("fp16x3", "3xtf32", "fp32"):
            plan = make_plan(cand)
            if plan is not None:
                prec = cand
                break
    else:
        prec = args.prec
        plan = make_plan(prec)
        if plan is None:
            raise SystemExit("precision %s not available" % prec)

    alpha = plan.alpha_local()
    beta = torch.empty((B, plan.n_max), dtype=torch.float64, device=dev)
    grad = torch.empty((B, plan.n_alm), dtype=torch.complex64, device=dev)
    # Seed the covariance sums with 2 n_max random vectors so that zeta is positive definite
    # from the first step on (a real run accumulates N_cov >> n_max simulations first).
    gen = torch.Generator(device=dev).manual_seed(5)
    plan.cov_accumulate(torch.randn((2 * plan.n_max, plan.n_max), generator=gen, device=dev, dtype=torch.float64))
    # the adjoint differentiates fNL: g = d fNL / d beta = zeta^-1 alpha / alpha^T zeta^-1 alpha
    w_fnl, _ = plan.fnl_weights(alpha)
    g = w_fnl[None, :].repeat(B, 1).contiguous()
    torch.cuda.synchronize()

    side = torch.cuda.Stream(device=dev)

    def step(pl, a, overlap=True, kept=None):
        pl.linear_term(a)
        if pl.reuse_maps:
            pl.cubic_retained(a, use_linear=True, out=beta)
        else:
            pl.cubic(a, use_linear=True, out=beta)
        pl.cov_accumulate(beta)
        backward = pl.backward_retained if (retain if kept is None else kept) else pl.backward
        if not overlap:                                  # per-stage timing: one stream, stages in order
            fnl, sigma = pl.solve(alpha, beta)
            backward(a, g, use_linear=True, out=grad)
            return fnl, sigma
        # the FP64 solve (latency-bound, a few CTAs) runs on a side stream beside the adjoint
        ready = torch.cuda.Event()
        ready.record(torch.cuda.current_stream())
        backward(a, g, use_linear=True, out=grad)
        side.wait_event(ready)
        fnl, sigma = M.modal_solve(pl.h, alpha, beta, beta.shape[0], stream=side)
        return fnl, sigma

    copy_stream = torch.cuda.Stream(device=dev)

    def run_steps(pl, a, n, e2e, profile, kept):
        """n steps on the current stream.  e2e: every step's a_lm is copied in from pinned
        host memory on a copy stream into one of two device buffers, so that the copy for
        step i + 1 runs beside the kernels of step i; the kernels of a step wait for its copy,
        and a copy waits until the step that last used its buffer is done."""
        cur = torch.cuda.current_stream()
        if not e2e:
            for _ in range(n):
                step(pl, a, overlap=not profile, kept=kept)
            return
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        free = [torch.cuda.Event(), torch.cuda.Event()]
        for ev in free:
            ev.record(cur)

        def issue_copy(i):
            j = i % 2
            copy_stream.wait_event(free[j])
            with torch.cuda.stream(copy_stream):
                a[j].copy_(alm_pinned, non_blocking=True)
            copied[j].record(copy_stream)

        if n > 0:
            issue_copy(0)
        for i in range(n):
            if i + 1 < n:
                issue_copy(i + 1)
            cur.wait_event(copied[i % 2])
            step(pl, a[i % 2], overlap=not profile, kept=kept)
            free[i % 2].record(cur)

    def timed(pl, a, steps, warmup, e2e=False, profile=False, kept=None):
        run_steps(pl, a, warmup, e2e, profile, kept)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        M.modal_get_profile(pl.h)                          # reset counters
        M.modal_set_profiling(pl.h, profile)
        st = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(st)
        run_steps(pl, a, steps, e2e, profile, kept)
        ev1.record(st)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        prof = M.modal_get_profile(pl.h)
        M.modal_set_profiling(pl.h, False)
        ms = max_over_ranks(ms, dev)
        return ms, prof

    # roofline denominators the measured-peaks file does not hold: FP32 SIMT, FP64 SIMT, tcgen05 tf32
    # and f16 rates, each probed once on this GPU before the timed region
    probe = {}
    for kind in ("fp32_simt", "fp64_simt", "tf32_tensor", "f16_tensor"):
        try:
            probe[kind] = round(M.modal_peak_probe(kind), 2)
        except M.ModalError as e:
            probe[kind + "_error"] = str(e)[:120]
    torch.cuda.synchronize()

    K, W = args.steps, args.warmup
    with ClockSampler(local) as clocks:
        ms, prof_plain_timing = timed(plan, alm, K, W)
    clk = clocks.summary()
    # kernel-level timing in a separate timed pass with per-launch events
    _, prof = timed(plan, alm, max(1, K // 2), 1, profile=True)
    launches = sum(n for (_, n) in prof_plain_timing.values())
    # end to end through the public API from pinned host memory
    a_e2e = [torch.empty_like(alm), torch.empty_like(alm)]
    with ClockSampler(local) as e2e_clocks:
        e2e_ms, _ = timed(plan, a_e2e, K, max(W, 2), e2e=True)
    # the same step with the adjoint on the cubic call's kept maps (or, under --adjoint kept,
    # with the maps synthesised again), device-timed
    other = None
    if kept_ok:
        oms, _ = timed(plan, alm, K, 1, kept=not retain)
        other = {"adjoint_maps": "synthesised again" if retain else "kept from the step's cubic call",
                 "value": round(job_throughput(B, K, world, oms), 3), "ms_per_step": round(oms / K, 3)}

    # the headline step's beta of map 0 (the step's coefficient pass, linear term on)
    beta_headline = beta[0].double().cpu().numpy().copy() if args.lmax == WORKLOAD["lmax"] else None
    value = job_throughput(B, K, world, ms)
    e2e_value = job_throughput(B, K, world, e2e_ms)
    n_prof_steps = max(1, K // 2)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    nsynth = (1 if retain else 2) if kept_ok else 3
    rooflines = stage_rooflines(prec, L, R, nphi, P, plan.n_max, plan.n_pair, min(B, args.chunk), B, prof,
                                n_prof_steps, peaks, nsynth=nsynth, probe=probe)
    top = rooflines[0]
    roof = {k: top[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "peak_source")}
    if top["traffic"] is not None:
        roof["traffic_unit"] = "GB per launch (ncu dram bytes read + written)"
    roof["kernel"] = "%s: the stage with the largest time per step (%.3f ms, %d launches), %s per launch" % (
        top["stage"], top["ms_per_step"], top["launches_per_step"], top["per_launch"])

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": "maps/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms / K, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "3xtf32": "tf32x3", "fp16x3": "f16x3", "bf16x3": "bf16x3", "bf16": "bf16"}[prec],
        "data": "synthetic",
        "config": {"workload": "lmax=%d GL %dx%d, P=%d (n_max=%d), batch %d maps/step/GPU, %s" % (
                       L, R, nphi, P, plan.n_max, B, prec),
                   "lmax": L, "nrings": R, "nphi": nphi, "P": P, "n_max": plan.n_max, "batch_per_gpu": B,
                   "precision": prec, "linear_means": args.linear,
                   "coefficient_maps": ("kept from the step's linear-term synthesis" if kept_ok
                                        else "synthesised again"),
                   "adjoint_maps": "kept from the step's cubic call" if retain else "synthesised again",
                   "syntheses_per_map_per_step": nsynth,
                   "l2": "inputs and intermediates > L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": {"value": round(e2e_value, 3), "unit": "maps/s",
                "h2d_bytes_per_step": int(alm.numel() * 8), "d2h_bytes_per_step": int(B * 8 + 8),
                "clocks": e2e_clocks.summary()},
        "roofline": roof,
        "rooflines": rooflines,
        "peak_probes_tflops": probe,
        "other_adjoint": other,
        "stage_ms_per_step": {k: round(v[0] / n_prof_steps, 3) for k, v in prof.items() if v[1]},
    }

    # the plain comparators time through the same barrier / max-over-ranks path, so they run
    # only in single-process runs (under torchrun rank 0 would wait on ranks that have left)
    if rank == 0 and world == 1 and args.lmax == WORKLOAD["lmax"] and not args.no_baseline:
        # the batched Monte Carlo configuration (l_max 500/1000/2000, 2:1:1, one captured graph),
        # timed on the same GPU after the headline step's plan is released
        plan.close()
        try:
            mx = mixed_measure(M, dev, prec, args.chunk, max(2, K // 2), 2)
            result["mixed_workload"] = {
                "metric": "maps/s, mixed l_max 500/1000/2000 (2:1:1) coefficient pass with linear term, P=16",
                "value": round(mx["value"], 3), "unit": "maps/s", "ms_per_step": round(mx["ms"], 3),
                "launch_shapes": "autotuned per plan (modal_autotune, untimed)",
                "default_shapes_value": round(mx["default_value"], 3),
                "default_shapes_ms_per_step": round(mx["default_ms"], 3),
                "shared_cubic_schedule_value": round(mx["shared_cubic_value"], 3),
                "tuning": mx.get("tuning"), "maps_per_step": mx["maps_per_step"],
                "steps": max(2, K // 2), "gpu_launches_per_step": int(mx["launches"]), "clocks": mx["clocks"]}
        except Exception as e:          # the headline line is printed whatever happens here
            result["mixed_workload"] = {"error": str(e)[:200]}
    if rank == 0 and world == 1 and not args.no_baseline and prec != "fp32":
        plan.close()                    # (a no-op when the mixed workload already released it)
        plain = make_plan("fp32")
        plain.cov_accumulate(torch.randn((2 * plain.n_max, plain.n_max), generator=gen, device=dev,
                                         dtype=torch.float64))
        pms, _ = timed(plain, alm, max(1, K // 2), 1)
        result["plain_fp32_value"] = round(B * max(1, K // 2) / (pms / 1e3), 3)
        result["speedup_vs_plain_fp32"] = round(value / world / result["plain_fp32_value"], 3)
        # the metric's comparator proper: the plain FP32 path one map per launch (the adjoint
        # synthesising its maps again, as in the default step)
        try:
            plain.set_chunk(1)
            plain.reuse_maps = False                   # one map per launch: every call synthesises
            oms, _ = timed(plain, alm, max(1, K // 2), 1, kept=False)
            result["plain_one_map_value"] = round(B * max(1, K // 2) / (oms / 1e3), 3)
            result["speedup_vs_plain_one_map"] = round(value / world / result["plain_one_map_value"], 3)
        except Exception as e:       # the measurement line is printed whatever happens here
            result["plain_one_map_error"] = str(e)[:200]
        plain.close()
    if rank == 0 and world == 1 and not args.no_baseline:
        result["cpu_baseline"], result["parity"] = cpu_baseline(args.cpu_rings, prec, beta_headline)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------- oracle (CPU baseline and reference arm)
def oracle_step_sample(nring_sample, seed=3):
    """One map of the workload through the oracle's per-map step (synthesis, pair means,
    cubic with the linear term, adjoint) on `nring_sample` rings spread pole to equator;
    returns (seconds, extrapolated seconds per map, rings, sample) where sample holds the
    map's a_lm (complex64 values), the rings and the oracle's maps on them."""
    import simgen
    from oracle import modal as om, sht as osh

    L, R, nphi, P = WORKLOAD["lmax"], WORKLOAD["nrings"], WORKLOAD["nphi"], WORKLOAD["P"]
    basis = simgen.shifted_legendre_basis(L, P)
    cl = simgen.cl_model(L)
    filt = osh.filter_table(basis, cl)
    a32 = simgen.gaussian_alm(cl, 1, seed=seed).astype(np.complex64)
    a = a32[0].astype(np.complex128)
    mu, w = osh.gl_nodes(R)
    rings = np.unique(np.linspace(0, R // 2, nring_sample).astype(int))
    t0 = time.perf_counter()
    maps = osh.synthesize(a, L, filt, mu[rings], nphi)
    pm = om.pair_means([maps])
    beta = om.cubic_beta(maps, om.pixel_weights(w[rings], nphi), pm)
    g = np.ones(beta.size) / beta.size
    om.adjoint_grad(a, g, L, filt, mu[rings], w[rings], nphi, None, pm)
    dt = time.perf_counter() - t0
    return dt, dt * R / len(rings), len(rings), {"alm": a32, "rings": rings, "maps": maps, "basis": basis, "cl": cl,
                                                 "filt": filt, "mu": mu, "w": w}


def gpu_beta_error(prec, sample, seed=4):
    """beta with the linear term of the oracle sample's map on the GPU, restricted by a ring
    mask to the sampled rings, against the oracle's on the same rings; the pair means come
    from one independent simulation, synthesised by each side.  Returns
    ||beta_gpu - beta_oracle||_2 / ||beta_oracle||_2."""
    import torch
    import simgen
    import paper_1105_2791_gb300 as M
    from oracle import modal as om, sht as osh

    L, R, nphi, P = WORKLOAD["lmax"], WORKLOAD["nrings"], WORKLOAD["nphi"], WORKLOAD["P"]
    rings = sample["rings"]
    sim = simgen.gaussian_alm(sample["cl"], 1, seed=seed, stream=simgen.STREAM_LINEAR).astype(np.complex64)
    sim_maps = osh.synthesize(sim[0].astype(np.complex128), L, sample["filt"], sample["mu"][rings], nphi)
    ref = om.cubic_beta(sample["maps"], om.pixel_weights(sample["w"][rings], nphi), om.pair_means([sim_maps]))
    mask = np.zeros(R)
    mask[rings] = 1.0
    plan = M.Plan(L, P, sample["basis"], sample["cl"], R, nphi, prec=prec, ring_mask=mask)
    try:
        plan.set_chunk(1)
        plan.linear_term(torch.from_numpy(sim).cuda(), finalize=True)
        beta = plan.cubic(torch.from_numpy(sample["alm"]).cuda(), use_linear=True).cpu().numpy()[0]
        plan.sync()
    finally:
        plan.close()
    return float(np.linalg.norm(beta - ref) / np.linalg.norm(ref))


def oracle_map_seconds(L, R, nphi, P, nring_sample=None, seed=5):
    """Seconds per map of the oracle's per-map step (synthesis, pair means, cubic with the
    linear term, adjoint) at l_max = L on an R x nphi grid, on all rings or on a sample of
    them spread pole to equator and extrapolated by ring count."""
    import simgen
    from oracle import modal as om, sht as osh
    basis, cl = simgen.shifted_legendre_basis(L, P), simgen.cl_model(L)
    filt = osh.filter_table(basis, cl)
    a = simgen.gaussian_alm(cl, 1, seed=seed)[0]
    mu, w = osh.gl_nodes(R)
    rings = np.arange(R) if nring_sample is None else np.unique(np.linspace(0, R // 2, nring_sample).astype(int))
    t0 = time.perf_counter()
    maps = osh.synthesize(a, L, filt, mu[rings], nphi)
    pm = om.pair_means([maps])
    beta = om.cubic_beta(maps, om.pixel_weights(w[rings], nphi), pm)
    om.adjoint_grad(a, np.ones(beta.size) / beta.size, L, filt, mu[rings], w[rings], nphi, None, pm)
    return (time.perf_counter() - t0) * R / len(rings)


FULLGRID_GOLDEN = os.path.join(ROOT, "tests", "golden", "fullsize_beta_l2000_p16.json")


def cpu_baseline(nring_sample, prec=None, beta_headline=None):
    """The oracle timed on a bounded sample; with prec, also the GPU's beta on that sample
    against the oracle's (the accepted error metric, tolerance 1e-5), and, with the headline
    step's beta of its first map, that beta against the stored full-grid oracle result."""
    dt, per_map, k, sample = oracle_step_sample(nring_sample)
    base = {"value": round(1.0 / per_map, 8), "unit": "maps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "1 map at lmax=2000 (P=16, 4096 longitudes) on %d of 2001 rings: synthesis, pair means, "
                      "cubic with linear term, adjoint; %.1f s, extrapolated by ring count" % (k, dt)}
    try:
        base["seconds_per_map"] = {
            "lmax32_P6_33x128_full_grid": round(oracle_map_seconds(32, 33, 128, 6), 4),
            "lmax500_P10_501x1024_64_rings_extrapolated": round(oracle_map_seconds(500, 501, 1024, 10, 64), 3),
            "lmax2000_P16_2001x4096_%d_rings_extrapolated" % k: round(per_map, 1)}
    except Exception as e:              # the measurement line is printed whatever happens here
        base["seconds_per_map_error"] = str(e)[:200]
    if prec is None:
        return base, None
    parity = {"metric": "||beta_gpu - beta_oracle||_2 / ||beta_oracle||_2", "tol": 1e-5, "precision": prec,
              "sample": "the oracle sample's map on its %d rings (ring-masked plan), linear term from one "
                        "independent simulation" % k}
    try:
        err = gpu_beta_error(prec, sample)
        parity.update(beta_rel_err=float("%.3g" % err), ok=bool(err <= 1e-5))
    except Exception as e:          # the measurement line is printed whatever happens here
        parity.update(error=str(e)[:200])
    if beta_headline is not None and os.path.exists(FULLGRID_GOLDEN):
        ref = np.array(json.load(open(FULLGRID_GOLDEN))["beta_lin_G"])
        fe = float(np.linalg.norm(beta_headline - ref) / np.linalg.norm(ref))
        parity["full_grid"] = {"beta_rel_err": float("%.3g" % fe), "ok": bool(fe <= 1e-5),
                               "sample": "the headline step's map 0 (seed 3) with the linear term of its 2 "
                                         "simulations (seed 4), every pixel of the 2001 x 4096 grid, against the "
                                         "oracle result stored by tests/golden/make_fullsize.py"}
    return base, parity


MIXED = [(500, 256), (1000, 128), (2000, 128)]      # (l_max, maps per step): the 2:1:1 batched mix


def mixed_measure(M, dev, prec, chunk, steps, warmup, rank=0, world=1, local=0, tune=True):
    """Batched Monte Carlo coefficient pass: 256 maps at l_max = 500, 128 at 1000 and 128 at
    2000 per step (P = 16, 20-degree band mask, linear term), one plan per l_max grouped in a
    modal batch and replayed as one CUDA graph.  Timed first with the default launch shapes
    (per-plan streams, then the shared-cubic schedule), then (tune) after modal_autotune has
    tuned each plan on its own maps (untimed; the batch graph is captured again).  Returns a
    dict: value / ms (tuned if tune, else default), default_value / default_ms,
    shared_cubic_value / shared_cubic_ms, tuning per l_max, kernels per step, clocks, maps
    per step."""
    import torch
    import simgen

    P = 16
    plans, alms = [], []
    for i, (L, nb) in enumerate(MIXED):
        R, nphi = L + 1, 1 << int(math.ceil(math.log2(2 * L + 2)))
        cl = simgen.cl_model(L)
        pl = M.Plan(L, P, simgen.shifted_legendre_basis(L, P), cl, R, nphi, prec=prec,
                    ring_mask=simgen.band_mask(R, 20.0))
        pl.set_chunk(min(chunk, nb))
        pl.linear_term(torch.from_numpy(simgen.gaussian_alm(cl, 4, seed=50 + i, stream=simgen.STREAM_LINEAR)
                                        .astype(np.complex64)).to(dev), finalize=True)
        plans.append(pl)
        alms.append(torch.from_numpy(simgen.gaussian_alm(cl, nb, seed=60 + i + 1000 * rank).astype(np.complex64)).to(dev))
    batch = M.Batch(plans)
    n_maps = sum(nb for _, nb in MIXED)
    st = torch.cuda.current_stream()

    def timed():
        for _ in range(warmup):
            batch.cubic(alms, use_linear=True, graph=True)
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clocks:
            ev0.record(st)
            for _ in range(steps):
                batch.cubic(alms, use_linear=True, graph=True)
            ev1.record(st)
            torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
        return job_throughput(n_maps, steps, world, ms), ms / steps, clocks.summary()

    out = {"maps_per_step": n_maps}
    out["default_value"], out["default_ms"], clk = timed()
    out["value"], out["ms"], out["clocks"] = out["default_value"], out["default_ms"], clk
    # the lockstep schedule with one persistent cubic launch per chunk pass (same betas)
    batch.set_schedule("shared_cubic")
    out["shared_cubic_value"], out["shared_cubic_ms"], _ = timed()
    batch.set_schedule("streams")
    if tune:
        out["tuning"] = {}
        for (L, nb), pl, a in zip(MIXED, plans, alms):
            best, _ = pl.autotune(a, use_linear=True)
            out["tuning"]["lmax%d" % L] = best
        out["value"], out["ms"], out["clocks"] = timed()
    # kernels per step: one direct (uncaptured) pass, counted by the plans
    for pl in plans:
        M.modal_get_profile(pl.h)
    batch.cubic(alms, use_linear=True, graph=False)
    torch.cuda.synchronize()
    out["launches"] = sum(sum(n for (_, n) in M.modal_get_profile(pl.h).values()) for pl in plans)
    for pl in plans:
        pl.sync()
    batch.close()
    for pl in plans:
        pl.close()
    return out


def run_mixed(args):
    """The batched Monte Carlo configuration as the timed workload (its own metric line)."""
    import torch
    import torch.distributed as dist

    import paper_1105_2791_gb300 as M

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = "fp16x3" if args.prec == "auto" else args.prec
    K, W = args.steps, args.warmup
    mx = mixed_measure(M, dev, prec, args.chunk, K, W, rank, world, local, tune=not args.no_tune)
    value, ms, launches, clk, n_maps = mx["value"], mx["ms"], mx["launches"], mx["clocks"], mx["maps_per_step"]
    if rank == 0:
        print(json.dumps({
            "metric": "maps/s, mixed l_max 500/1000/2000 (2:1:1) coefficient pass with linear term, P=16",
            "value": round(value, 3), "unit": "maps/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "3xtf32": "tf32x3", "fp16x3": "f16x3", "bf16x3": "bf16x3", "bf16": "bf16"}[prec],
            "data": "synthetic",
            "config": {"workload": "batched Monte Carlo: 256 @ l_max 500, 128 @ 1000, 128 @ 2000 per step, "
                                   "P=16, band mask, one captured CUDA graph", "maps_per_step": n_maps,
                       "precision": prec, "l2": "inputs and intermediates > L2 (no flush)",
                       "launch_shapes": "default" if args.no_tune else "autotuned per plan (modal_autotune, untimed)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "default_shapes_value": round(mx["default_value"], 3), "tuning": mx.get("tuning"),
            "shared_cubic_schedule_value": round(mx["shared_cubic_value"], 3),
            "clocks": clk, "gpu_launches": int(launches) * K,
            "roofline": None, "e2e": None,
        }), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_trispectrum(args):
    """Trispectrum modal coefficients (Sec. IV) at l_max = 2000, 16 basis functions (3876
    quartic modes), 20-degree band mask, per-ring Monte Carlo means: one step = B maps
    through synthesis and modal_quartic with the single-pair and two-pair terms."""
    import torch
    import torch.distributed as dist

    import simgen
    import paper_1105_2791_gb300 as M

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L, P = args.lmax, WORKLOAD["P"]
    R, nphi = L + 1, 1 << int(math.ceil(math.log2(2 * L + 2)))
    B = args.batch
    prec = "fp16x3" if args.prec == "auto" else args.prec
    cl = simgen.cl_model(L)
    plan = M.Plan(L, P, simgen.shifted_legendre_basis(L, P), cl, R, nphi, prec=prec,
                  ring_mask=simgen.band_mask(R, 20.0))
    plan.set_chunk(min(args.chunk, B))
    plan.set_linear_mode("ring")
    plan.linear_term(torch.from_numpy(simgen.gaussian_alm(cl, 4, seed=70 + 1000 * rank, stream=simgen.STREAM_LINEAR)
                                      .astype(np.complex64)).to(dev), finalize=True)
    alm_pinned = torch.from_numpy(simgen.gaussian_alm(cl, B, seed=71 + 1000 * rank).astype(np.complex64)).pin_memory()
    alm = alm_pinned.to(dev)
    tau = torch.empty((B, plan.n_quad), dtype=torch.float64, device=dev)
    tau_host = torch.empty((B, plan.n_quad), dtype=torch.float64).pin_memory()

    def timed(a, steps, warmup, e2e=False, profile=False):
        for _ in range(warmup):
            plan.quartic(a, use_linear=True, out=tau)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        M.modal_get_profile(plan.h)
        M.modal_set_profiling(plan.h, profile)
        st = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(st)
        for _ in range(steps):
            if e2e:
                a.copy_(alm_pinned, non_blocking=True)
            plan.quartic(a, use_linear=True, out=tau)
            if e2e:
                tau_host.copy_(tau, non_blocking=True)
        ev1.record(st)
        torch.cuda.synchronize()
        prof = M.modal_get_profile(plan.h)
        M.modal_set_profiling(plan.h, False)
        return max_over_ranks(ev0.elapsed_time(ev1), dev), prof

    # roofline denominators the measured-peaks file does not hold: FP32 SIMT, FP64 SIMT, tcgen05 tf32
    # and f16 rates, each probed once on this GPU before the timed region
    probe = {}
    for kind in ("fp32_simt", "fp64_simt", "tf32_tensor", "f16_tensor"):
        try:
            probe[kind] = round(M.modal_peak_probe(kind), 2)
        except M.ModalError as e:
            probe[kind + "_error"] = str(e)[:120]
    torch.cuda.synchronize()

    K, W = args.steps, args.warmup
    with ClockSampler(local) as clocks:
        ms, prof0 = timed(alm, K, W)
    n_prof = max(1, K // 2)
    _, prof = timed(alm, n_prof, 1, profile=True)
    e2e_ms, _ = timed(torch.empty_like(alm), K, max(W, 2), e2e=True)
    value = job_throughput(B, K, world, ms)
    q_ms, q_n = prof["quartic"]
    npix = R * nphi
    useful = 2.0 * plan.n_quad * npix * B * n_prof
    achieved = useful / (q_ms / 1e3) / 1e12
    if "fp32_simt" in probe:
        peak, peak_source = probe["fp32_simt"], "measured in this run: packed f32x2 FMA probe"
    else:
        peak, peak_source = 152 * 128 * 2 * 2.07e9 / 1e12, "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
    roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
            "peak_source": peak_source,
            "frac": round(achieved / peak, 4), "traffic": None,
            "kernel": "quartic (sum_x W M_p M_r M_s M_u, 3876 modes), %d launches, %.3f ms per launch; useful "
                      "flops 2 x n_quad x npix per map" % (q_n, q_ms / max(q_n, 1))}
    result = {
        "metric": "maps/s, trispectrum modal coefficients at l_max=%d, %d modes, per-ring MC terms" % (L, plan.n_quad),
        "value": round(value, 3), "unit": "maps/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms / K, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "3xtf32": "tf32x3", "fp16x3": "f16x3", "bf16x3": "bf16x3", "bf16": "bf16"}[prec],
        "data": "synthetic",
        "config": {"workload": "trispectrum: lmax=%d GL %dx%d, P=%d (3876 quartic modes), band mask 20 deg, "
                               "per-ring means, batch %d maps/step/GPU, %s synthesis" % (L, R, nphi, P, B, prec),
                   "lmax": L, "nrings": R, "nphi": nphi, "P": P, "n_quad": plan.n_quad, "batch_per_gpu": B,
                   "precision": prec, "l2": "inputs and intermediates > L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clocks.summary(),
        "gpu_launches": int(sum(n for (_, n) in prof0.values())),
        "e2e": {"value": round(job_throughput(B, K, world, e2e_ms), 3), "unit": "maps/s",
                "h2d_bytes_per_step": int(alm.numel() * 8), "d2h_bytes_per_step": int(tau.numel() * 8)},
        "roofline": roof,
        "stage_ms_per_step": {k: round(v[0] / n_prof, 3) for k, v in prof.items() if v[1]},
    }
    if rank == 0 and world == 1 and not args.no_baseline:
        result["cpu_baseline"] = cpu_baseline_trispectrum(args.cpu_rings)
    if rank == 0:
        print(json.dumps(result))
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline_trispectrum(nring_sample, seed=71):
    """The oracle's synthesis and quartic_tau (with ring means of the same rings) for one
    map at l_max = 2000 on `nring_sample` rings, extrapolated by ring count."""
    import simgen
    from oracle import modal as om, sht as osh

    L, R, nphi, P = WORKLOAD["lmax"], WORKLOAD["nrings"], WORKLOAD["nphi"], WORKLOAD["P"]
    cl = simgen.cl_model(L)
    filt = osh.filter_table(simgen.shifted_legendre_basis(L, P), cl)
    a = simgen.gaussian_alm(cl, 1, seed=seed)[0]
    mu, w = osh.gl_nodes(R)
    rings = np.unique(np.linspace(0, R // 2, nring_sample).astype(int))
    t0 = time.perf_counter()
    maps = osh.synthesize(a, L, filt, mu[rings], nphi)
    om.quartic_tau(maps, om.pixel_weights(w[rings], nphi), om.ring_pair_means(om.pair_means([maps])))
    dt = time.perf_counter() - t0
    return {"value": round(len(rings) / (dt * R), 8), "unit": "maps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "1 map at lmax=2000 (P=16, 3876 quartic modes) on %d of 2001 rings: synthesis and quartic "
                      "modes with the Monte Carlo terms; %.1f s, extrapolated by ring count" % (len(rings), dt)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_step_sample(2)
    total, per_maps = 0.0, []
    for _ in range(args.steps):
        dt, per_map, k, _ = oracle_step_sample(args.cpu_rings)
        total += dt
        per_maps.append(per_map)
    per_map = float(np.mean(per_maps))
    value = 1.0 / per_map
    sample = ("1 map per step at lmax=2000 (P=16, 4096 longitudes) on %d of 2001 rings, extrapolated by ring "
              "count" % k)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": "maps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "lmax=2000 GL 2001x4096, P=16 (n_max=816), FP64 CPU oracle", "lmax": 2000,
                   "nrings": 2001, "nphi": 4096, "P": 16},
        "cpu_baseline": {"value": round(value, 8), "unit": "maps/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 8), "unit": "maps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mixed":
        run_mixed(args)
    elif args.workload == "trispectrum":
        run_trispectrum(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
