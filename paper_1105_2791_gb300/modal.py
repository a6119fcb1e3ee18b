"""Tensor-level convenience over the C ABI: a Plan object and the autograd Function.

Every method forwards to one entry point of include/modal.h (argument marshalling
and output allocation only).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from . import tuning as T


class Plan:
    """Owns one modal plan (device tables, workspace, Monte Carlo accumulators)."""

    def __init__(self, lmax, P, basis, C_l, nrings, nphi, prec="fp32", ring_mask=None, pix_mask=None):
        self.h = B.modal_init(lmax, P, basis, C_l, nrings, nphi, prec, ring_mask, pix_mask)
        info = B.modal_get_info(self.h)
        self.lmax, self.P, self.nrings, self.nphi = info.lmax, info.P, info.nrings, info.nphi
        self.n_alm, self.n_max, self.n_pair, self.npix = info.n_alm, info.n_max, info.n_pair, info.npix
        self.n_quad = info.n_quad
        self.prec = info.prec
        self.linear_mode = "pixel"
        self.masked = ring_mask is not None or pix_mask is not None

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None) is not None:
            B.modal_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return B.modal_get_info(self.h)

    def set_linear_mode(self, mode):
        """"pixel" (default) or "ring": how the Monte Carlo pair means of the linear term
        are kept (clears the linear-term sums)."""
        B.modal_set_linear_mode(self.h, mode)
        self.linear_mode = mode

    # -- per-map stages
    def synthesize(self, alm, out=None):
        nb = alm.shape[0]
        if out is None:
            out = torch.empty((nb, self.P, self.nrings, self.nphi), dtype=torch.float32, device=alm.device)
        B.modal_synthesize(self.h, alm, nb, out)
        return out

    def analyze(self, maps, out=None):
        nb = maps.shape[0]
        if out is None:
            out = torch.empty((nb, self.n_alm), dtype=torch.complex64, device=maps.device)
        B.modal_analyze(self.h, maps, nb, out)
        return out

    def linear_term(self, alm_sims, finalize=False):
        nb = 0 if alm_sims is None else alm_sims.shape[0]
        B.modal_linear_term(self.h, alm_sims, nb, finalize)

    def cubic(self, alm, use_linear=False, out=None):
        nb = alm.shape[0]
        if out is None:
            out = torch.empty((nb, self.n_max), dtype=torch.float64, device=alm.device)
        B.modal_cubic(self.h, alm, nb, use_linear, out)
        return out

    def cubic_retained(self, alm, use_linear=False, out=None):
        """cubic() of the batch whose maps the last linear_term() or cubic() call kept (same
        alm tensor, set_retain_maps on): no second synthesis."""
        nb = alm.shape[0]
        if out is None:
            out = torch.empty((nb, self.n_max), dtype=torch.float64, device=alm.device)
        B.modal_cubic_retained(self.h, alm, nb, use_linear, out)
        return out

    def quartic(self, alm, use_linear=False, out=None):
        """Trispectrum modal coefficients tau [B][n_quad] float64 (modal_quartic)."""
        nb = alm.shape[0]
        if out is None:
            out = torch.empty((nb, self.n_quad), dtype=torch.float64, device=alm.device)
        B.modal_quartic(self.h, alm, nb, use_linear, out)
        return out

    def cov_accumulate(self, beta):
        B.modal_cov_accumulate(self.h, beta, beta.shape[0])

    def solve(self, alpha, beta=None):
        nb = 0 if beta is None else beta.shape[0]
        return B.modal_solve(self.h, alpha, beta, nb)

    def fnl_weights(self, alpha):
        """(w, sigma): w = d fNL / d beta = zeta^-1 alpha / (alpha^T zeta^-1 alpha), dev [n_max]
        float64, from the accumulated covariance (modal_fnl_weights)."""
        w = torch.empty(self.n_max, dtype=torch.float64, device="cuda")
        sigma = B.modal_fnl_weights(self.h, alpha, w)
        return w, sigma

    def bivector_fit(self, zeta0):
        """(bt, l1): the Monte Carlo zeta fitted as L0 (I + bt bt^T) L0^T, zeta0 = L0 L0^T."""
        return B.modal_bivector_fit(self.h, zeta0)

    def solve_bivector(self, zeta0, bt, alpha, beta=None):
        nb = 0 if beta is None else beta.shape[0]
        return B.modal_solve_bivector(self.h, zeta0, bt, alpha, beta, nb)

    def bivector_rotate(self, zeta0, bt, x, out=None):
        """Lt^-1 L0^-1 x for dev x [B][n_max] float64 (the orthonormal frame of the bivector model)."""
        if out is None:
            out = torch.empty_like(x)
        B.modal_bivector_rotate(self.h, zeta0, bt, x, x.shape[0], out)
        return out

    def backward(self, alm, g, use_linear=False, out=None):
        nb = alm.shape[0]
        if out is None:
            out = torch.empty((nb, self.n_alm), dtype=torch.complex64, device=alm.device)
        B.modal_backward(self.h, alm, nb, g, use_linear, out)
        return out

    def set_retain_maps(self, on=True):
        """Keep the maps of each cubic() call of at most one chunk of maps for
        backward_retained()."""
        B.modal_set_retain_maps(self.h, on)

    def backward_retained(self, alm, g, use_linear=False, out=None):
        """backward() of the last cubic() call (same alm tensor), from the maps it kept."""
        nb = alm.shape[0]
        if out is None:
            out = torch.empty((nb, self.n_alm), dtype=torch.complex64, device=alm.device)
        B.modal_backward_retained(self.h, alm, nb, g, use_linear, out)
        return out

    # -- host-side helpers and accumulators
    def alpha_local(self, C_signal=None):
        return B.modal_alpha_local(self.h, C_signal)

    def rings(self):
        return B.modal_get_rings(self.h)

    def pair_mean(self, device="cuda"):
        """[n_pair][npix] (pixel mode) or [n_pair][nrings] (ring mode) float32."""
        n = self.nrings if self.linear_mode == "ring" else self.npix
        out = torch.empty((self.n_pair, n), dtype=torch.float32, device=device)
        B.modal_get_pair_mean(self.h, out)
        return out

    def zeta(self):
        return B.modal_get_zeta(self.h)

    def reset(self, what=3):
        B.modal_reset(self.h, what)

    def set_chunk(self, chunk):
        B.modal_set_chunk(self.h, chunk)

    def sync(self):
        B.modal_sync(self.h)

    # -- launch shapes
    def tuning(self):
        """The plan's launch shapes (modal_get_tuning) as a dict."""
        return B.modal_get_tuning(self.h)

    def set_tuning(self, tuning):
        """Set launch shapes from a dict (modal_set_tuning; unspecified keys keep their value)."""
        cur = B.modal_get_tuning(self.h)
        cur.update({k: v for k, v in tuning.items() if k in B.TUNING_FIELDS})
        B.modal_set_tuning(self.h, cur)

    def autotune(self, alm, use_linear=False, cache=None):
        """Tune the launch shapes for coefficient passes over batches like `alm` (dev
        [B][n_alm]).  With `cache` (a JSON file path), a configuration tuned before is taken
        from the file without timing, and a new result is added to it.  Returns
        (tuning dict, "cache" or "measured")."""
        key = None
        if cache:
            key = T.tuning_key(torch.cuda.get_device_name(alm.device), self.lmax, self.P, self.nrings, self.nphi,
                               self.prec, alm.shape[0], use_linear, self.linear_mode, self.masked)
            entry = T.load(cache).get(key)
            if entry is not None and T.valid_entry(entry):
                self.set_tuning(entry)
                return dict(self.tuning(), ms=float(entry.get("ms", 0.0))), "cache"
        best = B.modal_autotune(self.h, alm, alm.shape[0], use_linear)
        if cache:
            T.store(cache, key, best)
        return best, "measured"

    def save_state(self, path):
        B.modal_save_state(self.h, path)

    def load_state(self, path):
        B.modal_load_state(self.h, path)


class ModalBeta(torch.autograd.Function):
    """beta = modal coefficients of alm (complex64 [B][n_alm]); backward through the
    library's adjoint (grad = dL/dRe a_lm + i dL/dIm a_lm, torch's convention for a
    real loss of complex inputs)."""

    @staticmethod
    def forward(ctx, alm, plan, use_linear):
        ctx.plan = plan
        ctx.use_linear = bool(use_linear)
        ctx.save_for_backward(alm)
        return plan.cubic(alm.detach().contiguous(), use_linear)

    @staticmethod
    def backward(ctx, gbeta):
        (alm,) = ctx.saved_tensors
        g = gbeta.detach().to(torch.float64).contiguous()
        return ctx.plan.backward(alm.detach().contiguous(), g, ctx.use_linear), None, None


def modal_beta(alm, plan, use_linear=False):
    return ModalBeta.apply(alm, plan, use_linear)


class ModalFnl(torch.autograd.Function):
    """fNL of each map (Eq. modalest with the plan's accumulated covariance and a shape
    alpha) as a function of its a_lm (complex64 [B][n_alm]).  fNL is linear in beta with
    d fNL / d beta = w = zeta^-1 alpha / (alpha^T zeta^-1 alpha) (modal_fnl_weights), so the
    backward is the library's adjoint with g_b = (d L / d fNL_b) w; zeta is held fixed."""

    @staticmethod
    def forward(ctx, alm, plan, alpha, use_linear):
        a = alm.detach().contiguous()
        beta = plan.cubic(a, use_linear)
        fnl, _ = plan.solve(alpha, beta)
        w, _ = plan.fnl_weights(alpha)
        ctx.plan, ctx.use_linear = plan, bool(use_linear)
        ctx.save_for_backward(alm, w)
        return torch.from_numpy(np.ascontiguousarray(fnl)).to(alm.device)

    @staticmethod
    def backward(ctx, gfnl):
        alm, w = ctx.saved_tensors
        g = (gfnl.detach().to(torch.float64)[:, None] * w[None, :]).contiguous()
        return ctx.plan.backward(alm.detach().contiguous(), g, ctx.use_linear), None, None, None


def modal_fnl(alm, plan, alpha, use_linear=True):
    return ModalFnl.apply(alm, plan, alpha, use_linear)


class Batch:
    """Plans of different l_max run as one coefficient pass (modal_batch_cubic).

    schedule: "streams" (each plan on its own stream) or "shared_cubic" (lockstep chunk
    passes with one persistent cubic launch over every plan's maps); see
    modal_batch_set_schedule.  The output tensors are owned by the batch and reused while
    the map counts stay the same, so that with graph=True the captured CUDA graph is
    replayed; copy a result to keep it past the next call."""

    def __init__(self, plans, schedule="streams"):
        self.plans = list(plans)
        self.h = B.modal_batch_create([p.h for p in self.plans])
        self._out = None
        self.set_schedule(schedule)

    def set_schedule(self, schedule):
        B.modal_batch_set_schedule(self.h, schedule)

    def close(self):
        if getattr(self, "h", None) is not None:
            B.modal_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cubic(self, alms, use_linear=False, graph=True):
        counts = [int(a.shape[0]) for a in alms]
        if self._out is None or [o.shape[0] for o in self._out] != counts:
            self._out = [torch.empty((n, p.n_max), dtype=torch.float64, device=a.device)
                         for n, p, a in zip(counts, self.plans, alms)]
        B.modal_batch_cubic(self.h, alms, counts, use_linear, self._out, graph)
        return self._out

