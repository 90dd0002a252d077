"""Differentiable non-local forward model and unrolled solve, for calibration.

``eikonal_forward(T, L, delta, beta, energy_keV=..., pixel=...)`` returns the
detector prediction P = sum_s M_s[f_s exp(-mu_s T)] (the transport of
arXiv 2601.22793, Eqs. 3, 5, 7 with the shift of Eq. 2) and differentiates
with respect to T, L, delta_s and beta_s through ``epr_vjp``, the library's
hand-written vector-Jacobian product.

``unrolled_solve(D, L, delta, beta, energy_keV=..., pixel=..., n_iter=...)``
returns the thickness after n_iter iterations of the non-local solve
("Iterative inversion", no early stop) and differentiates with respect to
the data D, the initial thickness T0, L, delta_s and beta_s through
``epr_solve_vjp``, the reverse pass through the unrolled iterations (with
checkpointing of the iterates every ``checkpoint_every`` iterations when
memory demands it).

Both directions run in libepr's CUDA kernels; this module only marshals
tensors.  The bilinear transport is piecewise smooth: where a mapped point
lies exactly on a pixel boundary the derivative jumps and the right
derivative is returned.  Plans are cached by grid, pixel, energies and
weights; L, delta and beta are set on the cached plan for every call
(epr_plan_set_params allocates nothing), so a calibration loop that changes
them each step reuses one plan.
"""
from __future__ import annotations

import threading
from collections import OrderedDict

import numpy as np
import torch

from . import epr

_CACHE_SIZE = 4
_plans: "OrderedDict[tuple, epr.Plan]" = OrderedDict()
_lock = threading.Lock()


def _plan(nx, ny, pixel, L, E, delta, beta, weights):
    """The cached plan of this geometry and spectrum, set to L, delta, beta."""
    key = (nx, ny, pixel, tuple(E), tuple(weights))
    with _lock:
        plan = _plans.get(key)
        if plan is None:
            plan = epr.Plan(nx, ny, pixel, L, list(E), list(delta), list(beta), list(weights))
            _plans[key] = plan
            while len(_plans) > _CACHE_SIZE:
                # a pending backward may still hold the plan: drop the cache's
                # reference only and let the last reference close it
                _plans.popitem(last=False)
        else:
            _plans.move_to_end(key)
            epr.epr_plan_set_params(plan.handle, L, delta, beta)
    return plan


def _scalars(L, delta, beta, energy_keV, weights):
    d = [float(v) for v in delta.reshape(-1).tolist()]
    b = [float(v) for v in beta.reshape(-1).tolist()]
    w = [1.0] * len(energy_keV) if weights is None else [float(v) for v in weights]
    return float(L), d, b, [float(e) for e in energy_keV], w


class EikonalForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T, L, delta, beta, energy_keV, weights, pixel):
        if not (T.is_cuda and T.dtype == torch.float32):
            raise ValueError("T must be a float32 CUDA tensor")
        Tc = T.contiguous()
        squeeze = Tc.dim() == 2
        T3 = Tc.unsqueeze(0) if squeeze else Tc
        batch, ny, nx = T3.shape
        Lf, d, b, E, w = _scalars(L, delta, beta, energy_keV, weights)
        plan = _plan(nx, ny, float(pixel), Lf, E, d, b, w)
        P = torch.empty_like(T3)
        epr.epr_forward(plan.handle, T3, P, batch=batch)
        ctx.save_for_backward(T3)
        ctx.plan = plan
        ctx.meta = (squeeze, batch, len(d), L, delta, beta, Lf, d, b)
        return P.squeeze(0) if squeeze else P

    @staticmethod
    def backward(ctx, gP):
        (T3,) = ctx.saved_tensors
        squeeze, batch, ns, L, delta, beta, Lf, d, b = ctx.meta
        # the cached plan may have been set to other values since the forward
        epr.epr_plan_set_params(ctx.plan.handle, Lf, d, b)
        g = (gP.unsqueeze(0) if squeeze else gP).contiguous().to(torch.float32)
        Tbar = torch.empty_like(T3)
        db, bb, lb = epr.epr_vjp(ctx.plan.handle, T3, g, Tbar, ns, batch=batch)
        gT = Tbar.squeeze(0) if squeeze else Tbar
        gL = torch.as_tensor(lb.sum(), dtype=L.dtype, device=L.device) if torch.is_tensor(L) else None
        gd = torch.as_tensor(db.sum(0), dtype=delta.dtype, device=delta.device).reshape(delta.shape)
        gb = torch.as_tensor(bb.sum(0), dtype=beta.dtype, device=beta.device).reshape(beta.shape)
        return gT, gL, gd, gb, None, None, None


def eikonal_forward(T, L, delta, beta, *, energy_keV, pixel, weights=None):
    """Differentiable P(T; L, delta, beta).  T: [ny, nx] or [B, ny, nx] float32
    CUDA tensor; L: scalar tensor (metres); delta, beta: 1-D tensors with one
    entry per spectral line; energy_keV, weights (spectral weights, normalised
    internally) and pixel (metres) are constants."""
    if not torch.is_tensor(L):
        L = torch.tensor(float(L), dtype=torch.float64)
    delta = torch.as_tensor(delta, dtype=torch.float64) if not torch.is_tensor(delta) else delta
    beta = torch.as_tensor(beta, dtype=torch.float64) if not torch.is_tensor(beta) else beta
    E = [float(e) for e in np.atleast_1d(energy_keV)]
    return EikonalForward.apply(T, L, delta, beta, E, weights, pixel)


class UnrolledSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, T0, L, delta, beta, energy_keV, weights, pixel, n_iter, omega, eps_I,
                checkpoint_every):
        if not (D.is_cuda and D.dtype == torch.float32):
            raise ValueError("D must be a float32 CUDA tensor")
        Dc = D.contiguous()
        squeeze = Dc.dim() == 2
        D3 = Dc.unsqueeze(0) if squeeze else Dc
        batch, ny, nx = D3.shape
        T03 = None
        if T0 is not None:
            T0c = T0.contiguous().to(torch.float32)
            T03 = T0c.unsqueeze(0) if squeeze else T0c
        Lf, d, b, E, w = _scalars(L, delta, beta, energy_keV, weights)
        plan = _plan(nx, ny, float(pixel), Lf, E, d, b, w)
        T = torch.zeros_like(D3) if T03 is None else T03.clone()
        epr.epr_solve_nonlocal(plan.handle, D3, T, batch=batch, n_iter=int(n_iter), omega=omega,
                               eps_I=eps_I, init=0 if T03 is None else 1, want_info=False)
        ctx.save_for_backward(D3, T03 if T03 is not None else torch.empty(0, device=D.device))
        ctx.plan = plan
        ctx.meta = (squeeze, batch, len(d), L, delta, beta, Lf, d, b, int(n_iter), float(omega),
                    float(eps_I), int(checkpoint_every), T03 is not None)
        return T.squeeze(0) if squeeze else T

    @staticmethod
    def backward(ctx, gT):
        D3, T03 = ctx.saved_tensors
        (squeeze, batch, ns, L, delta, beta, Lf, d, b, n_iter, omega, eps_I, ck,
         has_t0) = ctx.meta
        epr.epr_plan_set_params(ctx.plan.handle, Lf, d, b)
        g = (gT.unsqueeze(0) if squeeze else gT).contiguous().to(torch.float32)
        t0b = torch.empty_like(D3)
        Db = torch.empty_like(D3)
        db, bb, lb = epr.epr_solve_vjp(ctx.plan.handle, D3, g, ns, n_iter, omega=omega,
                                       T0=T03 if has_t0 else None, eps_I=eps_I,
                                       checkpoint_every=ck, batch=batch, T0_bar=t0b, D_bar=Db)
        gD = Db.squeeze(0) if squeeze else Db
        gT0 = (t0b.squeeze(0) if squeeze else t0b) if has_t0 else None
        gL = torch.as_tensor(lb.sum(), dtype=L.dtype, device=L.device) if torch.is_tensor(L) else None
        gd = torch.as_tensor(db.sum(0), dtype=delta.dtype, device=delta.device).reshape(delta.shape)
        gb = torch.as_tensor(bb.sum(0), dtype=beta.dtype, device=beta.device).reshape(beta.shape)
        return gD, gT0, gL, gd, gb, None, None, None, None, None, None, None


def unrolled_solve(D, L, delta, beta, *, energy_keV, pixel, n_iter, omega=1.0, T0=None,
                   weights=None, eps_I=1e-8, checkpoint_every=0):
    """Differentiable tau_N(D, T0; L, delta, beta): n_iter non-local solver
    iterations from T0 (the flat field when None).  D (and T0): [ny, nx] or
    [B, ny, nx] float32 CUDA tensors; L a scalar tensor (metres); delta, beta
    1-D tensors, one entry per line.  checkpoint_every = m > 1 keeps every
    m-th iterate and recomputes the others in the backward pass."""
    if not torch.is_tensor(L):
        L = torch.tensor(float(L), dtype=torch.float64)
    delta = torch.as_tensor(delta, dtype=torch.float64) if not torch.is_tensor(delta) else delta
    beta = torch.as_tensor(beta, dtype=torch.float64) if not torch.is_tensor(beta) else beta
    E = [float(e) for e in np.atleast_1d(energy_keV)]
    return UnrolledSolve.apply(D, T0, L, delta, beta, E, weights, pixel, n_iter, omega, eps_I,
                               checkpoint_every)
