"""Differentiable non-local forward model for calibration.

``eikonal_forward(T, L, delta, beta, energy_keV=..., pixel=...)`` returns the
detector prediction P = sum_s M_s[f_s exp(-mu_s T)] (the transport of
arXiv 2601.22793, Eqs. 3, 5, 7 with the shift of Eq. 2) and differentiates
with respect to T, L, delta_s and beta_s through ``epr_vjp``, the library's
hand-written vector-Jacobian product.  Both directions run in libepr's CUDA
kernels; this module only marshals tensors.

The bilinear transport is piecewise smooth: where a mapped point lies
exactly on a pixel boundary the derivative jumps and the right derivative is
returned.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np
import torch

from . import epr

_CACHE_SIZE = 4
_plans: "OrderedDict[tuple, epr.Plan]" = OrderedDict()


def _plan(nx, ny, pixel, L, E, delta, beta, weights):
    key = (nx, ny, pixel, L, tuple(E), tuple(delta), tuple(beta), tuple(weights))
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
    return plan


class EikonalForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T, L, delta, beta, energy_keV, weights, pixel):
        if not (T.is_cuda and T.dtype == torch.float32):
            raise ValueError("T must be a float32 CUDA tensor")
        Tc = T.contiguous()
        squeeze = Tc.dim() == 2
        T3 = Tc.unsqueeze(0) if squeeze else Tc
        batch, ny, nx = T3.shape
        Lf = float(L)
        d = [float(v) for v in delta.reshape(-1).tolist()]
        b = [float(v) for v in beta.reshape(-1).tolist()]
        w = [1.0] * len(energy_keV) if weights is None else [float(v) for v in weights]
        plan = _plan(nx, ny, float(pixel), Lf, [float(e) for e in energy_keV], d, b, w)
        P = torch.empty_like(T3)
        epr.epr_forward(plan.handle, T3, P, batch=batch)
        ctx.save_for_backward(T3)
        ctx.plan = plan
        ctx.meta = (squeeze, batch, len(d), L, delta, beta)
        return P.squeeze(0) if squeeze else P

    @staticmethod
    def backward(ctx, gP):
        (T3,) = ctx.saved_tensors
        squeeze, batch, ns, L, delta, beta = ctx.meta
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
