"""torch.autograd.Function wrappers of the closure and its hand-written adjoint.

Both directions run in libfpclosure's kernels: the forward is fp_closure_exact
(or fp_closure_solve), the backward fp_closure_backward (implicit-function
transpose solve per cell, factors recomputed, then the moment-gather adjoint
down to the particle velocities).
"""

from __future__ import annotations

import torch

from . import api


class ClosureFunction(torch.autograd.Function):
    """(v, offsets, tau) -> (moments, coeffs, flags); differentiable in v."""

    @staticmethod
    def forward(ctx, v, offsets, tau, prec="fp64", params=None):
        mom, y, fl = api.fp_closure_exact(v, offsets, tau, params=params, prec=prec)
        ctx.save_for_backward(v, offsets, tau, mom, y, fl)
        ctx.params = params
        ctx.mark_non_differentiable(fl)
        return mom, y, fl

    @staticmethod
    def backward(ctx, g_mom, g_y, g_fl):
        v, offsets, tau, mom, y, fl = ctx.saved_tensors
        if g_y is None:
            g_y = torch.zeros_like(y)
        gm_in = None if g_mom is None else g_mom.contiguous()
        _, gv = api.fp_closure_backward(v, offsets, tau, mom, y, fl, g_y.contiguous(), grad_moments_in=gm_in,
                                        params=ctx.params, want_grad_moments=False,
                                        want_grad_v=ctx.needs_input_grad[0])
        return gv, None, None, None, None


class ClosureFromMomentsFunction(torch.autograd.Function):
    """(moments, tau) -> coeffs; differentiable in the moments."""

    @staticmethod
    def forward(ctx, moments, tau, prec="fp64", params=None):
        y, fl = api.fp_closure_solve(moments, tau, params=params, prec=prec)
        ctx.save_for_backward(moments, tau, y, fl)
        ctx.params = params
        return y

    @staticmethod
    def backward(ctx, g_y):
        moments, tau, y, fl = ctx.saved_tensors
        n = moments.shape[0]
        dummy_v = torch.zeros((3, 1), dtype=torch.float64, device=moments.device)
        offsets = torch.zeros(n + 1, dtype=torch.int64, device=moments.device)
        gm, _ = api.fp_closure_backward(dummy_v, offsets, tau, moments, y, fl, g_y.contiguous(), params=ctx.params,
                                        want_grad_v=False)
        return gm, None, None, None


def closure(v, offsets, tau, prec="fp64", params=None):
    return ClosureFunction.apply(v, offsets, tau, prec, params)


def closure_from_moments(moments, tau, prec="fp64", params=None):
    return ClosureFromMomentsFunction.apply(moments, tau, prec, params)
