"""torch.autograd.Function around the forward and adjoint split-step sweeps.

``SHGEfficiency.apply(plan, w0, z_focus, t_off, dT)`` returns eta (a 0-d
double tensor) computed by ``shg_propagate`` / ``shg_efficiency``; its backward
calls ``shg_propagate_adjoint`` (the reverse sweep of the exact discrete map,
with sqrt(nz) checkpoints) and returns d eta / d(w0, z_focus, T_off, dT).
Only argument marshalling happens here; both sweeps run in libshg.
"""
from __future__ import annotations

import torch

from . import (SHG_FLAG_ADJOINT, Plan, shg_propagate_adjoint, shg_set_beams, shg_beams_t)


class SHGEfficiency(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: Plan, w0, z_focus, t_off, dT):
        if not plan.flags & SHG_FLAG_ADJOINT:
            raise ValueError("the plan needs SHG_FLAG_ADJOINT (Plan(w, adjoint=True))")
        w = plan.w
        shg_set_beams(plan.handle, shg_beams_t(w.p1, float(w0), float(z_focus), float(t_off),
                                               1 if w.undepleted else 0))
        if dT is not None:
            plan.set_temperature(dT.detach().to(torch.float32), w.t_lx, w.t_ly)
        plan.propagate()
        eta, _, _ = plan.efficiency()
        ctx.plan = plan
        ctx.dT_shape = None if dT is None else tuple(dT.shape)
        ctx.dT_dtype = None if dT is None else dT.dtype
        return torch.tensor(eta, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_eta):
        plan = ctx.plan
        g_dT = None
        if ctx.dT_shape is not None:
            g_dT = torch.empty(ctx.dT_shape, dtype=torch.float32, device="cuda")
        gw, gz, gt = shg_propagate_adjoint(plan.handle, float(grad_eta), g_dT)
        dev_out = g_dT.to(ctx.dT_dtype) if g_dT is not None else None
        need = ctx.needs_input_grad  # plain-number inputs get None

        def to(i, v):
            return torch.tensor(v, dtype=torch.float64) if need[i] else None

        return None, to(1, gw), to(2, gz), to(3, gt), dev_out if need[4] else None


def efficiency(plan: Plan, w0, z_focus, t_off, dT=None):
    """eta(w0, z_focus, T_off, dT) with gradients through the adjoint sweep."""
    return SHGEfficiency.apply(plan, w0, z_focus, t_off, dT)
