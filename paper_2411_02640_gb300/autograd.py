"""torch.autograd bindings of the production rates.

``KxRates.apply(mech, T, p, Y)`` returns wdot[N_s, n] from the float64
kernel; its backward calls the hand-written adjoint kernel
(kx_production_rates_vjp) for d/dT and d/dY at fixed p, the quantity an
implicit stiff integrator needs for Newton iterations (Jacobian-vector
products).  ``jacobian`` assembles the dense d wdot/d(T, Y) of every point
from the adjoint with unit cotangents (N_s of them per point, fused into
few calls).
"""
from __future__ import annotations

import torch

from .kx import Mechanism


class KxRates(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mech: Mechanism, T: torch.Tensor, p: torch.Tensor, Y: torch.Tensor):
        T, p, Y = T.contiguous(), p.contiguous(), Y.contiguous()
        ctx.mech = mech
        ctx.save_for_backward(T, p, Y)
        return mech.production_rates(T, p, Y)

    @staticmethod
    def backward(ctx, gw: torch.Tensor):
        T, p, Y = ctx.saved_tensors
        gT, gY = ctx.mech.production_rates_vjp(T, p, Y, gw.contiguous())
        return None, gT, None, gY


def production_rates(mech: Mechanism, T, p, Y):
    """Differentiable production rates (float64)."""
    return KxRates.apply(mech, T, p, Y)


def jacobian(mech: Mechanism, T, p, Y, max_states: int = 1 << 22):
    """Dense Jacobian J[n, N_s, 1 + N_s]: J[i, k, 0] = d wdot_k/dT and
    J[i, k, 1 + j] = d wdot_k/dY_j at point i, from the adjoint with unit
    cotangents.  The N_s adjoint evaluations of a batch are fused into as
    few calls as fit max_states states each: the states are repeated once per
    cotangent, each copy carrying its own unit cotangent (every state is
    evaluated on its own, so the result equals N_s separate calls)."""
    n, ns = T.shape[0], mech.n_species
    J = torch.empty((n, ns, 1 + ns), dtype=torch.float64, device=T.device)
    if n == 0:
        return J
    kb = max(1, min(ns, max_states // n))
    for k0 in range(0, ns, kb):
        kk = min(kb, ns - k0)
        Tb, pb, Yb = T.repeat(kk), p.repeat(kk), Y.repeat(1, kk).contiguous()
        v = torch.zeros((ns, kk * n), dtype=torch.float64, device=T.device)
        for j in range(kk):
            v[k0 + j, j * n:(j + 1) * n] = 1.0
        gT, gY = mech.production_rates_vjp(Tb, pb, Yb, v)
        J[:, k0:k0 + kk, 0] = gT.view(kk, n).t()
        J[:, k0:k0 + kk, 1:] = gY.view(ns, kk, n).permute(2, 1, 0)
    return J
