"""torch.autograd bindings of the production rates.

``KxRates.apply(mech, T, p, Y)`` returns wdot[N_s, n] from the float64
kernel; its backward calls the hand-written adjoint kernel
(kx_production_rates_vjp) for d/dT and d/dY at fixed p, the quantity an
implicit stiff integrator needs for Newton iterations (Jacobian-vector
products).  ``jacobian`` assembles the dense d wdot/d(T, Y) of every point
from N_s adjoint calls with unit cotangents.
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


def jacobian(mech: Mechanism, T, p, Y):
    """Dense Jacobian J[n, N_s, 1 + N_s]: J[i, k, 0] = d wdot_k/dT and
    J[i, k, 1 + j] = d wdot_k/dY_j at point i, from N_s adjoint calls."""
    n, ns = T.shape[0], mech.n_species
    J = torch.empty((n, ns, 1 + ns), dtype=torch.float64, device=T.device)
    v = torch.zeros((ns, n), dtype=torch.float64, device=T.device)
    gT = torch.empty(n, dtype=torch.float64, device=T.device)
    gY = torch.empty((ns, n), dtype=torch.float64, device=T.device)
    for k in range(ns):
        v.zero_()
        v[k].fill_(1.0)
        mech.production_rates_vjp(T, p, Y, v, out=(gT, gY))
        J[:, k, 0] = gT
        J[:, k, 1:] = gY.t()
    return J
