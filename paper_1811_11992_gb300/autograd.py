"""torch.autograd bridge of the discrete adjoint (isc_adjoint).

``oil_production(sim, dts, log_k, Ea, lnA)`` returns the cumulative produced
oil mass L (kg) of the implicit-Euler loop with the frozen step sizes ``dts``
as a 0-d float64 tensor that is differentiable with respect to the per-cell
ln k multipliers and the reactions' E_a and ln A. The time loop and its
reverse sweep run in libisc; this module only moves the parameters and the
gradients between torch tensors and the C ABI. When any input requires a
gradient, the gradient is computed together with L in the forward call (one
forward sweep plus one reverse sweep) and ``backward`` scales it.
"""
from __future__ import annotations

import numpy as np
import torch


def _host(t):
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy())


class CumulativeOilProduction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_k, Ea, lnA, sim, dts, checkpoint_every, tol_adjoint, initial_state):
        sim.set_parameters(_host(log_k), _host(Ea), _host(lnA))
        if initial_state is None:
            sim.init_equilibrium()
        else:
            u0, c0 = initial_state
            sim.set_state(u0, c0)
            sim.begin_step()
        want = any(ctx.needs_input_grad[:3])
        L, gk, ge, ga, info = sim.adjoint(dts, checkpoint_every, tol_adjoint, gradient=want)
        ctx.info = info
        if want:
            dev = log_k.device
            ctx.save_for_backward(torch.from_numpy(gk).to(dev), torch.from_numpy(ge).to(Ea.device),
                                  torch.from_numpy(ga).to(lnA.device))
        return torch.tensor(L, dtype=torch.float64, device=log_k.device)

    @staticmethod
    def backward(ctx, gL):
        gk, ge, ga = ctx.saved_tensors
        return (gL * gk if ctx.needs_input_grad[0] else None, gL * ge if ctx.needs_input_grad[1] else None,
                gL * ga if ctx.needs_input_grad[2] else None, None, None, None, None, None)


def oil_production(sim, dts, log_k, Ea, lnA, checkpoint_every=5, tol_adjoint=0.0, initial_state=None):
    """L(log_k, Ea, lnA) from the flash-consistent initial state of the case
    (or ``initial_state`` = (u, coke) host arrays)."""
    return CumulativeOilProduction.apply(log_k, Ea, lnA, sim, list(map(float, dts)), int(checkpoint_every),
                                         float(tol_adjoint), initial_state)
