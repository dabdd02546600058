"""torch.autograd bridge of the discrete adjoint (isc_adjoint_forward /
isc_adjoint_backward).

``oil_production(sim, dts, log_k, Ea, lnA)`` returns the cumulative produced
oil mass L (kg) of the implicit-Euler loop with the frozen step sizes ``dts``
as a 0-d float64 tensor that is differentiable with respect to the per-cell
ln k multipliers and the reactions' E_a and ln A. ``forward`` runs the time
loop in libisc and keeps its checkpoints on the device (the loss only);
``backward`` runs the reverse sweep (one transposed solve per step, segments
recomputed from their checkpoints) and scales the gradient by the incoming
one. This module only moves the parameters and the gradients between torch
tensors and the C ABI. The handle must not get new parameters or options
between the two calls (the library then refuses the reverse sweep).
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
        L, info = sim.adjoint_forward(dts, checkpoint_every, tol_adjoint)
        ctx.sim = sim
        ctx.info = info
        ctx.devices = (log_k.device, Ea.device, lnA.device)
        return torch.tensor(L, dtype=torch.float64, device=log_k.device)

    @staticmethod
    def backward(ctx, gL):
        gk, ge, ga, info = ctx.sim.adjoint_backward()
        ctx.info_backward = info
        dk, de, da = ctx.devices
        g = float(gL)
        return (torch.from_numpy(g * gk).to(dk) if ctx.needs_input_grad[0] else None,
                torch.from_numpy(g * ge).to(de) if ctx.needs_input_grad[1] else None,
                torch.from_numpy(g * ga).to(da) if ctx.needs_input_grad[2] else None, None, None, None, None, None)


def oil_production(sim, dts, log_k, Ea, lnA, checkpoint_every=5, tol_adjoint=0.0, initial_state=None):
    """L(log_k, Ea, lnA) from the flash-consistent initial state of the case
    (or ``initial_state`` = (u, coke) host arrays)."""
    return CumulativeOilProduction.apply(log_k, Ea, lnA, sim, list(map(float, dts)), int(checkpoint_every),
                                         float(tol_adjoint), initial_state)
