"""``torch.autograd.Function`` over the adjoint sweep.

``signal(solver, D, T2, kappa)`` returns S = |Z|/N at the echo as a 0-d
float64 tensor whose backward gives dS/dD_p, dS/dT2_p and dS/dkappa from the
library's hand-written adjoint sweep (``lbmbt_grad``), for microstructure
fitting.  The forward and the reverse sweep both run in the CUDA library; the
Function only moves the parameters in and the gradients out.
"""
from __future__ import annotations

import torch


class SignalFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, T2, kappa, solver, checkpoint_every):
        solver.set_phases(D.detach().double().cpu().numpy(), T2.detach().double().cpu().numpy())
        solver.set_permeability(float(kappa))
        g = solver.grad(checkpoint_every)
        ctx.save_for_backward(torch.as_tensor(g["dD"]), torch.as_tensor(g["dT2"]),
                              torch.as_tensor(g["dkappa"], dtype=torch.float64))
        return torch.as_tensor(g["S"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        dD, dT2, dk = ctx.saved_tensors
        return gout * dD, gout * dT2, gout * dk, None, None


def signal(solver, D, T2, kappa, checkpoint_every=64):
    """Differentiable dMRI signal of the solver's geometry and sequence."""
    return SignalFn.apply(D, T2, kappa, solver, checkpoint_every)
