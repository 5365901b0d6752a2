"""``torch.autograd.Function`` over the adjoint sweep.

``signal(solver, D, T2, kappa)`` returns S = |Z|/N at the echo as a 0-d
float64 tensor whose backward gives dS/dD_p, dS/dT2_p and dS/dkappa from the
library's hand-written adjoint sweep (``lbmbt_grad``), for microstructure
fitting.  The forward and the reverse sweep both run in the CUDA library; the
Function only moves the parameters in and the gradients out.  When no
gradient can be asked for (grad mode off, or no input requires one) the
signal comes from a plain forward run (``lbmbt_run``), without the ~4x cost
of the checkpointed adjoint.
"""
from __future__ import annotations

import torch


def _like(x):
    """(device, dtype) a gradient for input x must have."""
    return (x.device, x.dtype) if isinstance(x, torch.Tensor) else (None, None)


class SignalFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, T2, kappa, solver, checkpoint_every):
        solver.set_phases(_as_np(D), _as_np(T2))
        solver.set_permeability(float(kappa))
        g = solver.grad(checkpoint_every)
        ctx.save_for_backward(torch.as_tensor(g["dD"], dtype=torch.float64),
                              torch.as_tensor(g["dT2"], dtype=torch.float64),
                              torch.as_tensor(g["dkappa"], dtype=torch.float64))
        ctx.like = (_like(D), _like(T2), _like(kappa))
        return torch.as_tensor(g["S"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        # each gradient on its input's device and in its dtype; none for an
        # input that needs none (a plain number, or requires_grad False)
        out = []
        for need, d, (dev, dt) in zip(ctx.needs_input_grad[:3], ctx.saved_tensors, ctx.like):
            out.append((gout.to(torch.float64).cpu() * d).to(device=dev, dtype=dt) if need else None)
        return out[0], out[1], out[2], None, None


def _as_np(x):
    return torch.as_tensor(x).detach().double().cpu().numpy()


def signal(solver, D, T2, kappa, checkpoint_every=64):
    """Differentiable dMRI signal of the solver's geometry and sequence."""
    wants = torch.is_grad_enabled() and any(isinstance(x, torch.Tensor) and x.requires_grad for x in (D, T2, kappa))
    if not wants:   # forward only
        solver.set_phases(_as_np(D), _as_np(T2))
        solver.set_permeability(float(kappa))
        return torch.as_tensor(solver.run()["S"], dtype=torch.float64)
    return SignalFn.apply(D, T2, kappa, solver, checkpoint_every)
