"""torch.autograd front end of the differentiable run.

Both functions run rsol_gradient once in the forward pass (checkpointed
forward sweep and reverse sweep, all in librsol's kernels) and hand the
stored gradient to autograd in the backward pass, scaled by the incoming
gradient.  The loss is L = ||sum_n S^n||_2 of the deposited momentum source.

    L = momentum_source_loss_fields(ctx, parts, fields, steps, dt)
    L.backward()          # fields.grad = dL/dF (components 0..5; 6..7 zero)

    L = momentum_source_loss_amplitudes(ctx, parts, amps, modes, steps, dt, vA=..)
    L.backward()          # amps.grad = dL/dA
"""
from __future__ import annotations

import torch


class _FieldsLoss(torch.autograd.Function):
    @staticmethod
    def forward(actx, fields, context, parts, steps, dt, every):
        o = context.gradient(parts, steps, dt, checkpoint_every=every, fields=fields.detach())
        g = o["field_bar"].clone()
        g[..., 6:] = 0
        actx.save_for_backward(g)
        return o["loss"][0].clone()

    @staticmethod
    def backward(actx, gL):
        (g,) = actx.saved_tensors
        return (gL.to(g.dtype) * g, None, None, None, None, None)


class _AmplitudeLoss(torch.autograd.Function):
    @staticmethod
    def forward(actx, amps, context, parts, modes, steps, dt, every, t0, B0, vA, u_gas):
        m = dict(modes)
        m["amp"] = amps.detach().cpu().double().numpy()
        o = context.gradient(parts, steps, dt, checkpoint_every=every, modes=m, t0=t0, B0=B0,
                             vA=vA, u_gas=u_gas)
        actx.save_for_backward(o["amp_bar"].clone())
        return o["loss"][0].clone()

    @staticmethod
    def backward(actx, gL):
        (g,) = actx.saved_tensors
        return (gL * g,) + (None,) * 10


def momentum_source_loss_fields(context, parts, fields, steps: int, dt: float,
                                checkpoint_every: int = 8):
    """L over `steps` steps in the static field grid `fields` (node-major
    (nz, ny, nx, 8) tensor); differentiable with respect to `fields`."""
    return _FieldsLoss.apply(fields, context, parts, int(steps), float(dt), int(checkpoint_every))


def momentum_source_loss_amplitudes(context, parts, amps, modes: dict, steps: int, dt: float,
                                    checkpoint_every: int = 8, t0: float = 0.0, B0: float = 1.0,
                                    vA: float = 0.0, u_gas=(0.0, 0.0, 0.0)):
    """L over `steps` steps in the Alfven fields of `modes` with amplitudes
    `amps` (float64 tensor on the GPU); differentiable with respect to `amps`."""
    return _AmplitudeLoss.apply(amps, context, parts, modes, int(steps), float(dt),
                                int(checkpoint_every), float(t0), float(B0), float(vA),
                                tuple(float(x) for x in u_gas))
