"""torch.autograd.Function over sim_adjoint.

``endpoint_loss(D, lam, emit, rate_map, workload, targets, nsteps, ckpt_every)``
returns the scalar loss L = mean_a |p_a(T) - t_a|^2 of a no-stopping run started
from the workload's initial state, differentiable with respect to the
diffusion coefficient D, the decay rate lam (0-d tensors), the per-step source
emissions ``emit`` (n_src,) and the dense rate map ``rate_map`` (field-shaped).
The forward call runs the coupled simulation and its adjoint together
(sim_adjoint computes the loss and all four gradients in one pass); backward
scales the stored gradients by the incoming gradient.
"""
from __future__ import annotations

import dataclasses

import torch

from . import cue


class EndpointLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, lam, emit, rate_map, workload, targets, nsteps, ckpt_every):
        w = dataclasses.replace(workload, D=float(D), lam=float(lam),
                                src_emit=emit.detach().float().cpu().numpy(),
                                src_map=rate_map.detach().float().cpu().numpy())
        sim = cue.Simulation(w, device=emit.device)
        try:
            g = sim.adjoint(targets, int(nsteps), int(ckpt_every), want_map=True)
            torch.cuda.current_stream(emit.device).synchronize()
        finally:
            sim.close()
        ctx.save_for_backward(g["dD"], g["dlambda"], g["dsrc"], g["dmap"])
        return g["loss"].clone()

    @staticmethod
    def backward(ctx, grad):
        dD, dl, ds, dm = ctx.saved_tensors
        return grad * dD, grad * dl, grad * ds, grad * dm, None, None, None, None


def endpoint_loss(D, lam, emit, rate_map, workload, targets, nsteps: int, ckpt_every: int = 64):
    return EndpointLoss.apply(D, lam, emit, rate_map, workload, targets, nsteps, ckpt_every)
