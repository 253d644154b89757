"""torch.autograd.Function over sim_adjoint.

:class:`EndpointProblem` holds one simulation handle, its workspace and the
adjoint workspace for a workload, targets and horizon; calling it with
``(D, lam, emit, rate_map)`` returns the scalar loss L = mean_a |p_a(T) - t_a|^2
of a no-stopping run started from the workload's initial state, differentiable
with respect to the diffusion coefficient D, the decay rate lam (0-d tensors),
the per-step source emissions ``emit`` (n_src,) and the dense rate map
``rate_map`` (field-shaped).  Every call reuses the same device buffers: the
emissions and the map are copied device to device into the handle's buffers
(nothing goes through the host but the two scalars D and lam, which the
library takes as host parameters), the state is reset from device copies of
the initial state, and only the library's kernels step the model.

When some input needs a gradient, the forward call runs sim_adjoint, which
computes the loss and all four gradients in one pass (its forward is part of
the adjoint's checkpointing), and backward scales them by the incoming
gradient; when none does, the forward runs the coupled steps and the loss
kernel only.  ``endpoint_loss(...)`` keeps one problem per (workload, device,
horizon) and calls it.
"""
from __future__ import annotations

import dataclasses

import torch

from . import cue


class EndpointProblem:
    """One reusable adjoint setup on ``device``: the workload's initial state, ``targets``
    (dim, n_axons), ``nsteps`` and checkpoint interval ``ckpt_every``."""

    def __init__(self, workload, targets, nsteps: int, ckpt_every: int = 64, device="cuda:0"):
        self.w = dataclasses.replace(workload, src_map=(workload.src_map if workload.src_map is not None
                                                        else torch.zeros(workload.shape).numpy()))
        self.nsteps, self.ckpt_every = int(nsteps), int(ckpt_every)
        self.sim = cue.Simulation(self.w, device=device)
        dev = self.sim.device
        self.device = dev
        self.targets = torch.as_tensor(targets, dtype=torch.float32, device=dev).contiguous()
        # device copies of the initial state, restored before every run
        self._C0 = self.sim.fields[0].clone()
        self._pos0, self._dir0, self._act0 = self.sim.pos.clone(), self.sim.dir.clone(), self.sim.active.clone()
        self._loss = torch.zeros((), dtype=torch.float32, device=dev)

    def _reset(self, D, lam, emit, rate_map):
        s = self.sim
        with torch.cuda.stream(s.stream):
            s.fields[0].copy_(self._C0)
            s.pos.copy_(self._pos0)
            s.dir.copy_(self._dir0)
            s.active.copy_(self._act0)
            if s.n_src:
                s.src_emit.copy_(emit.detach().reshape(-1).to(torch.float32))
            s.src_map.copy_(rate_map.detach().reshape(s.src_map.shape).to(torch.float32))
        cue._check(cue.cue_set_physics(s.h, float(D), float(lam)), "cue_set_physics")
        cue._check(cue.cue_set_state(s.h, 0, 0, 0), "cue_set_state")

    def run(self, D, lam, emit, rate_map, with_grad: bool):
        """Loss (0-d device tensor) and, with ``with_grad``, the dict of gradients."""
        s = self.sim
        self._reset(D, lam, emit, rate_map)
        if with_grad:
            g = s.adjoint(self.targets, self.nsteps, self.ckpt_every, want_map=True)
            return g["loss"], g
        s.sim_run(self.nsteps)
        cue._check(cue.cue_endpoint_loss(s.h, self.targets.data_ptr(), self._loss.data_ptr()), "cue_endpoint_loss")
        return self._loss.clone(), None

    def __call__(self, D, lam, emit, rate_map):
        return EndpointLoss.apply(D, lam, emit, rate_map, self)

    def close(self):
        self.sim.close()


class EndpointLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, lam, emit, rate_map, problem):
        need = any(ctx.needs_input_grad[:4])
        loss, g = problem.run(D, lam, emit, rate_map, with_grad=need)
        # the library works on its own stream: make the caller's stream wait for it
        torch.cuda.current_stream(problem.device).wait_stream(problem.sim.stream)
        if need:
            ctx.save_for_backward(g["dD"], g["dlambda"], g["dsrc"], g["dmap"])
        return loss.clone()

    @staticmethod
    def backward(ctx, grad):
        dD, dl, ds, dm = ctx.saved_tensors
        return grad * dD, grad * dl, grad * ds, grad * dm, None


_problems = {}


def endpoint_loss(D, lam, emit, rate_map, workload, targets, nsteps: int, ckpt_every: int = 64):
    """L for the workload's initial state after ``nsteps`` no-stopping steps; one
    :class:`EndpointProblem` per (workload, targets, device, nsteps, ckpt_every) is kept
    and reused."""
    key = (id(workload), id(targets), str(emit.device), int(nsteps), int(ckpt_every))
    entry = _problems.get(key)
    if entry is None or entry[0] is not workload or entry[1] is not targets:
        entry = (workload, targets, EndpointProblem(workload, targets, nsteps, ckpt_every, device=emit.device))
        _problems[key] = entry
    return entry[2](D, lam, emit, rate_map)
