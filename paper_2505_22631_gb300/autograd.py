"""torch.autograd binding of the schedule adjoint (oim_backward).

``schedule_loss(problem, K, Ks, Kn, dt, replicas, seed)`` returns the relaxed loss
L_g = mean_r E_g(theta_T) of every graph as a differentiable function of the
per-step schedules K, Ks, Kn ([graphs, steps] float32 tensors).  The forward runs
the FP32 stream form with phase checkpoints; the backward calls the library's
adjoint, which recomputes the phases between checkpoints.  Argument marshalling
only: both directions run in liboim's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from .capi import oim_backward, oim_default_opts, oim_destroy_run, oim_run, OIM_FORM_STREAM, OIM_PREC_FP32


class ScheduleLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, K, Ks, Kn, problem, dt, replicas, seed, checkpoint_every):
        G, T = K.shape
        o = oim_default_opts()
        o.form = OIM_FORM_STREAM
        o.precision = OIM_PREC_FP32
        o.checkpoint_every = int(checkpoint_every)
        o.use_graph = 0
        dev = lambda x: x.detach().to(device="cuda", dtype=torch.float32).contiguous()  # noqa: E731
        run = oim_run(problem.handle, dev(K), dev(Ks), dev(Kn), dt, T, replicas, seed, o)
        dK = np.zeros((G, T))
        dKs = np.zeros((G, T))
        dKn = np.zeros((G, T))
        loss = np.zeros(G)
        try:
            oim_backward(run, dK, dKs, dKn, loss)
        finally:
            oim_destroy_run(run)
        ctx.save_for_backward(*(torch.from_numpy(a).to(K.device, torch.float64) for a in (dK, dKs, dKn)))
        return torch.from_numpy(loss).to(K.device)

    @staticmethod
    def backward(ctx, grad_loss):
        dK, dKs, dKn = ctx.saved_tensors
        gl = grad_loss.to(torch.float64).reshape(-1, 1)
        return ((gl * dK).to(torch.float32), (gl * dKs).to(torch.float32), (gl * dKn).to(torch.float32),
                None, None, None, None, None)


def schedule_loss(problem, K, Ks, Kn, dt, replicas, seed, checkpoint_every=100):
    """Differentiable L_g for [graphs, steps] schedules (the adjoint runs eagerly in forward)."""
    return ScheduleLoss.apply(K, Ks, Kn, problem, float(dt), int(replicas), int(seed), int(checkpoint_every))
