"""torch.autograd wrapper of the hand-written adjoint.

``witness_loss(theta, profile, workload, steps)`` returns
L = -mean(E_z over the witness slab after ``steps`` steps) as a differentiable
scalar of theta = (n_b/n0, sigma_r, sigma_z) and of the radial density profile.
The forward pass records the run with sqrt(steps) checkpointing through the C
ABI (pwfa_lbm_record; ckpt_every = steps keeps the whole run as one segment
where device memory allows, and the backward pass then recomputes no
forward step) and evaluates the loss in the library
(pwfa_lbm_witness_loss); the backward pass calls the adjoint with the
built-in witness seed (pwfa_lbm_adjoint_step with a NULL seed). All
arithmetic runs in the CUDA library; this module only marshals arguments.
"""
from __future__ import annotations

import torch

from . import lbm
from . import workloads as W


class _WitnessLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, profile, workload, steps, ckpt_every):
        th = theta.detach().double().cpu().numpy()
        prof = profile.detach().double().cpu().numpy()
        w = workload.replace(alpha=float(th[0]), sigma_r=float(th[1]), sigma_z=float(th[2]), profile=prof)
        sim = lbm.Simulation(w)
        sim.record(steps, ckpt_every)
        loss = sim.witness_loss()
        ctx.sim = sim
        ctx.theta_dtype, ctx.prof_dtype = theta.dtype, profile.dtype
        return torch.tensor(loss, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        # gradient of the built-in witness loss over the recorded run
        g = ctx.sim.adjoint_step(None) * float(grad_out)
        ctx.sim.close()
        ctx.sim = None
        gt = torch.from_numpy(g[:3]).to(ctx.theta_dtype)
        gp = torch.from_numpy(g[3:]).to(ctx.prof_dtype)
        return gt, gp, None, None, None


def witness_loss(theta: torch.Tensor, profile: torch.Tensor, workload: W.Workload, steps: int,
                 ckpt_every: int = 0) -> torch.Tensor:
    """Differentiable witness-slab loss (see module docstring)."""
    return _WitnessLoss.apply(theta, profile, workload, steps, ckpt_every)
