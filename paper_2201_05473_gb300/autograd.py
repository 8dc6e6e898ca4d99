"""torch.autograd wrapper of the hand-written adjoint.

``witness_loss(theta, profile, workload, steps)`` returns
L = -mean(E_z over the witness slab after ``steps`` steps) as a differentiable
scalar of theta = (n_b/n0, sigma_r, sigma_z) and of the radial density profile.
The forward pass records the run with sqrt(steps) checkpointing through the C
ABI (pwfa_lbm_record); the backward pass seeds dL/dE on the slab and calls the
adjoint kernels (pwfa_lbm_adjoint_step). All arithmetic runs in the CUDA
library; this module only marshals arguments.
"""
from __future__ import annotations

import numpy as np
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
        k, mask = W.witness_slab(w, steps)
        ez = sim.fields(lbm.FIELD_EZ | lbm.RAW_YEE)[0, k]
        m = torch.from_numpy(mask).to(ez.device)
        loss = -(ez[m].double().sum() / float(mask.sum()))
        ctx.sim, ctx.k, ctx.mask = sim, k, mask
        ctx.shape = (3, w.nz, w.ny, w.nx)
        ctx.theta_dtype, ctx.prof_dtype = theta.dtype, profile.dtype
        return loss.to(theta.dtype).cpu()

    @staticmethod
    def backward(ctx, grad_out):
        seed = torch.zeros(ctx.shape, dtype=torch.float32, device="cuda")
        seed[2, ctx.k][torch.from_numpy(ctx.mask).cuda()] = -float(grad_out) / float(ctx.mask.sum())
        g = ctx.sim.adjoint_step(seed)
        ctx.sim.close()
        ctx.sim = None
        gt = torch.from_numpy(g[:3]).to(ctx.theta_dtype)
        gp = torch.from_numpy(g[3:]).to(ctx.prof_dtype)
        return gt, gp, None, None, None


def witness_loss(theta: torch.Tensor, profile: torch.Tensor, workload: W.Workload, steps: int,
                 ckpt_every: int = 0) -> torch.Tensor:
    """Differentiable witness-slab loss (see module docstring)."""
    return _WitnessLoss.apply(theta, profile, workload, steps, ckpt_every)
