"""torch.autograd binding of the Lennard-Jones forces and their reverse-mode derivatives.

`lj_forces(pos, eps, sigma, system, species)` returns the forces F (N x 3, float64) of
the positions `pos` under the pair parameters (eps, sigma) on a `mdgb.System`; its
backward pass calls md_forces_backward, the hand-written CUDA kernel for dL/dx, dL/deps
and dL/dsigma (pair set held fixed at the cutoff).  Argument marshalling only: every
step runs in the library.

The system holds one state: the backward pass uses the positions and parameters of the
last forward call on that system, so run backward before the next forward (as a
training step does).
"""
from __future__ import annotations

import numpy as np
import torch


class _LJForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, eps, sigma, system, species, rcut):
        system.set_params(eps.detach().cpu().double().numpy(), sigma.detach().cpu().double().numpy(), rcut)
        p = pos.detach().to(torch.float64).contiguous()
        v = torch.zeros_like(p)
        torch.cuda.current_stream(p.device).synchronize()  # the library runs on its own stream
        system.set_state(p, v, species)
        F = torch.empty_like(p)
        system.forces(out=F)
        ctx.system = system
        ctx.param_like = (eps.dtype, eps.device)
        ctx.pos_dtype = pos.dtype
        return F

    @staticmethod
    def backward(ctx, grad_f):
        g = grad_f.detach().to(torch.float64).contiguous()
        torch.cuda.current_stream(g.device).synchronize()
        gpos, ge, gs = ctx.system.forces_backward(g)
        dt, dev = ctx.param_like
        return (gpos.to(ctx.pos_dtype), torch.from_numpy(ge).to(dtype=dt, device=dev),
                torch.from_numpy(gs).to(dtype=dt, device=dev), None, None, None)


def lj_forces(pos: torch.Tensor, eps: torch.Tensor, sigma: torch.Tensor, system, species: torch.Tensor,
              rcut: np.ndarray | None = None) -> torch.Tensor:
    """Forces (N x 3, float64, on pos's device) differentiable in pos, eps and sigma.

    pos: (N, 3) CUDA tensor; eps, sigma: (n_species, n_species) symmetric tensors (any
    device); species: (N,) int32 CUDA tensor; rcut: optional cutoff table (numpy), no
    larger than the system was created with.
    """
    return _LJForces.apply(pos, eps, sigma, system, species, rcut)
