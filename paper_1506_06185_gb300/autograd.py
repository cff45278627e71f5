"""torch.autograd wrapper of the HHG solve.

``solve(mesh, f, k, g=None, **opts)`` returns the discrete solution u of
A(k) u = f (Dirichlet values g on the boundary nodes, zero if None) as a
differentiable function of the load vector f and the per-macro coefficients
k.  The backward pass solves the adjoint problem A(k)_FF lam = dL/du_F with the
same library solve (A is symmetric, so the adjoint reuses the V-cycle
kernels) and returns dL/df = lam (zero on Dirichlet nodes) and
dL/dk_T = -lam^T A_T u (``hhg_grad_coeff``).  All arithmetic runs in the CUDA
library; this module only moves tensors.
"""

from __future__ import annotations

import numpy as np
import torch

from . import hhg as _h


def _dirichlet_mask(mesh, device):
    nz1, ny1, nx1 = mesh.shape
    z = torch.arange(nz1, device=device).view(-1, 1, 1)
    y = torch.arange(ny1, device=device).view(1, -1, 1)
    x = torch.arange(nx1, device=device).view(1, 1, -1)
    return (x == 0) | (x == nx1 - 1) | (y == 0) | (y == ny1 - 1) | (z == 0) | (z == nz1 - 1)


class HHGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, k, g, mesh, opts):
        mesh.set_coefficients(k.detach().cpu().numpy())
        u = torch.zeros(mesh.shape, dtype=torch.float64, device=f.device)
        if g is not None:
            u.copy_(g)
        mesh.set_problem(f.detach().contiguous(), u)
        mesh.solve(**opts)
        mesh.get_solution(u)
        ctx.mesh, ctx.opts = mesh, opts
        ctx.save_for_backward(u, k)
        return u

    @staticmethod
    def backward(ctx, gu):
        u, k = ctx.saved_tensors
        mesh, opts = ctx.mesh, ctx.opts
        mesh.set_coefficients(k.detach().cpu().numpy())
        mask = _dirichlet_mask(mesh, gu.device)
        rhs = gu.detach().clone().contiguous()
        rhs[mask] = 0.0
        lam = torch.zeros_like(rhs)
        mesh.set_problem(rhs, lam)
        mesh.solve(**opts)
        mesh.get_solution(lam)
        lam[mask] = 0.0
        grad_k = torch.from_numpy(mesh.grad_coeff(u.contiguous(), lam)).to(k.device, k.dtype)
        return lam, grad_k, None, None, None


def solve(mesh, f, k, g=None, **opts):
    """Differentiable solve; ``opts`` are hhg_solve options (rtol, max_cycles,
    ...), used for both the forward and the adjoint solve."""
    opts = dict(opts)
    opts.setdefault("rtol", 1e-10)
    opts.setdefault("max_cycles", 60)
    return HHGSolve.apply(f, k, g, mesh, opts)
