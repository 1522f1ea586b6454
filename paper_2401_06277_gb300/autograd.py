"""Differentiable Stokes solve: u(f) with a backward pass through the adjoint solve.

forward:  b = R f + lifting(u_D) (stokes_assemble_rhs), x = A^-1 b (FGMRES + V-cycle)
backward: A lambda = dL/dx with the same solver (A is symmetric), dL/df = R^T lambda
          (stokes_solve_adjoint, which also applies R^T on the device).
The Dirichlet data u_D receives no gradient.
"""
from __future__ import annotations

import torch

from . import stokes as _s


class StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, u_dirichlet: torch.Tensor, hier: "_s.Hierarchy") -> torch.Tensor:
        n = hier.n
        nq = 2 * n + 1
        b = hier.empty()
        _s.stokes_assemble_rhs(hier.handle, f.detach().contiguous(), u_dirichlet.detach().contiguous(), b, n)
        x, it, rel = hier.solve(b)
        ctx.hier = hier
        ctx.fshape = (2, nq, nq)
        return x

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        hier = ctx.hier
        lam = torch.empty_like(grad_x)
        grad_f = torch.empty(ctx.fshape, dtype=torch.float64, device=grad_x.device)
        _s.stokes_solve_adjoint(hier.handle, grad_x.contiguous(), lam, grad_f)
        return grad_f, None, None


def stokes_solve(f: torch.Tensor, u_dirichlet: torch.Tensor, hier: "_s.Hierarchy") -> torch.Tensor:
    """Solution vector x = [u_x, u_y, p] of the Stokes problem with body force f; differentiable in f."""
    return StokesSolve.apply(f, u_dirichlet, hier)
