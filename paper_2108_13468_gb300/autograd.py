"""torch.autograd.Function around blp_solve: the backward pass runs the
adjoint solve A^T lambda = dJ/du with the transposed preconditioner
(blp_solve_adjoint) and assembles the field gradients with blp_grad.
Only the forward solution u is kept for the backward pass, not the Krylov
basis.  The solver handle lives as long as the autograd graph (it is
released when the graph is), so a retained graph can run backward again."""
from __future__ import annotations

import torch

from . import Solver


class BLPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, c1, c2, r, N, eps, tol, adjoint_tol, params):
        solver = Solver(N, eps, c1.detach(), c2.detach(), r.detach(), **(params or {}))
        u, info = solver.solve(f.detach().contiguous(), tol=tol)
        ctx.solver = solver
        ctx.tol = tol if adjoint_tol is None else adjoint_tol
        ctx.save_for_backward(u)
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        solver = ctx.solver
        lam, _ = solver.solve_adjoint(gu.detach().contiguous(), tol=ctx.tol)
        g1, g2, gr = solver.grad(u, lam)
        return lam, g1, g2, gr, None, None, None, None, None
