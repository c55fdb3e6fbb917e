"""Differentiation through the multilevel-preconditioned solve.

u = A(vals)^{-1} b.  For a loss L(u) with g = dL/du, the adjoint lam solves A lam = g (A is
symmetric, so the forward hierarchy serves), and
    dL/db    = lam
    dL/dvals = -lam_i u_j  on every stored entry (i, j)      (sampled outer product)
Both the adjoint solve and the sampled outer product run in libr3mg.  When the matrix values
change, the hierarchy's numeric part (Galerkin levels, smoother intervals, coarsest factor) is
rebuilt from the new values rather than stored per value set.
"""
from __future__ import annotations

import torch

from .solver import Hierarchy


class R3MGSolver:
    """A hierarchy bound to one sparsity pattern; solve(vals, b) is differentiable in vals and b."""

    def __init__(self, coords, rowptr, colidx, vals, rtol: float = 1e-10, maxit: int = 500, **params):
        self.H = Hierarchy(coords, rowptr, colidx, vals, **params)
        self.rtol, self.maxit = rtol, maxit
        self._vals_ref = None            # the values the hierarchy was last built from
        self.rebuilds = 0

    def ensure_values(self, vals: torch.Tensor):
        """Rebuild the numeric hierarchy if vals differ from the ones it was built from."""
        v = vals.detach()
        if self._vals_ref is None or self._vals_ref.shape != v.shape or not torch.equal(self._vals_ref, v):
            self.H.update_values(v.contiguous())
            self._vals_ref = v.clone()
            self.rebuilds += 1

    def solve(self, vals: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        return R3MGSolve.apply(vals, b, self)


class R3MGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, solver: R3MGSolver):
        solver.ensure_values(vals)
        u, it, rel = solver.H.pcg(b.detach().contiguous(), rtol=solver.rtol, maxit=solver.maxit)
        ctx.solver = solver
        ctx.save_for_backward(vals, u)
        ctx.forward_iterations = it
        return u

    @staticmethod
    def backward(ctx, g):
        vals, u = ctx.saved_tensors
        solver = ctx.solver
        solver.ensure_values(vals)
        lam, it, rel = solver.H.pcg(g.detach().contiguous(), rtol=solver.rtol, maxit=solver.maxit)
        grad_vals = solver.H.sampled_outer(lam, u, alpha=-1.0) if ctx.needs_input_grad[0] else None
        grad_b = lam if ctx.needs_input_grad[1] else None
        return grad_vals, grad_b, None


def solve(solver: R3MGSolver, vals: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return R3MGSolve.apply(vals, b, solver)
