"""Differentiable composite solve: a torch.autograd.Function whose backward is the adjoint
solve with the transposed composite operator (amr_solve_transpose).  No iterate is stored:
the backward runs its own V-cycles on A^T.

    phi = AmrSolve.apply(f, op, params)      # A phi = f  (valid cells; invalid = averages)
    loss(phi).backward()                     # f.grad = A^{-T} E^T dloss/dphi  (valid cells)

Only the valid and invalid interior cells of phi carry gradient; ghost entries of the
incoming gradient are ignored.  The operator must be non-singular (not the pure-Neumann
PPE).
"""
import torch

from . import amr


class AmrSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, op, params=None):
        p = params or amr.default_params(rtol=1e-12, max_vcycles=200, use_graph=1)
        phi = torch.zeros_like(f)
        op.solve(phi, f.detach().contiguous(), params=p)
        ctx.op = op
        ctx.params = p
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        p = amr.default_params(rtol=ctx.params.rtol, max_vcycles=ctx.params.max_vcycles,
                               precision=ctx.params.precision)
        lam = torch.zeros_like(grad_phi)
        ctx.op.solve_transpose(lam, grad_phi.contiguous(), params=p)
        return lam, None, None


def solve(f, op, params=None):
    return AmrSolve.apply(f, op, params)
