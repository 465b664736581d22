"""Differentiable composite solve and projection: torch.autograd.Functions whose backward
passes are the adjoint maps of the library (amr_solve_transpose, amr_project_transpose).
No iterate is stored: each backward runs its own V-cycles on the transposed operator.

    phi = AmrSolve.apply(f, op, params)          # A phi = f  (valid cells; invalid = averages)
    loss(phi).backward()                         # f.grad = A^{-T} E^T dloss/dphi  (valid cells)

    u = AmrProject.apply(ppe, vel_bc, params, *w)  # u = P^comp w (Eq. comp_ProjOp)
    loss(u).backward()                           # w[d].grad = (P^T dloss/du)_d

For the pure-Neumann operator AmrSolve differentiates the whole solve map of amr_solve
(solvability correction, solve, mean zero).  Ghost entries of incoming gradients are
ignored.
"""
import torch

from . import amr


def _adjoint_params(p):
    return amr.default_params(rtol=p.rtol, max_vcycles=p.max_vcycles, precision=p.precision)


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
        lam = torch.zeros_like(grad_phi)
        ctx.op.solve_transpose(lam, grad_phi.contiguous(), params=_adjoint_params(ctx.params))
        return lam, None, None


class AmrProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ppe, vel_bc_types, params, *w):
        p = params or amr.default_params(rtol=1e-12, max_vcycles=200, use_graph=1)
        # the projection fills ghost cells of its inputs: give it copies
        wc = [x.detach().clone().contiguous() for x in w]
        u = [torch.zeros_like(x) for x in wc]
        phi = torch.zeros_like(wc[0])
        amr.project(ppe, list(vel_bc_types), wc, u, phi, params=p)
        ctx.ppe, ctx.vbc, ctx.params = ppe, list(vel_bc_types), p
        return tuple(u)

    @staticmethod
    def backward(ctx, *grad_u):
        ref = next(g for g in grad_u if g is not None)
        gu = [torch.zeros_like(ref) if g is None else g.contiguous() for g in grad_u]
        out = [torch.zeros_like(ref) for _ in gu]
        lam = torch.zeros_like(ref)
        amr.project_transpose(ctx.ppe, ctx.vbc, gu, out, lam, params=_adjoint_params(ctx.params))
        return (None, None, None) + tuple(out)


def solve(f, op, params=None):
    return AmrSolve.apply(f, op, params)


def project(ppe, vel_bc_types, w, params=None):
    return AmrProject.apply(ppe, vel_bc_types, params, *w)
