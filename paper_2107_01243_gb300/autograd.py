"""Differentiable variable-coefficient Helmholtz solve.

x = H(h1)^{-1} b with H(h1) = mask o QQ^T (D^T (h1 G) D + h2 B) (arXiv
2107.01243 §2, Eq. 9-10).  The backward pass solves the adjoint system with
the same SPD operator, H lambda = mask o QQ^T (dL/dx), and the library's
gradient kernel returns dL/dh1 = -(D^ lambda)^T G (D^ x) at every local GLL
point.  b is treated as a constant (no gradient).
"""
import torch

from .api import sem_cg_solve, sem_dssum, sem_helmholtz_grad


class HelmholtzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h1, b, handle, h2=1.0, tol=1e-12, maxit=20000):
        x = torch.empty_like(b)
        info = sem_cg_solve(handle, b, x, h1_field=h1.contiguous(), h2=h2, tol=tol, maxit=maxit)
        ctx.handle, ctx.h2, ctx.tol, ctx.maxit = handle, h2, tol, maxit
        ctx.info = info
        ctx.save_for_backward(h1, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        h1, x = ctx.saved_tensors
        rhs = gx.contiguous().clone()
        sem_dssum(ctx.handle, rhs, apply_mask=True)
        lam = torch.empty_like(x)
        sem_cg_solve(ctx.handle, rhs, lam, h1_field=h1.contiguous(), h2=ctx.h2, tol=ctx.tol,
                     maxit=ctx.maxit)
        g = torch.empty_like(x)
        sem_helmholtz_grad(ctx.handle, x, lam, g)
        return g, None, None, None, None, None


def helmholtz_solve(h1, b, handle, h2=1.0, tol=1e-12, maxit=20000):
    """x = H(h1)^{-1} b, differentiable in h1."""
    return HelmholtzSolve.apply(h1, b, handle, h2, tol, maxit)
