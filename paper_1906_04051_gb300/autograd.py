"""Differentiable deflated GMRES solve x = A(kappa)^-1 b for the Q1 problem.

forward:  assembles A(kappa) on the device (q1_assemble), creates the solver (T = U^T A U,
          T^-1) and solves A x = b (gmres_solve).
backward: one adjoint solve A^T lam = dL/dx with the transposed deflation preconditioner
          (gmres_adjoint_solve), then dL/db = lam and
          dL/dkappa_e = -lam^T (dA/dkappa_e) x  (q1_kappa_grad, one pass over elements).
A is affine in kappa and b does not depend on kappa, so these are the exact derivatives
of the discrete solution (up to the solver tolerance).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _native as N
from .api import Solver, q1_assemble, q1_kappa_grad


@dataclass
class Q1Setup:
    """Fixed data of the differentiable solve: mesh size, convection, deflation space and
    solver settings."""
    n: int
    beta: tuple
    agg: torch.Tensor | None = None  # int32 device tensor, (n+1)^2 entries
    r: int = 0
    m: int = 50
    tol: float = 1e-10
    maxit: int = 100000
    deflation_mode: int = N.DEFL_EBP
    ortho: int = N.ORTHO_CGS2


class GmresSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa: torch.Tensor, b: torch.Tensor, setup: Q1Setup):
        n = setup.n
        zeros_f = torch.zeros((n + 1) ** 2, dtype=torch.float64, device=kappa.device)
        rowptr, col, val, _ = q1_assemble(n, kappa.detach().contiguous(), setup.beta, zeros_f)
        solver = Solver(rowptr, col, val, setup.agg, setup.r,
                        deflation_mode=setup.deflation_mode, ortho=setup.ortho)
        x, info = solver.solve(b.detach().contiguous(), m=setup.m, tol=setup.tol,
                               maxit=setup.maxit)
        if info["status"] != N.GMRES_OK:
            raise N.GmresError(info["status"], "forward solve did not converge")
        ctx.solver = solver
        ctx.setup = setup
        ctx.info = info
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (x,) = ctx.saved_tensors
        setup = ctx.setup
        lam, info = ctx.solver.adjoint_solve(gx.detach().contiguous(), m=setup.m, tol=setup.tol,
                                             maxit=setup.maxit)
        if info["status"] != N.GMRES_OK:
            raise N.GmresError(info["status"], "adjoint solve did not converge")
        grad_kappa = q1_kappa_grad(setup.n, lam, x) if ctx.needs_input_grad[0] else None
        grad_b = lam if ctx.needs_input_grad[1] else None
        ctx.solver.close()
        ctx.solver = None
        return grad_kappa, grad_b, None


def q1_solve(kappa: torch.Tensor, b: torch.Tensor, setup: Q1Setup) -> torch.Tensor:
    """x = A(kappa)^-1 b, differentiable in kappa and b."""
    return GmresSolve.apply(kappa, b, setup)
