"""Differentiable JFNK solve of the coefficient problem.

    u = JFNKSolve.apply(kappa, problem)

forward:  sets kappa on the problem (jfnk_set_kappa) and solves F(u; kappa) = 0
          from u0 = 0 with the inexact JFNK-MG method (jfnk_solve).
backward: with g = dL/du, solves J(u)^T lambda = g by FGMRES preconditioned by
          the multigrid cycle run on J^T with the hand-written vector-Jacobian
          product, and returns dL/dkappa = -(dF/dkappa)^T lambda
          (jfnk_adjoint_solve).  Boundary entries of g are ignored (they are not
          unknowns).

All work runs in libjfnk.so; this file only orders the calls.
"""
import torch


class JFNKSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, problem, rtol_adjoint=1e-10):
        if problem.kind != "ndk3d":
            raise ValueError("JFNKSolve differentiates the coefficient problem (ndk3d)")
        kappa64 = kappa.detach().to(problem.device, torch.float64).contiguous()
        problem.set_kappa(kappa64)
        u = torch.zeros(problem.shape(), dtype=torch.float64, device=problem.device)
        problem.solve(u)
        ctx.problem = problem
        ctx.rtol = rtol_adjoint
        ctx.save_for_backward(kappa64, u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        kappa64, u = ctx.saved_tensors
        p = ctx.problem
        p.set_kappa(kappa64)
        _, gk, _ = p.adjoint_solve(u, grad_u.to(torch.float64).contiguous(), rtol=ctx.rtol, grad=True)
        return gk, None, None


def solve(kappa, problem, rtol_adjoint=1e-10):
    return JFNKSolve.apply(kappa, problem, rtol_adjoint)
