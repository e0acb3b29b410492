"""torch.autograd.Function around the HDG solve: lambda = A(kappa)^-1 b(kappa, f).

forward:  builds the solver for kappa = exp(log_kappa) (hdg_setup), forms the
          condensed right-hand side (hdg_condense_rhs) and solves with
          multigrid-preconditioned CG (hdg_solve).
backward: for an upstream gradient g = dL/dlambda, the adjoint solve
          A psi = g reuses the same multigrid CG (A is symmetric) inside
          hdg_adjoint_grad, which returns dL/dlog(kappa) per element and dL/df at
          the source sample points. hdg_adjoint_grad differentiates
          J = 1/2 |lambda - lambda_obs|^2; with lambda_obs = lambda - g its
          gradient is exactly the chain rule for g.
All device work happens in the CUDA library; torch holds the tensors.
"""
import torch

from . import hdg


class HDGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_kappa, f_q, nx, ny, k, rtol, maxit, options):
        opts = dict(options or {})
        solver = hdg.HDGSolver(nx, ny, k, torch.exp(log_kappa.detach()).contiguous(), **opts)
        f_d = f_q.detach().to(torch.float64).contiguous()
        b = solver.condense_rhs(f_d)
        lam, info = solver.solve(b, rtol=rtol, maxit=maxit)
        # the solver lives as long as the autograd node (its context is released
        # when the node is freed), so a graph kept with retain_graph=True can be
        # differentiated more than once
        ctx.solver = solver
        ctx.rtol, ctx.maxit = rtol, maxit
        ctx.dtypes = (log_kappa.dtype, f_q.dtype)
        ctx.save_for_backward(f_d, lam)
        return lam

    @staticmethod
    def backward(ctx, g):
        f_d, lam = ctx.saved_tensors
        solver = ctx.solver
        lam_obs = (lam - g.to(torch.float64)).contiguous()
        _, dth, df, _ = solver.adjoint_grad(f_d, lam, lam_obs, rtol=ctx.rtol, maxit=ctx.maxit)
        dth = dth.to(ctx.dtypes[0])
        df = df.to(ctx.dtypes[1])
        return dth, df, None, None, None, None, None, None


def hdg_solve(log_kappa, f_q, nx, ny, k, rtol=1e-12, maxit=300, **options):
    """Differentiable trace solve: returns lambda [n_edges*(k+1)] (float64, CUDA)."""
    return HDGSolve.apply(log_kappa, f_q, nx, ny, k, rtol, maxit, options)
