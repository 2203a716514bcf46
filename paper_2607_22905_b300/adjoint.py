"""Differentiable TPFA pressure solve: p(ln K) with a hand-written adjoint.

Not in the paper.  forward: assemble A(ln K), f(ln K) (caller-supplied TPFA assembly),
numeric AlgMortar setup on the new values, PCG solve A p = f.  backward: the adjoint
A lambda = dL/dp by the same AlgMortar-PCG (A is symmetric), then dL/d ln K by the
library's gradient kernel (algmortar_tpfa_grad_lnK) -- dL/dA_kl = -lambda_k p_l chained
through the harmonic-mean transmissibilities and the Dirichlet half-faces.
"""
from __future__ import annotations

import torch


class AlgMortarTPFASolve(torch.autograd.Function):
    """p = AlgMortarTPFASolve.apply(lnK, solver, assemble, tol)

    lnK: CUDA float64 tensor (N,), original cell ordering.
    solver: paper_2607_22905_b300.solver.AlgMortar set up on the same sparsity pattern.
    assemble(lnK) -> (values, f, tb, tbp): CSR values of A (setup order), right-hand side,
        per-cell sums of Dirichlet half-face transmissibilities tb and of T_b p_bc (tbp);
        f may be numpy or torch.
    """

    @staticmethod
    def forward(ctx, lnK, solver, assemble, tol):
        vals, f, tb, tbp = assemble(lnK.detach())
        solver.update_values(vals)
        token = solver.values_token
        p, st = solver.solve(f, tol=tol)
        dev = lnK.device
        as_t = lambda v: torch.as_tensor(v, dtype=torch.float64, device=dev).contiguous()
        ctx.solver, ctx.tol, ctx.vals, ctx.token = solver, tol, vals, token
        ctx.stats = st
        ctx.save_for_backward(torch.exp(lnK.detach()).contiguous(), as_t(tb), as_t(tbp), p)
        return p

    @staticmethod
    def backward(ctx, g):
        K, tb, tbp, p = ctx.saved_tensors
        s = ctx.solver
        if s.values_token is not ctx.token:      # the handle was re-used for another sample
            s.update_values(ctx.vals)
        lam, st = s.solve(g.detach().to(torch.float64).contiguous(), tol=ctx.tol)
        return s.tpfa_grad_lnK(K, tb, tbp, p, lam), None, None, None
