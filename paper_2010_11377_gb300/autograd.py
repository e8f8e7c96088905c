"""torch.autograd.Function wrappers of the IRK time loop and its discrete
adjoint (marshalling only: forward and backward run in libirk).

    uN = IRKTrajectory.apply(u0, kappa, solver, nsteps, ckpt_every)
    L  = MassMisfit.apply(uN - d, solver)          # 1/2 e^T M e

Forward: irk_set_kappa (F = sum_e kappa_e K_e re-assembled on the GPU, AMG
hierarchies rebuilt) and irk_run storing u every `ckpt_every` steps.
Backward: irk_adjoint_run recomputes each segment from its checkpoint and
solves the transposed stage systems backwards, giving dL/du0 and dL/dkappa.
"""
from __future__ import annotations

import torch

from . import binding as B


class Solver:
    """A heat-problem context with its mesh, for the autograd functions."""

    def __init__(self, ctx: B.Context):
        if ctx.n_tri == 0:
            raise ValueError("the context needs the mesh (irk_setup mesh=...)")
        self.ctx = ctx
        self.kappa_tag = None

    def set_kappa(self, kappa: torch.Tensor):
        tag = (kappa.data_ptr(), kappa._version)
        if tag != self.kappa_tag:
            B.irk_set_kappa(self.ctx, kappa.detach().contiguous())
            self.kappa_tag = tag


class IRKTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(fctx, u0, kappa, solver: Solver, nsteps: int, ckpt_every: int):
        kappa_c = kappa.detach().contiguous()
        solver.set_kappa(kappa_c)
        n = solver.ctx.n
        nck = (nsteps + ckpt_every - 1) // ckpt_every
        ck = torch.empty(nck, n, dtype=torch.float64, device=u0.device)
        uN = torch.empty(n, dtype=torch.float64, device=u0.device)
        B.irk_run(solver.ctx, u0.detach().contiguous(), nsteps, uN, ckpt=ck, ckpt_every=ckpt_every)
        fctx.solver = solver
        fctx.nsteps = nsteps
        fctx.every = ckpt_every
        fctx.save_for_backward(ck, kappa_c)
        return uN

    @staticmethod
    def backward(fctx, grad_uN):
        ck, kappa_c = fctx.saved_tensors
        solver = fctx.solver
        solver.set_kappa(kappa_c)
        lam = grad_uN.detach().contiguous().clone()
        gk = torch.zeros(solver.ctx.n_tri, dtype=torch.float64, device=lam.device)
        B.irk_adjoint_run(solver.ctx, ck, fctx.nsteps, fctx.every, lam, gk)
        return lam, gk, None, None, None


class MassMisfit(torch.autograd.Function):
    """1/2 e^T M e with the context's mass matrix (M symmetric)."""

    @staticmethod
    def forward(fctx, e, solver: Solver):
        e = e.detach().contiguous()
        Me = torch.empty_like(e)
        value = torch.empty(1, dtype=torch.float64, device=e.device)
        B.irk_misfit(solver.ctx, e, torch.zeros_like(e), value, grad=Me)
        fctx.save_for_backward(Me)
        return value[0]

    @staticmethod
    def backward(fctx, g):
        (Me,) = fctx.saved_tensors
        return g * Me, None
