"""torch.autograd wrapper of the K-cycle solve with a hand-written adjoint.

For the SWIP operator A(nu) of a cell-wise coefficient field, ``KCycleSolve.apply(b,
log_nu, op)`` returns u = A(nu)^{-1} b computed by kcmg_solve.  Its backward pass, given
dL/du, solves the adjoint system A^T lambda = dL/du with kcmg_solve_adjoint and returns

    dL/db       = lambda
    dL/dlog nu  = -lambda^T (dA/dlog nu_K) u          (kcmg_grad_lognu, one value per cell)

A(nu) is problem input: the operator object assembles its blocks from the coefficient
field with the problem's reference matrices and builds a fresh context for every new
field.  Everything the solve and the gradient compute runs in libkcmg's kernels.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import kcmg as K


@dataclasses.dataclass
class SolveOptions:
    rtol: float = 1e-10
    maxiter: int = 4000
    precision: str = "fp64"
    lmax: int = 200


class SWIPOperator:
    """Coefficient field -> block operator of a Cartesian SIPG problem (grid, degree,
    reference matrices and hierarchy of ``problem``)."""

    def __init__(self, problem, assemble=None, options: SolveOptions | None = None):
        if assemble is None:
            from workloads.sipg import assemble as _assemble
            assemble = _assemble
        self.pr = problem
        self._assemble = assemble
        self.options = options or SolveOptions()

    def solver(self, nu: np.ndarray):
        """A context for A(nu) (the caller closes it).  ``last_setup`` records what the new
        field cost before the solve: the host assembly of the blocks and the context's
        setup (hierarchy, inverses, coarsest factor), in seconds."""
        t0 = time.perf_counter()
        blocks, _ = self._assemble(self.pr.n, self.pr.p, self.pr.h, nu, self.pr.eta, self.pr.ref)
        t1 = time.perf_counter()
        shell = dataclasses.replace(self.pr, blocks=blocks, nu=nu)
        o = self.options
        s = K.KCycleSolver(shell, precision=o.precision, lmax=o.lmax)
        torch.cuda.synchronize()
        self.last_setup = {"assemble_s": t1 - t0, "context_s": time.perf_counter() - t1}
        return s

    def solve(self, nu, b: torch.Tensor, x0: torch.Tensor | None = None, rtol=None, atol=0.0,
              strict=True, maxiter=None):
        """u = A(nu)^{-1} b, optionally warm-started from x0.  The solve stops at
        ||b - A u|| <= max(rtol ||b - A x0||, atol); with ``strict`` a solve that ends
        without meeting it raises KcmgError, otherwise the caller reads ``last_info``."""
        s = self.solver(np.asarray(nu, dtype=np.float64))
        x = torch.zeros_like(b) if x0 is None else x0.detach().clone()
        info = K.kcmg_solve(s.ctx, b.contiguous(), x, self.options.rtol if rtol is None else rtol,
                            atol, self.options.maxiter if maxiter is None else maxiter)
        s.close()
        self.last_info = info
        if strict and info["status"] != K.KCMG_OK:
            raise K.KcmgError(info["status"], f"solve did not converge: {info['rel_res']:.2e}")
        return x


class KCycleSolve(torch.autograd.Function):
    """u = A(exp(log_nu))^{-1} b with the adjoint backward described in the module doc."""

    @staticmethod
    def forward(ctx, b, log_nu, op: SWIPOperator):
        if not (b.is_cuda and b.dtype == torch.float64):
            raise ValueError("b must be a float64 CUDA tensor")
        nu = torch.exp(log_nu.detach()).double().cpu().numpy()
        s = op.solver(nu)
        u = torch.zeros_like(b)
        info = K.kcmg_solve(s.ctx, b.contiguous(), u, op.options.rtol, 0.0, op.options.maxiter)
        if info["status"] != K.KCMG_OK:
            s.close()
            raise K.KcmgError(info["status"], f"forward solve: {info['rel_res']:.2e}")
        ctx.solver, ctx.op, ctx.nu = s, op, nu
        ctx.save_for_backward(u, log_nu)
        return u

    @staticmethod
    def backward(ctx, gu):
        u, log_nu = ctx.saved_tensors
        s, op = ctx.solver, ctx.op
        lam = torch.zeros_like(gu)
        info = K.kcmg_solve_adjoint(s.ctx, gu.contiguous().double(), lam, op.options.rtol, 0.0,
                                    op.options.maxiter)
        if info["status"] != K.KCMG_OK:
            s.close()
            raise K.KcmgError(info["status"], f"adjoint solve: {info['rel_res']:.2e}")
        ref = op.pr.ref
        nu_d = torch.from_numpy(ctx.nu).to(u.device)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(u.device)
        g = K.kcmg_grad_lognu(s.ctx, nu_d, dev(ref["V"]), dev(ref["F"]), dev(ref["B"]), lam, u)
        s.close()
        return lam, g.to(log_nu.dtype).to(log_nu.device), None
