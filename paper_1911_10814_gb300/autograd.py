"""torch.autograd.Function around the nested solve and its adjoint.

forward(b, r) -> x = A(r)^{-1} b, with A(r) the tangent whose velocity block
carries sum_k r_k a^k a^kT (paper Sec. 2.5, K term; r_k = alpha_f gamma dt m^k).
backward(dL/dx) -> (dL/db, dL/dr) with lambda = A^{-T} dL/dx from the
transposed nested solve, dL/db = lambda and
dL/dr_k = -(lambda_v . a^k)(a^k . x_v), all computed by the library
(nbp_adjoint).  The preconditioner built by the last setup is kept when r
changes; pass resetup=True to rebuild it (S_hat depends on r through diag A).
"""
from __future__ import annotations

import numpy as np
import torch


class NestedSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, r, solver, resetup=False):
        solver.set_resistances(r.detach().to("cpu", torch.float64).numpy())
        if resetup:
            solver.setup()
        x, info = solver.solve(b.detach().contiguous())
        ctx.solver = solver
        ctx.r_meta = (r.dtype, r.device)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, dldr, _ = ctx.solver.adjoint(gx.detach().contiguous().to(torch.float64), x)
        dt, dev = ctx.r_meta
        return lam, torch.as_tensor(np.asarray(dldr), dtype=dt, device=dev), None, None


def nested_solve(b: torch.Tensor, r: torch.Tensor, solver, resetup: bool = False) -> torch.Tensor:
    """Differentiable x = A(r)^{-1} b on the solver's device."""
    return NestedSolveFn.apply(b, r, solver, resetup)


def physical_resistance_gradient(dL_dr, alpha_f_gamma_dt: float):
    """dL/dR_k from dL/dr_k, since r_k = alpha_f gamma dt R_k (resistance outlets)."""
    return alpha_f_gamma_dt * dL_dr
