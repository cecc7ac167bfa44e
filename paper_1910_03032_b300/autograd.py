"""Differentiable solves and applies on top of the C-ABI (torch.autograd.Function).

``solve(op, alpha, nu_q, f_q)`` returns u with A_c(nu) u = P b(f), the constrained
Helmholtz system of the paper's operator (Sec. 3.1) with viscosity nu_q and load
f_q given at the quadrature points.  Its backward is the adjoint method (not in
the paper): A_c is symmetric, so one more solve A_c lam = P dL/du gives
  dL/dnu_q = -w_q detJ_q (J^-T grad lam)_q . (J^-T grad u)_q,
  dL/df_q  =  w_q detJ_q lam(x_q),
both formed by ``hx_op_gradient``.  ``apply(op, x)`` is y = A x (unconstrained,
symmetric: its backward applies A again), e.g. the mass matrix of an operator
with alpha = 1, nu = 0 for a mass-weighted loss.

Every step runs in the library's kernels; torch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import Operator


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nu_q, f_q, op, alpha, rtol, max_it):
        nu_q = nu_q.detach().contiguous()
        f_q = f_q.detach().contiguous()
        op.set_coefficients(alpha, 0.0, nu_q)
        b = op.load_vector(f_q)
        u, info = op.solve(b, rtol=rtol, max_it=max_it)
        ctx.op, ctx.alpha, ctx.rtol, ctx.max_it = op, alpha, rtol, max_it
        ctx.token = op.coef_token
        ctx.shapes = (nu_q.shape, f_q.shape)
        ctx.save_for_backward(nu_q, u)
        return u

    @staticmethod
    def backward(ctx, gu):
        nu_q, u = ctx.saved_tensors
        op = ctx.op
        if op.coef_token is not ctx.token:  # the operator was changed since the forward solve
            op.set_coefficients(ctx.alpha, 0.0, nu_q)
            ctx.token = op.coef_token
        lam, _ = op.solve(gu.detach().contiguous(), rtol=ctx.rtol, max_it=ctx.max_it)
        dnu, df = op.gradient(u, lam)
        return dnu.view(ctx.shapes[0]), df.view(ctx.shapes[1]), None, None, None, None


class _Apply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op):
        ctx.op = op
        return op.apply(x.detach().contiguous())

    @staticmethod
    def backward(ctx, gy):
        return ctx.op.apply(gy.detach().contiguous()), None


def solve(op: Operator, alpha: float, nu_q: torch.Tensor, f_q: torch.Tensor, rtol: float = 1e-12,
          max_it: int = 20000) -> torch.Tensor:
    """u = A_c(alpha, nu_q)^-1 P b(f_q); differentiable in nu_q and f_q (n_elem x q^3, FP64, CUDA)."""
    return _Solve.apply(nu_q, f_q, op, float(alpha), float(rtol), int(max_it))


def apply(op: Operator, x: torch.Tensor) -> torch.Tensor:
    """y = A x with the operator's current coefficients; differentiable in x."""
    return _Apply.apply(x, op)
