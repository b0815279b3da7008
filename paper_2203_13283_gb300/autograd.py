"""Differentiable solve of the preconditioned system of Eq. (5) with respect
to its right-hand side.

x = C^-1 b is linear in b, so the vector-Jacobian product is the adjoint
solve: grad_b = C^-H grad_x (PyTorch's conjugate-Wirtinger convention for a
C-linear map).  Both directions run in libwcs.so through the same skeleton
and factors (Eq. 9 and its adjoint), each refined against the exact product.
The operator itself is fixed: no gradient flows to the contour."""

import torch


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, solver, allow_unconverged):
        ctx.solver = solver
        ctx.allow = allow_unconverged
        x = solver.solve(b, allow_unconverged=allow_unconverged)
        return x.contiguous() if b.dim() == 2 else x[:, 0].contiguous()

    @staticmethod
    def backward(ctx, g):
        gb = ctx.solver.solve_adjoint(g, allow_unconverged=ctx.allow)
        return (gb if g.dim() == 2 else gb[:, 0]), None, None


def solve(solver, b, allow_unconverged=False):
    """x = C^-1 b for a factored ``Solver``; b is (N,) or (N, B) complex128 on
    the solver's device.  Differentiable in b (backward = adjoint solve)."""
    if not torch.is_complex(b) or b.dtype != torch.complex128:
        raise TypeError("b must be complex128")
    return _SolveFn.apply(b, solver, allow_unconverged)
