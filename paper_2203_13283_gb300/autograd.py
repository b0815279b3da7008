"""PyTorch autograd over the solver.

solve: x = C^-1 b of Eq. (5) for a general right-hand side.  x is linear in
b, so the vector-Jacobian product is the adjoint solve: grad_b = C^-H grad_x
(PyTorch's conjugate-Wirtinger convention for a C-linear map).  Both
directions run in libwcs.so through the same skeleton and factors (Eq. 9 and
its adjoint), each refined against the exact product; the operator is fixed.

shape_objective: the far-field objective as a function of a Fourier
perturbation of the contour, with the gradient of wcs_shape_gradient."""

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


class _ShapeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, build, M, angles, phi_obs, delta):
        s = build(p.detach().cpu().numpy())
        try:
            J, g = s.shape_gradient(angles, phi_obs, M, delta)
        finally:
            s.close()
        ctx.save_for_backward(torch.as_tensor(g, dtype=p.dtype, device=p.device))
        return p.new_tensor(J)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None, None, None


def shape_objective(p, family, params, N, k, angles, phi_obs, skeleton_tol=1e-10, max_rank=0,
                    delta=1e-6, **options):
    """J(p) = sum over incidences and observation angles of |F|^2 for the
    contour `family(**params)` plus the Fourier perturbation p = (alpha_0..
    alpha_{M-1}, beta_1..beta_M) of its radial function, at fixed N and k.

    Differentiable in p: the forward pass builds and factors a solver at the
    perturbed contour and calls wcs_shape_gradient, whose gradient (adjoint
    route, in libwcs.so) the backward pass returns scaled by the incoming
    gradient.  p is a real 1-D tensor of even length 2M."""
    from .solver import Solver
    if p.dim() != 1 or p.numel() % 2:
        raise ValueError("p must be 1-D of length 2M")
    M = p.numel() // 2

    def build(pv):
        s = Solver(**options)
        s.contour(family, **params).perturb(pv[:M], pv[M:]).mesh(N, k).assemble()
        s.skeleton(skeleton_tol, max_rank=max_rank, seed=1, allow_cap=True)
        s.factor()
        return s

    return _ShapeFn.apply(p, build, M, angles, phi_obs, delta)
