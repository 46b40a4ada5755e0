"""torch.autograd wrappers of the square and cube solves.

The solve map F -> X of (3.6) is linear and self-adjoint in the Frobenius inner
product (it is a rational function of the commuting symmetric operators
Y -> A~ Y and Y -> Y A~, wrapped by the diagonal scalings of (3.9)), so the
backward pass is the same solve applied to dL/dX through ``fps_poisson_adjoint``.
The forward pass saves nothing but the plan handle.  The cube map of (5.2) is
self-adjoint for the same reason (T_01, T_02, T_12 are commuting symmetric
operators on the symmetrised tensor), so its backward is the cube solve.

With nonhomogeneous Dirichlet data (Sec. 6.1) the map (G, bc) -> U is linear but
not square; its backward is ``fps_poisson_dirichlet_adjoint``, which gives the
gradients in both the right-hand side and the boundary traces.
"""
from __future__ import annotations

import torch

from . import api


class PoissonSquareFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F: torch.Tensor, plan: api.Plan) -> torch.Tensor:
        ctx.plan = plan
        return api.poisson_square_solve(plan, F.contiguous())

    @staticmethod
    def backward(ctx, gX: torch.Tensor):
        return api.poisson_adjoint(ctx.plan, gX.contiguous()), None


def poisson_square(F: torch.Tensor, plan: api.Plan) -> torch.Tensor:
    """Differentiable X = solve(F) on the plan's device (CUDA float64 tensors)."""
    return PoissonSquareFn.apply(F, plan)


class PoissonCubeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F: torch.Tensor, plan: api.Plan) -> torch.Tensor:
        ctx.plan = plan
        return api.poisson_cube_solve(plan, F.contiguous())

    @staticmethod
    def backward(ctx, gX: torch.Tensor):
        return api.poisson_adjoint(ctx.plan, gX.contiguous()), None


def poisson_cube(F: torch.Tensor, plan: api.Plan) -> torch.Tensor:
    """Differentiable X = cube solve(F) (n x n x n CUDA float64 tensors)."""
    return PoissonCubeFn.apply(F, plan)


class PoissonDirichletFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G: torch.Tensor, bc: torch.Tensor, plan: api.Plan) -> torch.Tensor:
        ctx.plan = plan
        return api.poisson_dirichlet_solve(plan, G.contiguous(), bc.contiguous())

    @staticmethod
    def backward(ctx, gU: torch.Tensor):
        gG, gbc = api.poisson_dirichlet_adjoint(ctx.plan, gU.contiguous())
        return gG, gbc, None


def poisson_dirichlet(G: torch.Tensor, bc: torch.Tensor, plan: api.Plan) -> torch.Tensor:
    """Differentiable U = Dirichlet solve(G, bc): Legendre coefficients in and out,
    gradients in G and in the boundary traces bc."""
    return PoissonDirichletFn.apply(G, bc, plan)
