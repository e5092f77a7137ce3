"""Compliances as torch.autograd.Functions.

`Compliance`: c(E) = u^T A(E) u for a fixed nodal field u.

For a fixed nodal field u the compliance is linear in the per-cell
coefficients (Eq. assembly: A = sum_K coef_K A^K / coef_K), so its gradient is
the vector of cell energies per unit coefficient, dc/dcoef_K = u_K^T (A^K /
coef_K) u_K. Both the forward value and the backward gradient come from the
adjoint kernel of libfeasm (fe_assemble_adjoint); u is treated as a constant
(no gradient with respect to u).

`SelfAdjointCompliance`: c(E) = f^T u(E) of a clamped structure, K(E) u = f on
the free DOFs. Its gradient is dc/dcoef_K = -u_K^T (A^K / coef_K) u_K; the
forward pass solves (fe_compliance) and keeps u, the backward pass evaluates
the gradient times grad_c with the adjoint kernel (grad_scale = -grad_c).
"""
from __future__ import annotations

import torch

from . import feasm


class Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef: torch.Tensor, u: torch.Tensor, space: "feasm.FESpace", prec: str = "fp64"):
        c = torch.empty(1, dtype=torch.float64, device=coef.device)
        g = torch.empty(space.n_cells, dtype=torch.float64, device=coef.device)
        feasm.fe_assemble_adjoint(space.handle, u, coef, 1.0, g, c, feasm.PRECISIONS[prec])
        ctx.space = space
        ctx.prec = prec
        ctx.save_for_backward(coef, u)
        return c[0]

    @staticmethod
    def backward(ctx, grad_c: torch.Tensor):
        coef, u = ctx.saved_tensors
        g = torch.empty(ctx.space.n_cells, dtype=torch.float64, device=coef.device)
        feasm.fe_assemble_adjoint(ctx.space.handle, u, None, float(grad_c), g, None, feasm.PRECISIONS[ctx.prec])
        return g, None, None, None


def compliance(coef: torch.Tensor, u: torch.Tensor, space: "feasm.FESpace", prec: str = "fp64") -> torch.Tensor:
    return Compliance.apply(coef, u, space, prec)


class SelfAdjointCompliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef: torch.Tensor, system: "feasm.DirichletSystem", prec: str = "fp64", rtol: float = 1e-10,
                max_iter: int = 20000):
        u, c, _, _, _ = system.compliance(coef, prec=prec, rtol=rtol, max_iter=max_iter, gradient=False)
        ctx.system = system
        ctx.prec = prec
        ctx.save_for_backward(coef, u)
        return c[0]

    @staticmethod
    def backward(ctx, grad_c: torch.Tensor):
        coef, u = ctx.saved_tensors
        space = ctx.system.space
        g = torch.empty(space.n_cells, dtype=torch.float64, device=coef.device)
        prec = "fp64" if ctx.prec == "fp64" else "fp32"
        feasm.fe_assemble_adjoint(space.handle, u, None, -float(grad_c), g, None, feasm.PRECISIONS[prec])
        return g, None, None, None, None


def self_adjoint_compliance(coef: torch.Tensor, system: "feasm.DirichletSystem", prec: str = "fp64",
                            rtol: float = 1e-10, max_iter: int = 20000) -> torch.Tensor:
    return SelfAdjointCompliance.apply(coef, system, prec, rtol, max_iter)
