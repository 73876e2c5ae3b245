"""torch.autograd.Function over the library's energies and adjoint gradient.

``PauliEnergies.apply(theta, problem)`` returns the energy of every instance
of ``problem`` (one batched launch of ``sv_energies``); its backward pass
calls ``sv_grad_adjoint`` with the incoming gradient as the instance weights
dL/dE_i, so any torch loss built on the energies differentiates through the
hand-written reverse sweep.
"""
from __future__ import annotations

import torch

from . import Problem, sv_energies, sv_grad_adjoint


class PauliEnergies(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, problem: Problem):
        th = theta.detach().to(torch.float64).contiguous()
        _, E = sv_energies(problem, th)
        ctx.problem = problem
        ctx.save_for_backward(th)
        return E

    @staticmethod
    def backward(ctx, grad_E: torch.Tensor):
        (th,) = ctx.saved_tensors
        w = grad_E.detach().to(torch.float64).contiguous()
        _, _, g = sv_grad_adjoint(ctx.problem, th, weights=w)
        return g[: ctx.problem.n_params].to(grad_E.dtype if grad_E.is_floating_point() else th.dtype), None


def energies(theta: torch.Tensor, problem: Problem) -> torch.Tensor:
    """Differentiable per-instance energies E_i(theta)."""
    return PauliEnergies.apply(theta, problem)
