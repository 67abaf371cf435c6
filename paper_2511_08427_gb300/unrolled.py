"""Unrolled gradient-descent reconstruction: a learnable-step iterative solver whose every step runs
through the projector and its matched adjoint (the "known operator" use of differentiable CT layers
described in Sec. 2.2 of the paper, where A and A^T sit inside a trainable network).

    x_{k+1} = x_k - alpha_k A^T (A x_k - p),   k = 0 .. K-1,   x_0 = 0 (or given)

alpha_k are trainable (initialised to 1 / (max(A 1) max(A^T 1)), which is at most 1 / ||A||^2 because
||A||^2 <= ||A||_1 ||A||_inf = max(A^T 1) max(A 1) for the non-negative system matrix, so the data
term 0.5 ||A x - p||^2 decreases at every step). Gradients reach the alphas and p through the
autograd functions of `operators` (backward of A = A^T, of A^T = A). With checkpoint=True each
iteration is recomputed in the backward pass instead of storing its intermediate sinogram and
volume (torch.utils.checkpoint), so memory stays at one iterate per step. With fused=True every
iteration is one projection and one fused adjoint update (operators.gradient_step: the residual is
formed while the adjoint reads the sinogram and the update accumulates into the iterate), and so is
its backward.
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint as tcp

from . import operators as ops


def step_bound(g: ops.Geometry, device=None) -> float:
    """1 / (max(A 1) max(A^T 1)) for geometry g: a step size that makes gradient descent on
    0.5 ||A x - p||^2 monotone."""
    dev = device or torch.device("cuda")
    ones_v = torch.ones(g.volume_shape, device=dev)
    a1 = ops.forward_project(ones_v, g).max().item()
    del ones_v
    ones_s = torch.ones(g.sinogram_shape, device=dev)
    at1 = ops.adjoint(ones_s, g).max().item()
    return 1.0 / (a1 * at1)


class UnrolledGD(torch.nn.Module):
    """K gradient-descent steps on 0.5 ||A x - p||^2 with one trainable step size per iteration."""

    def __init__(self, g: ops.Geometry, iterations: int = 10, alpha0: float | None = None, checkpoint: bool = True,
                 device=None, fused: bool = True):
        super().__init__()
        self.g = g
        self.iterations = int(iterations)
        self.checkpoint = bool(checkpoint)
        self.fused = bool(fused)
        a = step_bound(g, device) if alpha0 is None else float(alpha0)
        self.alpha = torch.nn.Parameter(torch.full((self.iterations,), a, device=device or torch.device("cuda")))

    def _step(self, x: torch.Tensor, p: torch.Tensor, k: int) -> torch.Tensor:
        if self.fused:
            return ops.gradient_step(x, p, self.alpha[k], self.g)
        r = ops.project(x, self.g) - p
        return x - self.alpha[k] * ops.project_adjoint(r, self.g)

    def forward(self, p: torch.Tensor, x0: torch.Tensor | None = None, return_all: bool = False):
        x = torch.zeros(self.g.volume_shape, device=p.device) if x0 is None else x0
        xs = []
        for k in range(self.iterations):
            if self.checkpoint and torch.is_grad_enabled():
                x = tcp.checkpoint(self._step, x, p, k, use_reentrant=False)
            else:
                x = self._step(x, p, k)
            if return_all:
                xs.append(x.detach())
        return (x, xs) if return_all else x
