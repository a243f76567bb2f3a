"""Differentiable frozen-field push (torch.autograd.Function over the library's adjoint).

push_adjoint(sim, state0, b0, qm, n_steps) pushes test particles through the fields the
FP64 Sim holds (frozen; steps 2-11 of Sec. 3.1 of arXiv:2511.17701, no deposit) and
returns their final state; backward() returns the gradients with respect to the initial
state and the field amplitude b0, computed by the library's reverse sweep (checkpoints
every ckpt_every steps, implicit-function theorem at the implicit substeps). Both
directions run in the library's kernels; this module only marshals arguments.

State: (6, n) float64 CUDA tensor with rows x1, x2 (absolute code coordinates), phi,
u_1, u_2, u_3 (covariant momenta per unit mass). Particles that reach the horizon layer,
the outer edge or an axis come back as NaN.
"""
from __future__ import annotations

import torch


class PushAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, state0, b0, sim, qm, n_steps, ckpt_every, n_iter):
        b0v = float(b0)
        out, ckpt = sim.adjoint_forward(state0.detach(), qm, b0v, n_steps, ckpt_every, n_iter)
        ctx.sim = sim
        ctx.args = (qm, b0v, n_steps, ckpt_every, n_iter)
        ctx.b0_like = (b0.dtype, b0.device, b0.shape)
        ctx.save_for_backward(ckpt)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (ckpt,) = ctx.saved_tensors
        qm, b0v, n_steps, ckpt_every, n_iter = ctx.args
        gin, _, gsum = ctx.sim.adjoint_backward(ckpt, grad_out, qm, b0v, n_steps, ckpt_every,
                                                n_iter)
        dtype, device, shape = ctx.b0_like
        gb0 = gsum.to(device=device, dtype=dtype).reshape(shape)
        return gin, gb0, None, None, None, None, None


def push_adjoint(sim, state0: torch.Tensor, b0, qm: float, n_steps: int, ckpt_every: int = 100,
                 n_iter: int = 64) -> torch.Tensor:
    """Final state (6, n) of the frozen-field push; differentiable in state0 and b0."""
    if not torch.is_tensor(b0):
        b0 = torch.tensor(float(b0), dtype=torch.float64)
    return PushAdjoint.apply(state0, b0, sim, float(qm), int(n_steps), int(ckpt_every),
                             int(n_iter))
