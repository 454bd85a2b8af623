"""Differentiable rollouts of sphere worlds behind torch.autograd.

The loss of a rollout (squared distance of every actuated entity to its goal
after T steps) and its gradient with respect to the actions both run in the
CUDA library: vmas_diff_rollout (forward, checkpoints every `ckpt_every`
steps) and vmas_diff_backward (hand-written adjoint of the contact force,
drag and semi-implicit Euler over every substep, replaying each checkpoint
segment on chip).  This module only allocates the buffers and passes
pointers.
"""
from __future__ import annotations

import torch

from . import _lib


def _stream():
    return torch.cuda.current_stream().cuda_stream


class DiffRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, actions, world, goals, ckpt_every):
        if actions.dtype != torch.float32 or not actions.is_cuda:
            raise ValueError("actions must be a CUDA float32 tensor [T, E, A, 3]")
        actions = actions.contiguous()
        goals = goals.contiguous()
        T = int(actions.shape[0])
        E, N, A = world.n_envs, world.n_entities, world.n_actuated
        if tuple(actions.shape) != (T, E, A, 3) or tuple(goals.shape) != (E, A, 2):
            raise ValueError("actions [T, E, A, 3] and goals [E, A, 2] expected")
        nseg = max(1, -(-T // ckpt_every))
        ckpt = torch.empty((nseg, E, N, 4), dtype=torch.float32, device=actions.device)
        loss = torch.empty(E, dtype=torch.float32, device=actions.device)
        L = _lib.load()
        _lib.check(L.vmas_diff_rollout(world._handle(), actions.data_ptr(), T, goals.data_ptr(),
                                       ckpt_every, ckpt.data_ptr(), loss.data_ptr(), _stream()))
        ctx.save_for_backward(actions, goals, ckpt)
        ctx.world, ctx.ckpt_every = world, ckpt_every
        return loss

    @staticmethod
    def backward(ctx, dloss):
        actions, goals, ckpt = ctx.saved_tensors
        grad = torch.empty_like(actions)
        dloss = dloss.contiguous().float()
        L = _lib.load()
        _lib.check(L.vmas_diff_backward(ctx.world._handle(), actions.data_ptr(), actions.shape[0],
                                        goals.data_ptr(), ctx.ckpt_every, ckpt.data_ptr(),
                                        dloss.data_ptr(), grad.data_ptr(), _stream()))
        return grad, None, None, None


def rollout_loss(world, actions: torch.Tensor, goals: torch.Tensor, ckpt_every: int = 10):
    """Per-env loss [E] of a rollout from the world's current state (left
    unchanged); differentiable with respect to `actions` [T, E, A, 3]."""
    return DiffRollout.apply(actions, world, goals, ckpt_every)
