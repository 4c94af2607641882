"""Differentiable fixed point: V* = MB-VI solution as a torch.autograd.Function.

Forward: P = softmax(logits) per (s,a) row (``rmb_softmax_rows``), then MB-VI to V* (``rmb_vi``).
Backward: ``rmb_fixed_point_grad`` solves the adjoint system (I - gamma P_pi)^T lambda = dL/dV* by
mini-batch sweeps on the transposed greedy chain and assembles dL/dcost and dL/dlogits.  Every step
runs in librmb's kernels; torch only provides the tensors.  Gradients are those of the Bellman
equation at the greedy policy, i.e. valid away from action ties.
"""
from __future__ import annotations

import torch

from . import DeviceMDP, Opts, rmb_vi, rmb_softmax_rows, rmb_fixed_point_grad


class RmbFixedPoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cost, logits, template: DeviceMDP, opts: Opts, grad_opts: Opts):
        prob = torch.empty_like(logits)
        dm = DeviceMDP(template.n, template.m, template.gamma, "csr", cost.contiguous(),
                       row_ptr=template.row_ptr, col=template.col, prob=prob, k_uniform=template.k_uniform)
        rmb_softmax_rows(dm, logits.contiguous(), prob)
        V = torch.zeros(template.n, dtype=torch.float32, device=cost.device)
        pi = torch.empty(template.n, dtype=torch.int32, device=cost.device)
        st = rmb_vi(dm, opts, V, pi)
        ctx.dm, ctx.grad_opts, ctx.stats = dm, grad_opts, st
        ctx.save_for_backward(V, pi, prob)
        ctx.mark_non_differentiable(pi)
        return V, pi

    @staticmethod
    def backward(ctx, gV, _gpi):
        V, pi, prob = ctx.saved_tensors
        dm = ctx.dm
        w = gV.contiguous().to(torch.float32)
        lam, gc, gz, _ = rmb_fixed_point_grad(dm, pi, V, w, ctx.grad_opts)
        return gc, gz, None, None, None


def fixed_point(cost, logits, template: DeviceMDP, opts: Opts, grad_opts: Opts = None):
    """V*, pi* of the MDP with transition logits `logits` (P = row softmax) and stage costs `cost`;
    differentiable in cost and logits."""
    grad_opts = grad_opts or Opts(batch=opts.batch, seed=opts.seed, eps=1e-7, max_sweeps=100000)
    return RmbFixedPoint.apply(cost, logits, template, opts, grad_opts)
