"""torch.autograd wrappers for fine-tuning the inpainter on the hole-L1 loss.

The forward pass and the weight gradient both run in the library (inpaint_batch and
inpaint_backward); the hole-L1 loss and its gradient too (inpaint_l1_hole_loss).  torch
only holds the weight tensor, the optimizer state and the streams.
"""
from __future__ import annotations

import torch

from . import binding


class InpaintFunction(torch.autograd.Function):
    """out = inpaint(weights; x, hole).  Gradient flows to `weights` only (frames and
    masks are data); the hole mask is an integer input and carries none."""

    @staticmethod
    def forward(ctx, weights, x, hole, engine):
        binding.inpaint_set_weights(engine.ctx, weights.detach())
        out = torch.empty_like(x)
        binding.inpaint_batch(engine.ctx, x, hole, out)
        ctx.engine = engine
        ctx.save_for_backward(x, hole)
        ctx.n = weights.numel()
        return out

    @staticmethod
    def backward(ctx, grad_out):
        x, hole = ctx.saved_tensors
        gw = torch.empty(ctx.n, dtype=torch.float32, device=x.device)
        binding.inpaint_backward(ctx.engine.ctx, x, hole, grad_out.contiguous(), gw)
        return gw, None, None, None


class HoleL1Loss(torch.autograd.Function):
    """Mean absolute error over hole pixels (sum / (3 * n_hole)); gradient sign / (3 n_hole)."""

    @staticmethod
    def forward(ctx, out, target, hole, engine):
        loss = torch.zeros(1, dtype=torch.float32, device=out.device)
        grad = torch.empty_like(out)
        binding.inpaint_l1_hole_loss(engine.ctx, out.contiguous(), target.contiguous(), hole, loss, grad)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None, None


class FineTuner:
    """Weights as a trainable CUDA tensor + a library context that runs the passes."""

    def __init__(self, cfg, weights_np, lr: float = 1e-4, optimizer: str = "adam"):
        self.engine = binding.Inpainter(cfg, weights_np)
        self.weights = torch.nn.Parameter(torch.from_numpy(weights_np).float().cuda())
        if optimizer == "adam":
            self.opt = torch.optim.Adam([self.weights], lr=lr)
        else:
            self.opt = torch.optim.SGD([self.weights], lr=lr)

    def step(self, x, hole, target) -> float:
        self.opt.zero_grad(set_to_none=True)
        out = InpaintFunction.apply(self.weights, x, hole, self.engine)
        loss = HoleL1Loss.apply(out, target, hole, self.engine)
        loss.backward()
        self.opt.step()
        return float(loss.detach())

    def close(self):
        self.engine.close()
