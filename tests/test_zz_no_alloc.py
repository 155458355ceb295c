"""The allocation-free hole-L1 loss (inpaint_l1_hole_loss_noalloc) against the
context-based inpaint_l1_hole_loss.

The allocation-free form exists for callers that cannot allocate device memory while
they run (their memory belongs to another allocator, or an allocation would stall a
real-time loop); its scratch is a fixed array inside the library.  Two calls in a row
with different inputs check that the shared scratch left by the first call does not
leak into the second.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2509_10466_gb300 import binding, synthetic as S
from paper_2509_10466_gb300.config import ModelConfig

from helpers import lib

pytestmark = pytest.mark.gpu

MAX_PIXELS = 4096 * 4096


def _case(B, H, W, seed):
    out = torch.from_numpy(S.make_frames(B, H, W, seed=seed)).cuda()
    tgt = torch.from_numpy(S.make_target(B, H, W, seed=seed)).cuda()
    hole = torch.from_numpy(S.make_hole(B, H, W, "ellipse_strokes", seed=seed)).cuda()
    return out, tgt, hole


def test_noalloc_loss_matches_context_loss_twice_in_a_row():
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=1, mlp_ratio=2)
    inp = binding.Inpainter(cfg, S.make_weights(cfg))
    try:
        # a large case first, then a smaller one: the second reads fewer scratch slots
        for (B, H, W, seed) in ((4, 512, 512, 1), (2, 70, 90, 2)):
            out, tgt, hole = _case(B, H, W, seed)
            ref_loss = torch.zeros(1, device="cuda")
            ref_grad = torch.empty_like(out)
            binding.inpaint_l1_hole_loss(inp.ctx, out, tgt, hole, ref_loss, ref_grad)
            loss = torch.full((1,), float("nan"), device="cuda")
            grad = torch.full_like(out, float("nan"))
            binding.inpaint_l1_hole_loss_noalloc(out, tgt, hole, loss, grad)
            torch.cuda.synchronize()
            assert abs(float(loss) - float(ref_loss)) <= 1e-6 * abs(float(ref_loss))
            np.testing.assert_allclose(grad.cpu().numpy(), ref_grad.cpu().numpy(), rtol=1e-6, atol=0)
    finally:
        inp.close()


def _dense_case(B, H, W, seed):
    # seeded uniform frames and a random 20 % hole, drawn on the device (a full-scratch
    # case has 16.7 M pixels)
    g = torch.Generator(device="cuda").manual_seed(seed)
    out = torch.rand(B, 3, H, W, device="cuda", generator=g)
    tgt = torch.rand(B, 3, H, W, device="cuda", generator=g)
    hole = (torch.rand(B, H, W, device="cuda", generator=g) < 0.2).to(torch.uint8)
    return out, tgt, hole


@pytest.mark.parametrize("B,H,W", [(1, 4096, 4096), (4, 2048, 2048)])
def test_noalloc_loss_with_its_scratch_exactly_full(B, H, W):
    # B * H * W == INPAINT_L1_NOALLOC_MAX_PIXELS: every partial-sum slot is in use
    assert B * H * W == MAX_PIXELS
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=1, mlp_ratio=2)
    inp = binding.Inpainter(cfg, S.make_weights(cfg))
    try:
        out, tgt, hole = _dense_case(B, H, W, seed=B)
        ref_loss = torch.zeros(1, device="cuda")
        ref_grad = torch.empty_like(out)
        binding.inpaint_l1_hole_loss(inp.ctx, out, tgt, hole, ref_loss, ref_grad)
        loss = torch.full((1,), float("nan"), device="cuda")
        grad = torch.full_like(out, float("nan"))
        binding.inpaint_l1_hole_loss_noalloc(out, tgt, hole, loss, grad)
        torch.cuda.synchronize()
        assert abs(float(loss) - float(ref_loss)) <= 1e-6 * abs(float(ref_loss))
        assert torch.equal(grad, ref_grad)
    finally:
        inp.close()


def test_noalloc_loss_without_gradient_on_a_side_stream():
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=1, mlp_ratio=2)
    inp = binding.Inpainter(cfg, S.make_weights(cfg))
    try:
        out, tgt, hole = _case(3, 200, 330, seed=5)
        ref_loss = torch.zeros(1, device="cuda")
        binding.inpaint_l1_hole_loss(inp.ctx, out, tgt, hole, ref_loss, None)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            loss = torch.full((1,), float("nan"), device="cuda")
            binding.inpaint_l1_hole_loss_noalloc(out, tgt, hole, loss, None, side)
        side.synchronize()
        assert abs(float(loss) - float(ref_loss)) <= 1e-6 * abs(float(ref_loss))
    finally:
        inp.close()


def test_noalloc_loss_rejects_inputs_beyond_its_scratch():
    lib()
    dummy = torch.zeros(1, device="cuda")
    hole = torch.zeros(1, 1, 1, dtype=torch.uint8, device="cuda")
    code = binding.load().inpaint_l1_hole_loss_noalloc(
        binding._ptr(dummy), binding._ptr(dummy), binding._ptr(hole), 2, 4096, 4097, binding._ptr(dummy), None,
        binding._stream(None))
    assert code == binding.E_INVAL
    assert 2 * 4096 * 4097 > MAX_PIXELS
