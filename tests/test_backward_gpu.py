"""GPU weight gradients (hand-written backward with per-block recomputation) against the
FP64 oracle's gradient; the oracle's gradient itself is pinned by FP64 finite differences
in test_oracle_pins.py."""
import numpy as np
import pytest
import torch

from oracle import inpaint_oracle as O
from paper_2509_10466_gb300 import binding, synthetic as S
from paper_2509_10466_gb300.config import BF16, FP32, ModelConfig, WORKLOAD_C, WORKLOAD_C_FD

from helpers import lib

pytestmark = pytest.mark.gpu

# FP32 gradients against FP64: relative L2 over the whole gradient and per tensor.
TOL_GRAD = 1e-4


def gpu_grad(cfg, weights, x, hole, gout):
    lib()
    inp = binding.Inpainter(cfg, weights)
    try:
        gw = torch.empty(S.num_params(cfg), dtype=torch.float32, device="cuda")
        binding.inpaint_backward(inp.ctx, torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda(),
                                 torch.from_numpy(gout).cuda(), gw)
        torch.cuda.synchronize()
        assert binding.inpaint_sync(inp.ctx, timeout_ms=10000) == 0
        return gw.cpu().numpy().astype(np.float64)
    finally:
        inp.close()


def compare(cfg, g, ref, tol=TOL_GRAD):
    assert np.isfinite(g).all()
    total = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    worst = []
    pos = 0
    for name, shape in S.param_shapes(cfg):
        n = int(np.prod(shape))
        r = ref[pos:pos + n]
        if np.linalg.norm(r) > 1e-8 * np.linalg.norm(ref):
            worst.append((float(np.linalg.norm(g[pos:pos + n] - r) / np.linalg.norm(r)), name))
        pos += n
    worst.sort(reverse=True)
    assert total <= tol, (total, worst[:5])
    assert worst[0][0] <= 10 * tol, worst[:5]
    return total, worst[:3]


def oracle_grad(cfg, weights, x, hole, gout):
    return O.weight_vjp(torch.from_numpy(x), torch.from_numpy(hole), torch.from_numpy(gout),
                        torch.from_numpy(weights.astype(np.float64)), cfg).numpy()


def test_backward_fd_instance_64():
    """64x64, 1 block, d32 h1: the instance whose oracle gradient is checked by finite differences."""
    w = WORKLOAD_C_FD
    weights = S.make_weights(w.model, seed=11, perturb=True)
    x = S.make_frames(1, 64, 64, seed=11)
    hole = S.make_hole(1, 64, 64, "ellipse_strokes", seed=11)
    tgt = S.make_target(1, 64, 64, seed=11)
    out = O.forward(torch.from_numpy(x), torch.from_numpy(hole), torch.from_numpy(weights.astype(np.float64)),
                    w.model)["out"]
    _, gout = O.l1_hole_loss(out, torch.from_numpy(tgt), torch.from_numpy(hole))
    gout = np.ascontiguousarray(gout.numpy(), dtype=np.float32)
    print(compare(w.model, gpu_grad(w.model, weights, x, hole, gout), oracle_grad(w.model, weights, x, hole, gout)))


@pytest.mark.parametrize("H,W,B,shift,blocks", [(64, 96, 2, 1, 2), (70, 45, 1, 1, 3), (96, 64, 2, 0, 1)])
def test_backward_small_shapes(H, W, B, shift, blocks):
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=blocks, mlp_ratio=2, shift=shift)
    weights = S.make_weights(cfg, seed=H + W, perturb=True)
    x = S.make_frames(B, H, W, seed=H)
    hole = S.make_hole(B, H, W, "large_and_thin", seed=W, area=(0.3, 0.7))
    gout = np.random.default_rng(0).standard_normal((B, 3, H, W)).astype(np.float32)
    print(compare(cfg, gpu_grad(cfg, weights, x, hole, gout), oracle_grad(cfg, weights, x, hole, gout)))


def test_backward_training_workload_256():
    """Differentiation workload: 8 frames of 256x256, d192 h6, 6 blocks, MLP ratio 4, hole-L1 gradient."""
    w = WORKLOAD_C
    weights = S.make_weights(w.model, seed=0)
    x = S.make_frames(w.batch, w.height, w.width, seed=2)
    hole = S.make_hole(w.batch, w.height, w.width, w.mask_kind, seed=2)
    tgt = S.make_target(w.batch, w.height, w.width, seed=2)
    with torch.no_grad():
        out = O.forward(torch.from_numpy(x), torch.from_numpy(hole), torch.from_numpy(weights.astype(np.float64)),
                        w.model)["out"]
    _, gout = O.l1_hole_loss(out, torch.from_numpy(tgt), torch.from_numpy(hole))
    # the oracle's gradient tensor can have permuted strides: the C ABI needs dense NCHW
    gout = np.ascontiguousarray(gout.numpy(), dtype=np.float32)
    print(compare(w.model, gpu_grad(w.model, weights, x, hole, gout), oracle_grad(w.model, weights, x, hole, gout)))


def test_backward_deterministic_and_precision_independent():
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2)
    weights = S.make_weights(cfg, seed=1, perturb=True)
    x = S.make_frames(2, 64, 64, seed=1)
    hole = S.make_hole(2, 64, 64, "polygons", seed=1)
    gout = np.random.default_rng(1).standard_normal((2, 3, 64, 64)).astype(np.float32)
    g1 = gpu_grad(cfg, weights, x, hole, gout)
    g2 = gpu_grad(cfg, weights, x, hole, gout)
    assert np.array_equal(g1, g2)
    g3 = gpu_grad(cfg.with_precision(BF16), weights, x, hole, gout)   # backward is FP32 in both forms
    assert np.array_equal(g1, g3)


def test_autograd_finetune_lowers_loss():
    from paper_2509_10466_gb300.autograd import FineTuner, HoleL1Loss, InpaintFunction
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2)
    weights = S.make_weights(cfg, seed=3)
    x = torch.from_numpy(S.make_frames(2, 64, 64, seed=3)).cuda()
    hole = torch.from_numpy(S.make_hole(2, 64, 64, "ellipse_strokes", seed=3)).cuda()
    tgt = torch.from_numpy(S.make_target(2, 64, 64, seed=3)).cuda()
    ft = FineTuner(cfg, weights, lr=1e-3)
    try:
        # autograd gradient == library backward of the library loss gradient
        out = InpaintFunction.apply(ft.weights, x, hole, ft.engine)
        loss = HoleL1Loss.apply(out, tgt, hole, ft.engine)
        loss.backward()
        g_auto = ft.weights.grad.detach().clone()
        ft.weights.grad = None
        losses = [ft.step(x, hole, tgt) for _ in range(20)]
        assert losses[-1] < 0.9 * losses[0], losses
        assert torch.isfinite(g_auto).all() and float(g_auto.abs().sum()) > 0
    finally:
        ft.close()


def test_train_step_equals_forward_loss_and_backward():
    """inpaint_train_step (forward once, in the backward's FP32-accurate form, then the hole-L1
    loss and the weight gradient) against the separate calls: the same output, loss and
    gradient within the FP32 tolerances (1e-5 relative on the output, 1e-5 on the loss,
    1e-4 on the gradient, which the separate path meets against FP64), with and without an
    output buffer."""
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, precision=FP32)
    weights = S.make_weights(cfg, seed=4, perturb=True)
    B, H, W = 2, 64, 96
    x = torch.from_numpy(S.make_frames(B, H, W, seed=4)).cuda()
    hole = torch.from_numpy(S.make_hole(B, H, W, "ellipse_strokes", seed=4)).cuda()
    tgt = torch.from_numpy(S.make_target(B, H, W, seed=4)).cuda()
    binding.load()
    inp = binding.Inpainter(cfg, weights)
    try:
        out = torch.empty_like(x)
        loss = torch.zeros(1, device="cuda")
        gout = torch.empty_like(x)
        gw = torch.empty(inp.n_params, device="cuda")
        binding.inpaint_batch(inp.ctx, x, hole, out)
        binding.inpaint_l1_hole_loss(inp.ctx, out, tgt, hole, loss, gout)
        binding.inpaint_backward(inp.ctx, x, hole, gout, gw)
        out2 = torch.empty_like(x)
        loss2 = torch.zeros(1, device="cuda")
        gw2 = torch.empty(inp.n_params, device="cuda")
        binding.inpaint_train_step(inp.ctx, x, hole, tgt, loss2, gw2, out2)
        loss3 = torch.zeros(1, device="cuda")
        gw3 = torch.empty(inp.n_params, device="cuda")
        binding.inpaint_train_step(inp.ctx, x, hole, tgt, loss3, gw3)
        torch.cuda.synchronize()
        assert float((out2 - out).norm() / out.norm()) < 1e-5
        assert abs(float(loss2) - float(loss)) <= 1e-5 * abs(float(loss))
        assert float((gw2 - gw).norm() / gw.norm()) < 1e-4
        assert torch.equal(loss2, loss3) and torch.equal(gw2, gw3)
    finally:
        inp.close()
