"""GPU parity of the CUDA path against the FP64 oracle (calls go through the C ABI)."""
import numpy as np
import pytest
import torch

from paper_2509_10466_gb300 import binding, synthetic as S
from paper_2509_10466_gb300.config import BF16, FP16, FP32, ModelConfig, WORKLOAD_A, WORKLOAD_B

from helpers import TOL_BF16, TOL_FP32, check_parity, gpu_forward, hole_rel_l2, inputs, lib, oracle_forward

pytestmark = pytest.mark.gpu


def small(precision, **kw):
    base = dict(dim=64, heads=2, window=8, blocks=3, mlp_ratio=2, precision=precision)
    base.update(kw)
    return ModelConfig(**base)


# ----------------------------------------------------------------------------- tensor-core GEMM unit

@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 256, 256), (384, 768, 256), (200, 128, 128),
                                   (1000, 1024, 256), (4096, 256, 1024), (130, 192, 320)])
def test_tcgen05_gemm_matches_fp32_matmul(M, N, K):
    lib()
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).bfloat16()
    Bt = torch.randn(N, K, generator=g).bfloat16()
    ref = A.float() @ Bt.float().T
    C = torch.full((M, N), float("nan"), device="cuda")
    binding.inpaint_test_gemm_bf16(A.cuda(), Bt.cuda(), C)
    torch.cuda.synchronize()
    got = C.cpu()
    assert torch.isfinite(got).all()
    rel = (got - ref).norm() / ref.norm()
    assert rel < 1e-5, float(rel)


def test_gelu_of_the_bf16_form_matches_erff():
    """The BF16 form's GELU, 0.5 x (1 + tanh(x P(x^2))) with the approximate hardware tanh:
    within 6e-6 + 2.5e-4 |x| of CUDA's erff GELU and of the FP64 closed form over [-12, 12]
    (the fit's error is 4.9e-6; the tanh's relative error of about 2^-11 scales with 0.5 |x|),
    which for x > 0 is 2.5e-4 relative, an eighth of the bf16 step of the output; the FP32
    form's erff GELU within 1e-6 of the closed form."""
    lib()
    x = torch.linspace(-12, 12, 200001, dtype=torch.float32)
    xd = x.cuda()
    a = torch.empty_like(xd)
    b = torch.empty_like(xd)
    binding.inpaint_test_gelu(xd, a, b)
    torch.cuda.synchronize()
    ref = 0.5 * x.double() * (1 + torch.erf(x.double() / 2 ** 0.5))
    bound = 6e-6 + 2.5e-4 * x.double().abs()
    assert bool(((a.cpu().double() - b.cpu().double()).abs() <= bound + 1e-6).all())
    assert bool(((a.cpu().double() - ref).abs() <= bound).all())
    pos = x > 0.5
    assert float(((a.cpu().double() - ref).abs() / ref.abs())[pos].max()) <= 2.6e-4
    assert float((b.cpu().double() - ref).abs().max()) <= 1e-6
    # saturation: x for large x, 0 (no NaN) for large negative x
    big = torch.tensor([-1e4, -100.0, -30.0, 30.0, 100.0, 1e4]).cuda()
    ya = torch.empty_like(big)
    yb = torch.empty_like(big)
    binding.inpaint_test_gelu(big, ya, yb)
    torch.cuda.synchronize()
    assert torch.isfinite(ya).all()
    assert torch.equal(ya.cpu()[3:], big.cpu()[3:]) and float(ya.cpu()[:3].abs().max()) == 0.0


def test_gelu_of_the_hidden_activations_in_fp16():
    """The 16-bit forms' hidden-activation GELU, the same 0.5 x (1 + tanh(x P(x^2))) in packed
    FP16 arithmetic: over [-12, 12] within 2e-3 |GELU(x)| + 1e-4 of the FP64 closed form
    for x > 0.5 (the input and each step rounded to FP16, 2^-11 relative, and the FP16
    tanh; measured 1.25e-3 relative), within 2e-3 + 1e-4 |x| absolute below (near 0 the
    output is small and the error absolute; measured 1.24e-3); every value then rounds to
    the bf16 step (2^-9 relative) or the fp16 one.  Saturation: x for large x, 0 for large
    negative x, no NaN or inf up to +-1e6."""
    lib()
    x = torch.linspace(-12, 12, 200001, dtype=torch.float32)
    y = torch.empty_like(x).cuda()
    binding.inpaint_test_gelu_h16(x.cuda(), y)
    torch.cuda.synchronize()
    yd = y.cpu().double()
    ref = 0.5 * x.double() * (1 + torch.erf(x.double() / 2 ** 0.5))
    err = (yd - ref).abs()
    pos = x > 0.5
    rel_pos = float((err[pos] / ref[pos].abs()).max())
    abs_neg = float((err[~pos] - 1e-4 * x.double().abs()[~pos]).max())
    print(f"fp16 GELU: max relative error (x > 0.5) {rel_pos:.3e}, max absolute error (x <= 0.5) "
          f"{float(err[~pos].max()):.3e}")
    assert bool((err[pos] <= 2e-3 * ref[pos].abs() + 1e-4).all()), rel_pos
    assert bool((err[~pos] <= 2e-3 + 1e-4 * x.double().abs()[~pos]).all()), abs_neg
    big = torch.tensor([-1e6, -1e4, -100.0, -30.0, 30.0, 100.0, 1e4, 1e6]).cuda()
    yb = torch.empty_like(big)
    binding.inpaint_test_gelu_h16(big, yb)
    torch.cuda.synchronize()
    yb = yb.cpu()
    assert torch.isfinite(yb).all()
    assert float(yb[:4].abs().max()) == 0.0
    assert torch.equal(yb[4:7], big.cpu()[4:7]) and float(yb[7]) == 65504.0


# ----------------------------------------------------------------------------- FP32 form

def test_fp32_plain_256_matches_oracle():
    """The plain FP32 workload: 256x256, d128 h4, 2 blocks, MLP ratio 2."""
    w = WORKLOAD_A
    weights = S.make_weights(w.model, seed=0, perturb=True)
    x, hole = inputs(w.batch, w.height, w.width, w.mask_kind, seed=0)
    check_parity(w.model, weights, x, hole, TOL_FP32)


@pytest.mark.parametrize("H,W,B,shift", [(64, 64, 1, 1), (70, 45, 2, 1), (96, 160, 3, 0), (33, 130, 1, 1)])
def test_fp32_ragged_shapes(H, W, B, shift):
    cfg = small(FP32, shift=shift)
    weights = S.make_weights(cfg, seed=H + W, perturb=True)
    x, hole = inputs(B, H, W, "ellipse_strokes", seed=H * W, area=(0.2, 0.5))
    check_parity(cfg, weights, x, hole, TOL_FP32)


def test_fp32_thin_strokes_leave_windows_empty():
    """Large holes: some windows have no valid key for several blocks."""
    cfg = small(FP32, blocks=4)
    weights = S.make_weights(cfg, seed=3, perturb=True)
    x, hole = inputs(2, 128, 128, "large_and_thin", seed=5, area=(0.4, 0.9))
    ref = oracle_forward(cfg, weights, x, hole)
    assert (ref["masks"][1] == 0).any(), "fixture should contain skipped windows"
    check_parity(cfg, weights, x, hole, TOL_FP32, ref=ref)


# ----------------------------------------------------------------------------- BF16 form

@pytest.mark.parametrize("H,W,B", [(64, 64, 1), (96, 128, 2), (70, 45, 1)])
def test_bf16_small_shapes(H, W, B):
    cfg = small(BF16)
    weights = S.make_weights(cfg, seed=11, perturb=True)
    x, hole = inputs(B, H, W, "polygons", seed=H + W)
    check_parity(cfg, weights, x, hole, TOL_BF16)


@pytest.mark.parametrize("H,W,B", [(64, 96, 2), (224, 100, 1), (96, 352, 1), (32, 64, 1)])
def test_bf16_d256_decoder_on_tensor_cores(H, W, B):
    """d256 puts both decoder stages on tcgen05 (c1 = 64, c2 = 32), with the parities
    stacked on M for inputs of at least 16 x 16 pixels; ragged tile edges.  At 32 x 64
    (8 x 16 tokens) the first stage takes the M = pixels form, the second the stacked one."""
    cfg = ModelConfig(dim=256, heads=8, window=8, blocks=2, mlp_ratio=4, precision=BF16)
    weights = S.make_weights(cfg, seed=21, perturb=True)
    x, hole = inputs(B, H, W, "polygons", seed=H * 7 + W)
    check_parity(cfg, weights, x, hole, TOL_BF16)


@pytest.mark.parametrize("dim,ratio,H,W", [(64, 4, 96, 96), (128, 4, 64, 224), (256, 2, 96, 352), (128, 8, 32, 32)])
def test_bf16_fused_mlp_odd_tile_counts(dim, ratio, H, W):
    """The fused MLP runs in CTA pairs that share weight stages: odd and partial row-tile
    counts leave one CTA of the last pair on a tile past the end (5, 7, 17 and 1 tiles)."""
    cfg = ModelConfig(dim=dim, heads=dim // 32, window=8, blocks=2, mlp_ratio=ratio, precision=BF16)
    weights = S.make_weights(cfg, seed=dim + ratio, perturb=True)
    x, hole = inputs(1, H, W, "polygons", seed=H + W + dim)
    check_parity(cfg, weights, x, hole, TOL_BF16)


@pytest.mark.parametrize("dim,H,W", [(384, 64, 96), (512, 96, 64)])
def test_bf16_wide_decoder_channels(dim, H, W):
    """Wider models put 96 and 128 channels on the tensor-core decoder (d/4), the head of
    d512 reads 64 channels."""
    cfg = ModelConfig(dim=dim, heads=dim // 32, window=8, blocks=1, mlp_ratio=1, precision=BF16)
    weights = S.make_weights(cfg, seed=dim, perturb=True)
    x, hole = inputs(1, H, W, "polygons", seed=dim + 1)
    check_parity(cfg, weights, x, hole, TOL_BF16)


def test_bf16_precision_workload_512_full_size():
    """Precision workload at full size: 4 frames of 512x512, d256 h8, 8 blocks, MLP ratio 4."""
    w = WORKLOAD_B
    weights = S.make_weights(w.model, seed=0)
    x, hole = inputs(w.batch, w.height, w.width, w.mask_kind, seed=1)
    gpu = gpu_forward(w.model, weights, x, hole)
    ref = oracle_forward(w.model, weights, x, hole)
    errs = check_parity(w.model, weights, x, hole, TOL_BF16, gpu=gpu, ref=ref)
    print("bf16 512 rel-L2 per frame:", errs)


def test_fp32_precision_workload_512_one_frame():
    w = WORKLOAD_B
    cfg = w.model.with_precision(FP32)
    weights = S.make_weights(cfg, seed=0)
    x, hole = inputs(1, w.height, w.width, w.mask_kind, seed=1)
    errs = check_parity(cfg, weights, x, hole, TOL_FP32)
    print("fp32 512 rel-L2:", errs)


# ----------------------------------------------------------------------------- edge cases and invariants

@pytest.mark.parametrize("precision", [FP32, BF16])
def test_all_hole_and_no_hole_frames(precision):
    cfg = small(precision)
    weights = S.make_weights(cfg, seed=2, perturb=True)
    x = S.make_frames(2, 64, 96, seed=2)
    hole = np.zeros((2, 64, 96), np.uint8)
    hole[0] = 1                                   # frame 0: everything private, frame 1: nothing
    gpu = gpu_forward(cfg, weights, x, hole)
    ref = oracle_forward(cfg, weights, x, hole)
    np.testing.assert_array_equal(gpu["masks"], ref["masks"])
    assert (gpu["masks"][:, 0] == 0).all() and (gpu["masks"][:, 1] == 1).all()
    np.testing.assert_array_equal(gpu["out"][1], x[1])
    tol = TOL_FP32 if precision == FP32 else TOL_BF16
    assert hole_rel_l2(gpu["out"][:1], ref["out"][:1], hole[:1])[0] <= tol


@pytest.mark.parametrize("precision", [FP32, BF16])
def test_tiny_frame(precision):
    cfg = small(precision, blocks=2)
    weights = S.make_weights(cfg, seed=4, perturb=True)
    x = S.make_frames(1, 5, 7, seed=4)
    hole = np.zeros((1, 5, 7), np.uint8)
    hole[0, 1:4, 2:5] = 1
    check_parity(cfg, weights, x, hole, TOL_FP32 if precision == FP32 else TOL_BF16)


@pytest.mark.parametrize("precision", [FP32, BF16])
def test_hole_invariance_and_determinism_bitwise(precision):
    cfg = small(precision)
    weights = S.make_weights(cfg, seed=5, perturb=True)
    x, hole = inputs(2, 96, 96, "ellipse_strokes", seed=6)
    a = gpu_forward(cfg, weights, x, hole)
    x2 = x.copy()
    rng = np.random.default_rng(0)
    noise = rng.uniform(-10, 10, x.shape).astype(np.float32)
    hm = np.broadcast_to((hole != 0)[:, None], x.shape)
    x2[hm] = noise[hm]
    b = gpu_forward(cfg, weights, x2, hole)
    np.testing.assert_array_equal(a["out"][hm], b["out"][hm])
    c = gpu_forward(cfg, weights, x, hole)
    np.testing.assert_array_equal(a["out"], c["out"])


def test_batch_ws_and_host_paths_equal_batch():
    cfg = small(BF16)
    weights = S.make_weights(cfg, seed=7, perturb=True)
    x, hole = inputs(2, 64, 128, "polygons", seed=7)
    lib()
    inp = binding.Inpainter(cfg, weights)
    try:
        xt, ht = torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda()
        out1 = inp(xt, ht)
        nbytes = binding.inpaint_workspace_bytes(inp.ctx, 2, 64, 128)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        out2 = torch.empty_like(xt)
        binding.inpaint_batch_ws(inp.ctx, ws, xt, ht, out2)
        out3 = torch.empty(x.shape, dtype=torch.float32).pin_memory()
        binding.inpaint_batch_host(inp.ctx, torch.from_numpy(x).pin_memory(), torch.from_numpy(hole).pin_memory(),
                                   out3)
        torch.cuda.synchronize()
        assert torch.equal(out1.cpu(), out2.cpu())
        assert torch.equal(out1.cpu(), out3)
        small_ws = torch.empty(nbytes // 2, dtype=torch.uint8, device="cuda")
        with pytest.raises(binding.InpaintError):
            binding.inpaint_batch_ws(inp.ctx, small_ws, xt, ht, out2)
    finally:
        inp.close()


@pytest.mark.parametrize("precision", [FP32, BF16, FP16])
def test_host_path_copies_frame_by_frame_equal_the_device_path(precision):
    """The host-buffer entry point copies and embeds frame by frame and copies each frame
    back once its head kernel has written it: pageable and pinned host memory, a ragged
    width, repeated calls and a batch size change give the device path's output bit for
    bit, and the token masks of the call are kept."""
    cfg = small(precision)
    weights = S.make_weights(cfg, seed=9, perturb=True)
    lib()
    inp = binding.Inpainter(cfg, weights)
    try:
        for B, H, W in [(3, 70, 45), (1, 64, 64), (4, 64, 96)]:
            x, hole = inputs(B, H, W, "polygons", seed=B + H)
            ref = inp(torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda()).cpu()
            ref_masks = inp.token_masks(B, H, W)
            for pinned in (False, True):
                xh, hh = torch.from_numpy(x), torch.from_numpy(hole)
                out = torch.full(x.shape, float("nan"), dtype=torch.float32)
                if pinned:
                    xh, hh, out = xh.pin_memory(), hh.pin_memory(), out.pin_memory()
                for _ in range(2):
                    binding.inpaint_batch_host(inp.ctx, xh, hh, out)
                    assert torch.equal(out, ref)
                np.testing.assert_array_equal(inp.token_masks(B, H, W), ref_masks)
    finally:
        inp.close()


def test_invalid_arguments_return_errors():
    lib()
    cfg = small(FP32)
    inp = binding.Inpainter(cfg, S.make_weights(cfg))
    try:
        x = torch.zeros(1, 3, 32, 32, device="cuda")
        h = torch.zeros(1, 32, 32, dtype=torch.uint8, device="cuda")
        with pytest.raises(binding.InpaintError) as e:
            binding.inpaint_batch(inp.ctx, x, h[:, :0], torch.empty_like(x))
        assert e.value.code == binding.E_INVAL
        with pytest.raises(binding.InpaintError):
            binding.inpaint_init(cfg, np.zeros(10, np.float32))
    finally:
        inp.close()


def test_hbm_budget_refuses_large_workspace():
    lib()
    cfg = small(FP32)
    w = S.make_weights(cfg)
    inp = binding.Inpainter(cfg, w, hbm_budget_bytes=64 << 20)
    try:
        x = torch.zeros(8, 3, 512, 512, device="cuda")
        h = torch.zeros(8, 512, 512, dtype=torch.uint8, device="cuda")
        with pytest.raises(binding.InpaintError) as e:
            binding.inpaint_batch(inp.ctx, x, h, torch.empty_like(x))
        assert e.value.code == binding.E_NOMEM
    finally:
        inp.close()


# ----------------------------------------------------------------------------- loss

def test_l1_hole_loss_matches_oracle():
    from oracle import inpaint_oracle as O
    lib()
    cfg = small(FP32)
    inp = binding.Inpainter(cfg, S.make_weights(cfg))
    try:
        B, H, W = 3, 70, 90
        out = S.make_frames(B, H, W, seed=1)
        tgt = S.make_target(B, H, W, seed=1)
        hole = S.make_hole(B, H, W, "ellipse_strokes", seed=1)
        tgt[0, :, :5, :5] = out[0, :, :5, :5]                       # exact ties: sign(0) = 0
        loss = torch.zeros(1, device="cuda")
        grad = torch.empty(B, 3, H, W, device="cuda")
        binding.inpaint_l1_hole_loss(inp.ctx, torch.from_numpy(out).cuda(), torch.from_numpy(tgt).cuda(),
                                     torch.from_numpy(hole).cuda(), loss, grad)
        torch.cuda.synchronize()
        rl, rg = O.l1_hole_loss(torch.from_numpy(out), torch.from_numpy(tgt), torch.from_numpy(hole))
        assert abs(float(loss) - float(rl)) <= 1e-6 * float(rl)
        np.testing.assert_allclose(grad.cpu().numpy(), rg.numpy(), rtol=1e-6, atol=0)
        zero_hole = torch.zeros(B, H, W, dtype=torch.uint8, device="cuda")
        binding.inpaint_l1_hole_loss(inp.ctx, torch.from_numpy(out).cuda(), torch.from_numpy(tgt).cuda(),
                                     zero_hole, loss, grad)
        torch.cuda.synchronize()
        assert float(loss) == 0.0 and float(grad.abs().max()) == 0.0
    finally:
        inp.close()


# ----------------------------------------------------------------------------- full-resolution pre/post

@pytest.mark.parametrize("precision", [FP32, BF16])
def test_fullres_pre_post_matches_oracle(precision):
    from oracle import inpaint_oracle as O
    lib()
    cfg = small(precision, blocks=2)
    weights = S.make_weights(cfg, seed=13, perturb=True)
    B, K, H, W = 2, 4, 136, 190
    rng = np.random.default_rng(13)
    x = S.make_frames(B, H, W, seed=13)
    masks = np.zeros((B, K, H // 2, W // 2), np.uint8)
    for b in range(B):
        for k in range(K):
            masks[b, k] = S.make_hole(1, H // 2, W // 2, "polygons", seed=100 * b + k, area=(0.02, 0.1))[0] * (k + 1)
    sel = (rng.random((B, K)) < 0.6).astype(np.uint8)
    sel[:, 0] = 1
    inp = binding.Inpainter(cfg, weights)
    try:
        xt = torch.from_numpy(x).cuda()
        out = torch.empty_like(xt)
        hole_half = torch.empty(B, H // 2, W // 2, dtype=torch.uint8, device="cuda")
        binding.inpaint_fullres(inp.ctx, xt, torch.from_numpy(masks).cuda(), torch.from_numpy(sel).cuda(), out,
                                hole_half)
        torch.cuda.synchronize()
        out, hole_half = out.cpu().numpy(), hole_half.cpu().numpy()
    finally:
        inp.close()
    with torch.no_grad():
        ref = O.fullres(torch.from_numpy(x), torch.from_numpy(masks), torch.from_numpy(sel),
                        torch.from_numpy(weights.astype(np.float64)), cfg)
    np.testing.assert_array_equal(hole_half, ref["hole_half"].numpy())
    hup = np.repeat(np.repeat(hole_half, 2, axis=1), 2, axis=2)
    known = np.broadcast_to((hup == 0)[:, None], x.shape)
    np.testing.assert_array_equal(out[known], x[known])
    errs = hole_rel_l2(out, ref["out"].numpy(), hup)
    assert max(errs) <= (TOL_FP32 if precision == FP32 else TOL_BF16), errs


# ----------------------------------------------------------------------------- default weights

@pytest.mark.parametrize("precision", [FP32, BF16])
def test_context_from_null_weights_runs_the_documented_default_blob(precision):
    """inpaint_init with NULL weights draws the documented counter-based blob of the
    config's seed; the exported blob equals the numpy restatement (within one float32
    ulp) and the forward pass of that context matches the oracle run on the exported blob."""
    lib()
    cfg = small(precision, blocks=2, pos_bias=1)
    inp = binding.Inpainter(cfg, None, seed=77)
    try:
        blob = binding.inpaint_get_weights(inp.ctx, inp.n_params)
        py = S.default_weights(cfg, 77)
        assert np.all(np.abs(blob - py) <= np.spacing(np.abs(py).astype(np.float32)))
        x, hole = inputs(2, 64, 96, "polygons", seed=77)
        out = inp(torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda())
        torch.cuda.synchronize()
        gpu = {"out": out.cpu().numpy(), "masks": inp.token_masks(2, 64, 96)}
    finally:
        inp.close()
    check_parity(cfg, blob, x, hole, TOL_FP32 if precision == FP32 else TOL_BF16, gpu=gpu)
