"""The FP16 operand form against the FP64 oracle.

The paper's inpainter runs as an FP16 TensorRT engine ("Inpainting Model", "Hardware");
the FP16 form here runs every tensor-core kernel with FP16 instead of BF16 operands (same
width; 11-bit significand instead of 8, exponent range 2^-14 .. 65504 instead of BF16's
FP32 range), with FP32 accumulation, softmax statistics, LayerNorms and residual stream.
The tolerance is the 16-bit one of relative L2 2e-2 on hole pixels per frame; masks and
known pixels are exact.  With three more significand bits the FP16 form's error is also
checked to be well below the BF16 form's on the same inputs (a form that kept BF16
rounding anywhere would not be).
"""
import numpy as np
import pytest

from paper_2509_10466_gb300 import synthetic as S
from paper_2509_10466_gb300.config import BF16, FP16, ModelConfig, WORKLOAD_B

from helpers import TOL_BF16, check_parity, gpu_forward, inputs, oracle_forward

pytestmark = pytest.mark.gpu

TOL_FP16 = 2e-2


@pytest.mark.parametrize("H,W,B", [(64, 64, 1), (96, 128, 2), (70, 45, 1)])
def test_fp16_small_shapes(H, W, B):
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=3, mlp_ratio=2, precision=FP16)
    weights = S.make_weights(cfg, seed=11, perturb=True)
    x, hole = inputs(B, H, W, "polygons", seed=H + W)
    check_parity(cfg, weights, x, hole, TOL_FP16)


@pytest.mark.parametrize("dim,ratio,H,W", [(256, 4, 64, 96), (128, 8, 32, 32), (64, 4, 96, 96)])
def test_fp16_fused_mlp_and_tensor_core_decoder(dim, ratio, H, W):
    cfg = ModelConfig(dim=dim, heads=dim // 32, window=8, blocks=2, mlp_ratio=ratio, precision=FP16)
    weights = S.make_weights(cfg, seed=dim + ratio, perturb=True)
    x, hole = inputs(1, H, W, "polygons", seed=H + W + dim)
    check_parity(cfg, weights, x, hole, TOL_FP16)


def test_fp16_relative_position_bias_and_wide_decoder():
    cfg = ModelConfig(dim=384, heads=12, window=8, blocks=1, mlp_ratio=1, precision=FP16, pos_bias=1)
    weights = S.make_weights(cfg, seed=5, perturb=True)
    x, hole = inputs(1, 64, 96, "polygons", seed=6)
    check_parity(cfg, weights, x, hole, TOL_FP16)


def test_fp16_precision_workload_512_error_below_bf16():
    """4 frames of 512x512, d256 h8, 8 blocks, MLP ratio 4: FP16 within the 16-bit
    tolerance, and its hole error at most half of the BF16 form's on the same frames."""
    w = WORKLOAD_B
    weights = S.make_weights(w.model, seed=0)
    x, hole = inputs(w.batch, w.height, w.width, w.mask_kind, seed=1)
    ref = oracle_forward(w.model, weights, x, hole)
    cfg16 = w.model.with_precision(FP16)
    e16 = check_parity(cfg16, weights, x, hole, TOL_FP16, gpu=gpu_forward(cfg16, weights, x, hole), ref=ref)
    eb = check_parity(w.model, weights, x, hole, TOL_BF16, gpu=gpu_forward(w.model, weights, x, hole), ref=ref)
    print("fp16 512 rel-L2 per frame:", e16, "bf16:", eb)
    assert max(e16) <= 0.5 * min(eb), (e16, eb)
