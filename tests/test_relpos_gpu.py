"""Relative-position bias on the GPU: forward parity in both forms (with and without
temporal memory) and the bias table's gradient from the hand-written backward, against
the FP64 oracle (its gradient is autograd of the pinned forward)."""
import numpy as np
import pytest
import torch

from paper_2509_10466_gb300 import synthetic as S
from paper_2509_10466_gb300.config import BF16, FP16, FP32, ModelConfig

from helpers import TOL_BF16, TOL_FP32, check_parity, inputs
from test_backward_gpu import compare, gpu_grad, oracle_grad
from test_memory_gpu import run_gpu, run_oracle, stream
from helpers import hole_rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(FP32, TOL_FP32), (BF16, TOL_BF16), (FP16, TOL_BF16)])
@pytest.mark.parametrize("H,W", [(64, 96), (100, 70)])
def test_forward_with_relative_position_bias(precision, tol, H, W):
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=3, mlp_ratio=2, precision=precision, pos_bias=1)
    weights = S.make_weights(cfg, seed=H + W, perturb=True)
    x, hole = inputs(2, H, W, "polygons", seed=H)
    check_parity(cfg, weights, x, hole, tol)


def test_bf16_d256_with_bias_and_memory():
    cfg = ModelConfig(dim=256, heads=8, window=8, blocks=4, mlp_ratio=4, precision=BF16, pos_bias=1, mem_slots=2)
    weights = S.make_weights(cfg, seed=3, perturb=True)
    x, hole = stream(3, 64, 128, seed=12)
    g_out, g_masks, _ = run_gpu(cfg, weights, x, hole, 2)
    r_out, r_masks, _ = run_oracle(cfg, weights, x, hole, 2)
    assert max(hole_rel_l2(g_out, r_out, hole)) <= TOL_BF16
    for a, b in zip(g_masks, r_masks):
        np.testing.assert_array_equal(a, b)


def test_fp32_memory_with_bias():
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, precision=FP32, pos_bias=1, mem_slots=1)
    weights = S.make_weights(cfg, seed=4, perturb=True)
    x, hole = stream(3, 64, 64, seed=13)
    g_out, _, _ = run_gpu(cfg, weights, x, hole, 1)
    r_out, _, _ = run_oracle(cfg, weights, x, hole, 1)
    assert max(hole_rel_l2(g_out, r_out, hole)) <= TOL_FP32


@pytest.mark.parametrize("H,W,blocks", [(64, 64, 1), (96, 64, 2)])
def test_backward_includes_the_bias_table(H, W, blocks):
    cfg = ModelConfig(dim=32, heads=1, window=8, blocks=blocks, mlp_ratio=2, precision=FP32, pos_bias=1)
    weights = S.make_weights(cfg, seed=21, perturb=True)
    x, hole = inputs(1, H, W, "ellipse_strokes", seed=21)
    gout = np.random.default_rng(21).standard_normal(x.shape).astype(np.float32) * (hole[:, None] != 0)
    g = gpu_grad(cfg, weights, x, hole, gout)
    ref = oracle_grad(cfg, weights, x, hole, gout)
    compare(cfg, g, ref)
    # the tables themselves carry gradient and match
    pos = 0
    for name, shape in S.param_shapes(cfg):
        n = int(np.prod(shape))
        if name.endswith("relpos"):
            r = ref[pos:pos + n]
            assert np.linalg.norm(r) > 0
            assert np.linalg.norm(g[pos:pos + n] - r) <= 1e-4 * np.linalg.norm(r)
        pos += n
