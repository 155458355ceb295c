"""GPU parity at the largest and deepest workloads against the FP64 oracle.

The BF16 form's error grows with depth (operands rounded to bf16 in every block), so the
1080p workload (12 blocks) and the serving model on a 720p frame are checked at their
full size: masks bit-exact, known pixels copied exactly, hole pixels within the BF16
tolerance of relative L2 per frame.  The oracle takes tens of seconds per 1080p frame.
"""
import numpy as np
import pytest

from paper_2509_10466_gb300 import synthetic as S
from paper_2509_10466_gb300.config import WORKLOAD_D_MODEL, WORKLOAD_E

from helpers import TOL_BF16, check_parity, gpu_forward, oracle_forward

pytestmark = pytest.mark.gpu


def test_bf16_hd_1080_twelve_blocks():
    """1080x1920 (padded to 1088x1920), d256 h8, 12 blocks, MLP ratio 4, BF16: one large
    contiguous hole plus thin strokes covering 5-50 % of the frame."""
    w = WORKLOAD_E
    weights = S.make_weights(w.model, seed=0)
    x = S.make_frames(1, w.height, w.width, seed=3)
    hole = S.make_hole(1, w.height, w.width, w.mask_kind, seed=3)
    gpu = gpu_forward(w.model, weights, x, hole)
    ref = oracle_forward(w.model, weights, x, hole)
    errs = check_parity(w.model, weights, x, hole, TOL_BF16, gpu=gpu, ref=ref)
    print("bf16 1080p 12-block hole rel-L2 per frame:", errs)


def test_bf16_serving_model_720p_frame():
    """The serving model (d256 h8, 8 blocks, MLP ratio 4, BF16) on one 720x1280 frame
    (padded to 736x1280) with the serving workload's drifting-blob hole."""
    cfg = WORKLOAD_D_MODEL
    weights = S.make_weights(cfg, seed=0)
    x = S.make_frames(1, 720, 1280, seed=9)
    hole = S.DriftingBlobs(720, 1280, seed=9).next()[None]
    assert 0 < hole.mean() < 1
    gpu = gpu_forward(cfg, weights, x, hole)
    ref = oracle_forward(cfg, weights, x, hole)
    errs = check_parity(cfg, weights, x, hole, TOL_BF16, gpu=gpu, ref=ref)
    print("bf16 720p serving-model hole rel-L2:", errs)
