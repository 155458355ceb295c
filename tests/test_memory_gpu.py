"""Temporal memory on the GPU against the FP64 oracle (calls go through the C ABI).

A stream of frames with moving holes runs frame by frame: frame t attends, in its odd
(temporal) blocks, to the memory tensors that frames t-1 and t-2 emitted.  Token masks
and known pixels must match bit-exactly and hole pixels within the form's tolerance at
every frame; batched calls over several streams must give the same bytes as separate
calls; every slot empty must reproduce the single-frame pass.
"""
import numpy as np
import pytest
import torch

from oracle import inpaint_oracle as O
from paper_2509_10466_gb300 import binding, synthetic as S
from paper_2509_10466_gb300.config import BF16, FP16, FP32, ModelConfig

from helpers import TOL_BF16, TOL_FP32, hole_rel_l2, lib

pytestmark = pytest.mark.gpu


def stream(n, H, W, seed):
    """n frames of one stream: drifting content and a moving hole."""
    x = S.make_frames(n, H, W, seed=seed)
    hole = S.make_hole(n, H, W, "polygons", seed=seed + 1)
    return x, hole


def run_gpu(cfg, weights, x, hole, m):
    """Frame by frame with m memory slots; returns outputs, token masks and the memory bytes."""
    lib()
    inp = binding.Inpainter(cfg, weights)
    try:
        n, H, W = hole.shape
        bufs, outs, masks = [], [], []
        for t in range(n):
            xt = torch.from_numpy(x[t:t + 1]).cuda()
            ht = torch.from_numpy(hole[t:t + 1]).cuda()
            slots = [bufs[t - 1 - j] if t - 1 - j >= 0 else None for j in range(m)]
            mine = inp.memory_buffer(H, W)
            out = inp.with_memory(xt, ht, [slots], [mine])
            torch.cuda.synchronize()
            assert binding.inpaint_sync(inp.ctx, timeout_ms=10000) == binding.INPAINT_OK
            outs.append(out.cpu().numpy()[0])
            masks.append(inp.token_masks(1, H, W))
            bufs.append(mine)
        return np.stack(outs), masks, [b.cpu().numpy() for b in bufs]
    finally:
        inp.close()


def run_oracle(cfg, weights, x, hole, m):
    w = torch.from_numpy(weights.astype(np.float64))
    mems, outs, masks = [], [], []
    with torch.no_grad():
        for t in range(hole.shape[0]):
            slots = [mems[t - 1 - j] if t - 1 - j >= 0 else None for j in range(m)]
            r = O.forward(torch.from_numpy(x[t:t + 1]), torch.from_numpy(hole[t:t + 1]), w, cfg, mem=[slots])
            outs.append(r["out"].numpy()[0])
            masks.append(r["masks"].numpy())
            mems.append(r["memory"][0])
    return np.stack(outs), masks, mems


@pytest.mark.parametrize("precision,tol", [(FP32, TOL_FP32), (BF16, TOL_BF16), (FP16, TOL_BF16)])
def test_stream_with_two_memory_slots_matches_oracle(precision, tol):
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=4, mlp_ratio=2, precision=precision, mem_slots=2)
    weights = S.make_weights(cfg, seed=5, perturb=True)
    x, hole = stream(4, 64, 96, seed=3)
    g_out, g_masks, g_mem = run_gpu(cfg, weights, x, hole, 2)
    r_out, r_masks, r_mem = run_oracle(cfg, weights, x, hole, 2)
    known = np.broadcast_to((hole == 0)[:, None], x.shape)
    np.testing.assert_array_equal(g_out[known], x[known])
    errs = hole_rel_l2(g_out, r_out, hole)
    assert max(errs) <= tol, errs
    for t in range(hole.shape[0]):
        np.testing.assert_array_equal(g_masks[t], r_masks[t])
    # the recorded key masks of each temporal block are the frame's own block-input masks
    N = (64 // 4) * (96 // 4)
    es = 4 if precision == FP32 else 2
    kv = N * 2 * cfg.dim * es
    stride = -(-(kv + N) // 256) * 256
    for t in range(hole.shape[0]):
        for l in (1, 3):
            got = g_mem[t][(l // 2) * stride + kv:(l // 2) * stride + kv + N]
            np.testing.assert_array_equal(got, r_mem[t][l][1].numpy())
    if precision == FP32:  # the recorded keys / values themselves
        for t in range(hole.shape[0]):
            for l in (1, 3):
                got = g_mem[t][(l // 2) * stride:(l // 2) * stride + kv].view(np.float32).reshape(N, 2 * cfg.dim)
                ref = r_mem[t][l][0].numpy()
                assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_all_slots_empty_equals_the_single_frame_pass():
    cfg = ModelConfig(dim=128, heads=4, window=8, blocks=4, mlp_ratio=2, precision=BF16, mem_slots=3)
    weights = S.make_weights(cfg, seed=6, perturb=True)
    x, hole = stream(2, 96, 160, seed=9)
    lib()
    inp = binding.Inpainter(cfg, weights)
    try:
        xt, ht = torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda()
        a = inp(xt, ht)
        b = inp.with_memory(xt, ht, [[None] * 3, [None] * 3], None)
        c = inp.with_memory(xt, ht, None, None)
        torch.cuda.synchronize()
        assert torch.equal(a, b) and torch.equal(a, c)
    finally:
        inp.close()


def test_batched_streams_equal_separate_calls():
    """Two streams batched frame by frame give the same bytes (outputs and memory) as each
    stream run on its own."""
    cfg = ModelConfig(dim=128, heads=4, window=8, blocks=4, mlp_ratio=4, precision=BF16, mem_slots=2)
    weights = S.make_weights(cfg, seed=8, perturb=True)
    H, W = 64, 128
    xa, ha = stream(3, H, W, seed=21)
    xb, hb = stream(3, H, W, seed=31)
    alone = [run_gpu(cfg, weights, xa, ha, 2), run_gpu(cfg, weights, xb, hb, 2)]
    lib()
    inp = binding.Inpainter(cfg, weights)
    try:
        bufs = {0: [], 1: []}
        for t in range(3):
            xt = torch.from_numpy(np.stack([xa[t], xb[t]])).cuda()
            ht = torch.from_numpy(np.stack([ha[t], hb[t]])).cuda()
            mem_in = [[bufs[s][t - 1 - j] if t - 1 - j >= 0 else None for j in range(2)] for s in (0, 1)]
            mine = [inp.memory_buffer(H, W), inp.memory_buffer(H, W)]
            out = inp.with_memory(xt, ht, mem_in, mine).cpu().numpy()
            for s in (0, 1):
                bufs[s].append(mine[s])
                np.testing.assert_array_equal(out[s], alone[s][0][t])
                np.testing.assert_array_equal(mine[s].cpu().numpy(), alone[s][2][t])
    finally:
        inp.close()


def test_memory_arguments_are_checked():
    lib()
    cfg0 = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, precision=BF16)
    cfg2 = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, precision=BF16, mem_slots=2)
    x, hole = stream(1, 64, 64, seed=1)
    xt, ht = torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda()
    inp0 = binding.Inpainter(cfg0, S.make_weights(cfg0, seed=1))
    inp2 = binding.Inpainter(cfg2, S.make_weights(cfg2, seed=1))
    try:
        assert binding.inpaint_memory_bytes(inp0.ctx, 64, 64) == 0
        with pytest.raises(binding.InpaintError):  # no slots, yet memory given
            inp0.with_memory(xt, ht, None, [inp0.memory_buffer(64, 64)])
        buf = inp2.memory_buffer(64, 64)
        with pytest.raises(binding.InpaintError):  # misaligned buffer
            inp2.with_memory(xt, ht, [[buf[1:], None]], None)
        with pytest.raises(binding.InpaintError):
            ModelConfig(dim=64, heads=2, mem_slots=5)
            binding.Inpainter(ModelConfig(dim=64, heads=2, mem_slots=5), S.make_weights(cfg0, seed=1))
    finally:
        inp0.close()
        inp2.close()
