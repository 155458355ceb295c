"""Serving loop on the GPU: continuous batching across collaborators at mixed resolutions;
every frame's result is bit-identical to the same frame inpainted alone."""
import numpy as np
import pytest
import torch

from paper_2509_10466_gb300 import binding, synthetic as S
from paper_2509_10466_gb300.config import BF16, FP16, FP32, ModelConfig
from paper_2509_10466_gb300.serving import serve

from helpers import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [BF16, FP16, FP32])
def test_each_result_is_the_same_alone_and_in_the_mix(precision):
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, precision=precision)
    weights = S.make_weights(cfg, seed=5, perturb=True)
    res = ((64, 64), (96, 160), (96, 160), (128, 128))
    rep, finished = serve(cfg, weights, resolutions=res, fps=80, seconds=1.0, slots=3, max_batch=3,
                          keep_outputs=True)
    assert rep["status"].get("done", 0) == rep["requests"] and rep["requests"] > 100
    assert rep["batches"] < rep["requests"]            # frames were batched
    assert rep["max_concurrent_batches"] >= 2          # batches overlapped on the device
    inp = binding.Inpainter(cfg, weights)
    try:
        for r in finished[::7]:
            alone = inp(r.x[None].cuda(), r.hole[None].cuda())
            torch.cuda.synchronize()
            assert torch.equal(alone[0].cpu(), r.out), (r.rid, r.H, r.W)
    finally:
        inp.close()


def test_with_memory_each_stream_matches_its_frames_run_alone_in_order():
    """Temporal memory in the serving loop: every collaborator's frames, replayed alone in
    order with the same memory rotation, give the same bytes as in the mix."""
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=4, mlp_ratio=2, precision=BF16, mem_slots=2)
    weights = S.make_weights(cfg, seed=9, perturb=True)
    res = ((64, 64), (96, 160), (96, 160))
    rep, finished = serve(cfg, weights, resolutions=res, fps=60, seconds=0.6, slots=3, max_batch=3,
                          keep_outputs=True)
    assert rep["status"].get("done", 0) == rep["requests"]
    inp = binding.Inpainter(cfg, weights)
    try:
        for c in range(len(res)):
            mine = sorted((r for r in finished if r.collab == c), key=lambda r: r.rid)
            H, W = res[c]
            bufs = []
            for k, r in enumerate(mine):
                slots = [bufs[k - 1 - j] if k - 1 - j >= 0 else None for j in range(2)]
                buf = inp.memory_buffer(H, W)
                alone = inp.with_memory(r.x[None].cuda(), r.hole[None].cuda(), [slots], [buf])
                torch.cuda.synchronize()
                bufs.append(buf)
                assert torch.equal(alone[0].cpu(), r.out), (c, k, r.rid)
    finally:
        inp.close()
