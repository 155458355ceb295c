"""Failure detection on the device, exercised without faulting or hanging the GPU.

A kernel's bounded wait that runs out writes an error code into the context's error word
and returns; inpaint_sync reports it as INPAINT_E_DEVICE and clears it.  The hook kernel
waits on an mbarrier that nothing arrives at, with a 1 ms limit, through the same wait
primitive the tensor-core kernels use.  A host deadline that passes while work is still
queued gives INPAINT_E_TIMEOUT and leaves the work running.
"""
import numpy as np
import pytest
import torch

from paper_2509_10466_gb300 import binding, synthetic as S
from paper_2509_10466_gb300.config import BF16, ModelConfig, WORKLOAD_B

from helpers import inputs, lib

pytestmark = pytest.mark.gpu


def test_expired_device_wait_is_reported_once_and_the_context_stays_usable():
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, precision=BF16)
    weights = S.make_weights(cfg, seed=1)
    inp = binding.Inpainter(cfg, weights)
    try:
        x, hole = inputs(1, 64, 64, "polygons", seed=1)
        xt, ht = torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda()
        ref = inp(xt, ht)
        assert binding.inpaint_sync(inp.ctx, timeout_ms=10000) == binding.INPAINT_OK
        binding.inpaint_test_wait_expiry(inp.ctx, 1000)
        assert binding.inpaint_sync(inp.ctx, timeout_ms=10000) == binding.E_DEVICE
        # the flag was cleared by the report; the context keeps working
        assert binding.inpaint_sync(inp.ctx, timeout_ms=10000) == binding.INPAINT_OK
        again = inp(xt, ht)
        assert binding.inpaint_sync(inp.ctx, timeout_ms=10000) == binding.INPAINT_OK
        assert torch.equal(ref, again)
    finally:
        inp.close()


def test_wait_expiry_hook_rejects_out_of_range_limits():
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=1, mlp_ratio=2, precision=BF16)
    inp = binding.Inpainter(cfg, S.make_weights(cfg))
    try:
        for bad in (0, -5, 1000001):
            with pytest.raises(binding.InpaintError) as e:
                binding.inpaint_test_wait_expiry(inp.ctx, bad)
            assert e.value.code == binding.E_INVAL
        assert binding.inpaint_sync(inp.ctx, timeout_ms=10000) == binding.INPAINT_OK
    finally:
        inp.close()


def test_host_deadline_passes_while_a_long_batch_runs():
    lib()
    w = WORKLOAD_B
    weights = S.make_weights(w.model, seed=0)
    inp = binding.Inpainter(w.model, weights)
    try:
        x, hole = inputs(8, 512, 512, w.mask_kind, seed=2)
        xt, ht = torch.from_numpy(x).cuda(), torch.from_numpy(hole).cuda()
        out = torch.empty_like(xt)
        binding.inpaint_batch(inp.ctx, xt, ht, out)  # warm-up: workspace, tensor maps
        torch.cuda.synchronize()
        for _ in range(12):  # about 40 ms of queued work
            binding.inpaint_batch(inp.ctx, xt, ht, out)
        assert binding.inpaint_sync(inp.ctx, timeout_ms=0) == binding.E_TIMEOUT
        # the work kept running and finishes normally
        assert binding.inpaint_sync(inp.ctx, timeout_ms=60000) == binding.INPAINT_OK
        assert torch.isfinite(out).all()
    finally:
        inp.close()
