"""GB300-native mask-aware windowed-transformer inpainting (arXiv 2509.10466 hot path).

The compute path is the C-ABI library ``libinpaint.so`` (hand-written sm_103a CUDA);
``binding`` marshals arguments into it.  Importing this package does not load the
library; ``binding.load()`` does and raises if it is missing.
"""
from .config import ModelConfig, Workload, FP32, BF16, FP16, WORKLOADS  # noqa: F401

__all__ = ["ModelConfig", "Workload", "FP32", "BF16", "FP16", "WORKLOADS"]
