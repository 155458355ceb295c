"""Model and workload configurations of the inpainting hot path.

Pure data: no arithmetic of the method lives here.  The five named workloads mirror
the shapes the paper's pipeline is exercised at (plain FP32 at 256x256, the BF16
precision form at 512x512, the fine-tuning step, the multi-collaborator serving mix
and the 1080p frame).  The paper itself fixes only the outline of the network
(a hybrid CNN/transformer inpainter that takes the frame with its masked regions set
to 0 and returns the completed frame, Section "Inpainting Manager"); the layer sizes
below are the stated workload sizes.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

FP32 = 0
BF16 = 1
FP16 = 2


@dataclass(frozen=True)
class ModelConfig:
    dim: int = 128          # d, token channels
    heads: int = 4          # h, attention heads (d / h = 32 everywhere)
    window: int = 8         # window side in tokens (8x8 = 64 tokens)
    blocks: int = 2         # L, transformer blocks
    mlp_ratio: int = 2      # r, MLP hidden = r * d
    patch: int = 4          # 4x4 stride-4 patch embedding
    dec_c1: int = 0         # decoder stage-1 channels (0 -> d/4)
    dec_c2: int = 0         # decoder stage-2 channels (0 -> d/8)
    precision: int = FP32   # FP32 plain form, or the BF16 / FP16 tensor-core forms
    shift: int = 1          # 1: odd blocks use windows offset by half a window
    mem_slots: int = 0      # m: temporal memory slots (odd blocks attend to m past frames)
    pos_bias: int = 0       # 1: learned relative-position bias (per head, 15 x 15) in the window softmax

    @property
    def c1(self) -> int:
        return self.dec_c1 or self.dim // 4

    @property
    def c2(self) -> int:
        return self.dec_c2 or self.dim // 8

    @property
    def head_dim(self) -> int:
        return self.dim // self.heads

    @property
    def hidden(self) -> int:
        return self.dim * self.mlp_ratio

    @property
    def pad_multiple(self) -> int:
        # frames are padded so that the token grid tiles into whole windows
        return self.patch * self.window

    def with_precision(self, precision: int) -> "ModelConfig":
        return replace(self, precision=precision)


@dataclass(frozen=True)
class Workload:
    name: str
    model: ModelConfig
    batch: int
    height: int
    width: int
    mask_kind: str          # generator recipe, see synthetic.make_hole


# Plain FP32 forward: 256x256, d128 h4, 2 blocks, MLP ratio 2.
WORKLOAD_A = Workload("plain_fp32_256", ModelConfig(128, 4, 8, 2, 2), 1, 256, 256, "ellipse_strokes")
# Precision form: 512x512 batch 4, d256 h8, 8 blocks, MLP ratio 4 (BF16 vs FP32).
WORKLOAD_B = Workload("precision_512", ModelConfig(256, 8, 8, 8, 4, precision=BF16), 4, 512, 512, "polygons")
# Differentiation: batch 8 at 256x256, d192 h6, 6 blocks (MLP ratio 4).
WORKLOAD_C = Workload("train_256", ModelConfig(192, 6, 8, 6, 4), 8, 256, 256, "ellipse_strokes")
# Finite-difference instance of the differentiation form: 64x64, 1 block, d32 h1.
WORKLOAD_C_FD = Workload("fd_64", ModelConfig(32, 1, 8, 1, 4), 1, 64, 64, "ellipse_strokes")
# Serving: d256 h8, 8 blocks, MLP ratio 4, BF16, mixed resolutions.
WORKLOAD_D_MODEL = ModelConfig(256, 8, 8, 8, 4, precision=BF16)
SERVING_RESOLUTIONS = ((256, 256), (512, 512), (720, 1280), (720, 1280))
# Largest: 1080x1920 padded to 1088x1920, batch 2, d256 h8, 12 blocks, BF16.
WORKLOAD_E = Workload("hd_1080", ModelConfig(256, 8, 8, 12, 4, precision=BF16), 2, 1080, 1920, "large_and_thin")

WORKLOADS = {w.name: w for w in (WORKLOAD_A, WORKLOAD_B, WORKLOAD_C, WORKLOAD_C_FD, WORKLOAD_E)}


def padded(n: int, multiple: int) -> int:
    return (n + multiple - 1) // multiple * multiple
