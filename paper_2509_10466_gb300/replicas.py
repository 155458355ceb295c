"""Replica (data-parallel) bookkeeping for multi-GPU runs.

Frames are independent, so N GPUs run N independent replicas of the inpainting pass
with no exchange on the data path.  The only collective is the timing reduction of a
measurement: every rank times its own steps, the job's time is the maximum over ranks,
and the job's throughput is the frames of all ranks divided by that time.
"""
from __future__ import annotations


def job_time_and_throughput(local_seconds: float, frames_per_rank: int, dist=None, device=None):
    """(max over ranks of local_seconds, world_size * frames_per_rank / that maximum).

    `dist` is torch.distributed with an initialized process group (None: one rank).
    """
    world = 1
    t = float(local_seconds)
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        buf = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(buf, op=dist.ReduceOp.MAX)
        t = float(buf.item())
    if t <= 0:
        raise ValueError("non-positive job time")
    return t, world * frames_per_rank / t


def frame_seed(rank: int, base: int = 1) -> int:
    """Seed of a rank's synthetic frames: ranks see different frames of the same workload."""
    return base + 1000 * rank
