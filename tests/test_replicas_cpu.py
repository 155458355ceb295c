"""The multi-rank (replica) path on CPU: two gloo ranks reduce their step times to the
job maximum and report whole-job throughput; no data-path collective exists."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_10466_gb300.replicas import frame_seed, job_time_and_throughput


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 2.0 + rank          # rank 1 is the slow one
        t, thr = job_time_and_throughput(local, frames_per_rank=40, dist=dist)
        out[rank] = (t, thr, frame_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_frames():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t, thr, seed = res[rank]
        assert t == 3.0                         # max over ranks
        assert thr == pytest.approx(2 * 40 / 3.0)
    assert res[0][2] != res[1][2]               # replicas see different frames


def test_single_rank_needs_no_process_group():
    t, thr = job_time_and_throughput(0.5, 4)
    assert t == 0.5 and thr == 8.0
    with pytest.raises(ValueError):
        job_time_and_throughput(0.0, 4)
