"""Scheduler logic of the serving loop on a fake device (CPU): bucketing, continuous
admission, the HBM budget, and host-side failure handling (a launch that raises, a
poll that raises, a batch that never finishes)."""
import pytest

from paper_2509_10466_gb300.serving import Request, Scheduler, SchedulerError, poisson_requests


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeDevice:
    """Each batch takes `per_frame` seconds per frame; optional failure injection."""

    def __init__(self, clock, per_frame=0.01, fail_launch=(), fail_poll=(), stall=()):
        self.clock = clock
        self.per_frame = per_frame
        self.fail_launch, self.fail_poll, self.stall = set(fail_launch), set(fail_poll), set(stall)
        self.launched = []

    def bytes_for(self, B, H, W):
        return B * H * W

    def launch(self, b):
        first = b.reqs[0].rid
        if first in self.fail_launch:
            raise RuntimeError("injected launch failure")
        self.launched.append([r.rid for r in b.reqs])
        return (first, self.clock() + self.per_frame * len(b.reqs))

    def poll(self, h):
        if h[0] in self.fail_poll:
            raise RuntimeError("injected device error")
        if h[0] in self.stall:
            return False
        return self.clock() >= h[1]

    def collect(self, h, b):
        for r in b.reqs:
            r.out = ("frame", r.rid)


def drive(sch, clock, reqs, dt=0.001, limit=10.0):
    reqs = sorted(reqs, key=lambda r: r.arrival)
    i = 0
    while (i < len(reqs) or sch.pending() or sch.running) and clock.t < limit:
        while i < len(reqs) and reqs[i].arrival <= clock.t:
            sch.submit(reqs[i])
            i += 1
        sch.poll()
        clock.t += dt
    return sch


def test_batches_are_single_resolution_and_oldest_bucket_first():
    clock = Clock()
    dev = FakeDevice(clock)
    sch = Scheduler(dev, slots=1, max_batch=3, hbm_budget=1 << 30, clock=clock, keep_outputs=True)
    reqs = [Request(0, 0, 64, 64, 0.000), Request(1, 1, 32, 32, 0.0001), Request(2, 0, 64, 64, 0.0002),
            Request(3, 1, 32, 32, 0.0003), Request(4, 0, 64, 64, 0.0004)]
    clock.t = 0.001
    for r in reqs:
        sch.submit(r)
    drive(sch, clock, [])
    assert dev.launched[0] == [0, 2, 4]          # 64x64 head is oldest; up to 3 frames
    assert dev.launched[1] == [1, 3]
    assert all(r.status == "done" and r.out == ("frame", r.rid) for r in sch.finished)


def test_requests_arriving_during_a_batch_join_later_batches():
    clock = Clock()
    dev = FakeDevice(clock, per_frame=0.02)
    sch = Scheduler(dev, slots=2, max_batch=4, hbm_budget=1 << 30, clock=clock)
    reqs = [Request(i, 0, 32, 32, 0.005 * i) for i in range(12)]
    drive(sch, clock, reqs)
    assert len(sch.finished) == 12 and all(r.status == "done" for r in sch.finished)
    assert len(dev.launched) > 1 and sch.max_concurrent >= 2
    # every request was launched after it arrived, none waited for a batch to fill up
    for r in sch.finished:
        assert r.done >= r.arrival


def test_memory_budget_is_never_exceeded_and_waits_are_counted():
    clock = Clock()
    dev = FakeDevice(clock, per_frame=0.01)
    budget = 3 * 64 * 64
    sch = Scheduler(dev, slots=4, max_batch=4, hbm_budget=budget, clock=clock)
    reqs = poisson_requests([(64, 64), (64, 64), (32, 32)], fps=200, seconds=0.2, seed=1)
    drive(sch, clock, reqs)
    assert sch.peak_in_use <= budget
    assert sch.admission_waits > 0
    assert all(r.status == "done" for r in sch.finished) and len(sch.finished) == len(reqs)


def test_failures_are_reported_and_resources_released():
    clock = Clock()
    dev = FakeDevice(clock, fail_launch={0}, fail_poll={3}, stall={6})
    sch = Scheduler(dev, slots=2, max_batch=1, hbm_budget=1 << 30, timeout_s=0.05, clock=clock)
    reqs = [Request(i, 0, 32, 32, 0.01 * i) for i in range(9)]
    drive(sch, clock, reqs, limit=2.0)
    st = {r.rid: r.status for r in sch.finished}
    assert st[0] == "failed" and st[3] == "failed" and st[6] == "timeout"
    assert all(st[i] == "done" for i in (1, 2, 4, 5, 7, 8))
    # the stalled batch keeps its slot (its kernels may still run); the others were released
    assert len(sch.slots_free) == 1 and sch.in_use == 32 * 32


def test_single_frame_above_budget_is_an_error():
    clock = Clock()
    sch = Scheduler(FakeDevice(clock), slots=1, max_batch=1, hbm_budget=100, clock=clock)
    sch.submit(Request(0, 0, 64, 64, 0.0))
    with pytest.raises(SchedulerError):
        sch.poll()


def test_poisson_workload_shape():
    reqs = poisson_requests([(256, 256), (512, 512), (720, 1280), (720, 1280)], fps=30, seconds=20, seed=0)
    assert 2200 < len(reqs) < 2600
    assert all(a.arrival <= b.arrival for a, b in zip(reqs, reqs[1:]))
    assert {(r.H, r.W) for r in reqs} == {(256, 256), (512, 512), (720, 1280)}


def test_with_memory_a_batch_takes_one_frame_per_collaborator_in_order():
    """With temporal memory a frame reads what its collaborator's previous frame writes:
    no batch holds two frames of one collaborator, and each collaborator's frames are
    launched in arrival order, while other collaborators still share batches."""
    clock = Clock()
    dev = FakeDevice(clock, per_frame=0.005)
    sch = Scheduler(dev, slots=2, max_batch=4, hbm_budget=1 << 40, clock=clock, one_per_collab=True)
    reqs = []
    for k in range(6):                 # collaborators 0 and 1 queue 3 frames each at t = 0
        reqs.append(Request(k, k % 2, 64, 64, 0.0))
    reqs.append(Request(6, 2, 64, 64, 0.0))
    drive(sch, clock, reqs)
    assert all(r.status == "done" for r in sch.finished) and len(sch.finished) == 7
    collab = {r.rid: r.collab for r in reqs}
    seen = {}
    for batch in dev.launched:
        cs = [collab[i] for i in batch]
        assert len(cs) == len(set(cs)), batch
        for i in batch:
            c = collab[i]
            assert seen.get(c, -1) < i
            seen[c] = i
    assert max(len(b) for b in dev.launched) >= 2
