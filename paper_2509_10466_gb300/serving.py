"""Continuous-batching request loop for several MR collaborators.

Each collaborator streams frames (one inpainting request per frame) at its own
resolution; the paper's pipeline runs one frame at a time per camera at >= 20 fps
(Section "Success Criteria") and hands frames to the inpainting process as they come
("Processing Server", I/O).  Here requests from several collaborators share one GPU:

  arrivals -> per-resolution queues -> the bucket whose head request is oldest is
  batched (up to `max_batch` frames that have already arrived) -> admitted when a
  stream slot is free and its device memory (workspace + frame buffers) fits the HBM
  budget -> launched asynchronously on that slot's stream -> a completion poller
  records latency = completion - arrival and releases the slot and the memory.

Requests that arrive while others are on the GPU join the next batches as slots and
memory free up, and batches on different streams overlap on the device.  The kernels
are batch-invariant, so a frame's result is the same alone and in the mix.

With temporal memory (m slots), a collaborator's frame reads the memory tensors of its
m previous frames: a batch then takes at most one frame per collaborator (in arrival
order), and the executor keeps each collaborator's ring of m + 1 memory buffers on the
device and orders a frame after its predecessor's batch with a CUDA event.

The scheduler is written against an executor interface (`launch`, `poll`, `bytes_for`)
so that its admission and failure logic is tested on the CPU with a fake device;
`GpuExecutor` runs the real library on CUDA streams.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    collab: int
    H: int
    W: int
    arrival: float                      # seconds on the scheduler clock
    x: object = None                    # host frame [3, H, W] float32 (pinned tensor or ndarray)
    hole: object = None                 # host hole mask [H, W] uint8
    done: Optional[float] = None
    status: str = "queued"              # queued | running | done | failed | timeout
    out: object = None


@dataclasses.dataclass
class Batch:
    reqs: List[Request]
    H: int
    W: int
    nbytes: int
    slot: int
    handle: object = None
    launched: float = 0.0


class SchedulerError(RuntimeError):
    pass


class Scheduler:
    """Resolution-bucketed continuous batching with admission by device memory.

    executor.bytes_for(B, H, W) -> device bytes one batch holds while in flight
    executor.launch(batch) -> handle           (asynchronous; may raise)
    executor.poll(handle) -> bool               (True once the batch has finished; may raise)
    executor.collect(handle, batch) -> None     (fills req.out for each request)
    """

    def __init__(self, executor, slots: int = 4, max_batch: int = 4, hbm_budget: int = 8 << 30,
                 timeout_s: float = 5.0, clock: Callable[[], float] = time.perf_counter, keep_outputs: bool = False,
                 one_per_collab: bool = False):
        if slots < 1 or max_batch < 1:
            raise ValueError("slots and max_batch must be >= 1")
        self.ex = executor
        self.slots_free = list(range(slots))
        self.max_batch = max_batch
        self.budget = hbm_budget
        self.timeout = timeout_s
        self.clock = clock
        self.keep_outputs = keep_outputs
        self.one_per_collab = one_per_collab
        self.queues: Dict[tuple, collections.deque] = collections.OrderedDict()
        self.running: List[Batch] = []
        self.in_use = 0
        self.peak_in_use = 0
        self.finished: List[Request] = []
        self.admission_waits = 0            # times a ready batch waited for memory
        self.batches = 0
        self.max_concurrent = 0

    # ------------------------------------------------------------------ queueing
    def submit(self, req: Request):
        key = (req.H, req.W)
        self.queues.setdefault(key, collections.deque()).append(req)

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def _oldest_bucket(self, now: float):
        best, best_t = None, None
        for key, q in self.queues.items():
            if q and q[0].arrival <= now and (best_t is None or q[0].arrival < best_t):
                best, best_t = key, q[0].arrival
        return best

    # ------------------------------------------------------------------ one scheduling round
    def poll(self):
        """Retire finished batches (and expired ones), then admit as many batches as fit."""
        now = self.clock()
        still = []
        for b in self.running:
            try:
                finished = self.ex.poll(b.handle)
            except Exception:
                self._retire(b, "failed", now)
                continue
            if finished:
                try:
                    self.ex.collect(b.handle, b)
                    self._retire(b, "done", self.clock())
                except Exception:
                    self._retire(b, "failed", now)
            elif now - b.launched > self.timeout:
                self._retire(b, "timeout", now, release=False)
            else:
                still.append(b)
        self.running = still
        self._admit()

    def _retire(self, b: Batch, status: str, t: float, release: bool = True):
        for r in b.reqs:
            r.status = status
            r.done = t
            if not self.keep_outputs:
                r.out = None
            self.finished.append(r)
        if release:
            self.in_use -= b.nbytes
            self.slots_free.append(b.slot)
        # a timed-out batch keeps its slot and memory: its kernels may still be running

    def _admit(self):
        while self.slots_free:
            now = self.clock()
            key = self._oldest_bucket(now)
            if key is None:
                return
            q = self.queues[key]
            # candidates in arrival order; with one_per_collab a collaborator's later frames
            # wait for a later batch (they read the memory its earlier frame writes)
            pick, seen = [], set()
            for i, r in enumerate(q):
                if len(pick) == self.max_batch or r.arrival > now:
                    break
                if self.one_per_collab:
                    if r.collab in seen:
                        continue
                    seen.add(r.collab)
                pick.append(i)
            n = len(pick)
            H, W = key
            need = self.ex.bytes_for(n, H, W)
            while n > 1 and self.in_use + need > self.budget:
                n -= 1
                need = self.ex.bytes_for(n, H, W)
            if self.in_use + need > self.budget:
                if not self.running:
                    raise SchedulerError(f"a single {H}x{W} frame needs {need} B, above the budget {self.budget} B")
                self.admission_waits += 1
                return
            chosen = set(pick[:n])
            reqs = [q[i] for i in pick[:n]]
            self.queues[key] = q = collections.deque(r for i, r in enumerate(q) if i not in chosen)
            slot = self.slots_free.pop(0)
            b = Batch(reqs, H, W, need, slot)
            for r in reqs:
                r.status = "running"
            b.launched = now
            try:
                b.handle = self.ex.launch(b)
            except Exception:
                self.slots_free.append(slot)
                for r in reqs:
                    r.status = "failed"
                    r.done = now
                    self.finished.append(r)
                continue
            self.in_use += need
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.running.append(b)
            self.batches += 1
            self.max_concurrent = max(self.max_concurrent, len(self.running))

    # ------------------------------------------------------------------ driver
    def run(self, requests: List[Request], idle_sleep: float = 50e-6, deadline_s: float = 600.0):
        """Feed `requests` (sorted by arrival, times relative to the start) in real time."""
        start = self.clock()
        for r in requests:
            r.arrival += start
        i = 0
        while i < len(requests) or self.pending() or self.running:
            now = self.clock()
            while i < len(requests) and requests[i].arrival <= now:
                self.submit(requests[i])
                i += 1
            self.poll()
            if now - start > deadline_s:
                raise SchedulerError("serving run exceeded its deadline")
            if idle_sleep:
                time.sleep(idle_sleep)
        return self.finished

    # ------------------------------------------------------------------ report
    def report(self) -> dict:
        by_res = collections.defaultdict(list)
        for r in self.finished:
            if r.status == "done":
                by_res[f"{r.H}x{r.W}"].append(1000.0 * (r.done - r.arrival))
        out = {}
        for k, v in sorted(by_res.items()):
            a = np.array(v)
            out[k] = {"n": int(a.size), "p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
                      "max_ms": float(a.max())}
        status = collections.Counter(r.status for r in self.finished)
        return {"latency": out, "status": dict(status), "batches": self.batches,
                "admission_waits": self.admission_waits, "peak_bytes": self.peak_in_use,
                "max_concurrent_batches": self.max_concurrent}


# ---------------------------------------------------------------------- workload
def poisson_requests(resolutions, fps: float, seconds: float, seed: int = 0) -> List[Request]:
    """Arrival times of each collaborator's frames: a Poisson process at `fps`."""
    rng = np.random.default_rng(seed)
    reqs = []
    for c, (H, W) in enumerate(resolutions):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / fps)
            if t >= seconds:
                break
            reqs.append(Request(0, c, H, W, t))
    reqs.sort(key=lambda r: r.arrival)
    for i, r in enumerate(reqs):
        r.rid = i
    return reqs


# ---------------------------------------------------------------------- GPU executor
class GpuExecutor:
    """Runs batches through the library (inpaint_batch_ws) on per-slot CUDA streams.

    Each batch copies its frames host -> device on its stream, runs the forward pass with
    its own workspace, copies the outputs back and records an event; memory comes from
    torch's caching allocator and is counted against the scheduler's budget.
    """

    def __init__(self, inpainter, slots: int):
        import torch
        from . import binding
        self.torch = torch
        self.binding = binding
        self.inp = inpainter
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.m = inpainter.cfg.mem_slots
        self.rings: Dict[int, list] = {}       # collaborator -> m + 1 memory buffers
        self.count: Dict[int, int] = {}        # collaborator -> frames launched
        self.last_ev: Dict[int, object] = {}   # collaborator -> event of its latest batch

    def bytes_for(self, B, H, W):
        ws = self.binding.inpaint_workspace_bytes(self.inp.ctx, B, H, W)
        return ws + B * H * W * (3 * 4 * 2 + 1) + 4096

    def launch(self, b: Batch):
        torch = self.torch
        st = self.streams[b.slot]
        B, H, W = len(b.reqs), b.H, b.W
        with torch.cuda.stream(st):
            ws = torch.empty(self.binding.inpaint_workspace_bytes(self.inp.ctx, B, H, W), dtype=torch.uint8,
                             device="cuda")
            x = torch.empty(B, 3, H, W, device="cuda")
            hole = torch.empty(B, H, W, dtype=torch.uint8, device="cuda")
            out = torch.empty_like(x)
            for i, r in enumerate(b.reqs):
                x[i].copy_(r.x, non_blocking=True)
                hole[i].copy_(r.hole, non_blocking=True)
            if self.m == 0:
                self.binding.inpaint_batch_ws(self.inp.ctx, ws, x, hole, out, None, st)
            else:
                mem_in, mem_out = [], []
                for r in b.reqs:
                    c = r.collab
                    if c not in self.rings:
                        self.rings[c] = [self.inp.memory_buffer(H, W) for _ in range(self.m + 1)]
                        self.count[c] = 0
                    ring, k = self.rings[c], self.count[c]
                    mem_in.append([ring[(k - 1 - j) % (self.m + 1)] if k - 1 - j >= 0 else None for j in range(self.m)])
                    mem_out.append(ring[k % (self.m + 1)])
                    self.count[c] = k + 1
                    if c in self.last_ev:
                        st.wait_event(self.last_ev[c])
                self.binding.inpaint_batch_mem(self.inp.ctx, x, hole, out, mem_in, mem_out, None, st, workspace=ws)
            host = torch.empty((B, 3, H, W), dtype=torch.float32, pin_memory=True)
            host.copy_(out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
            if self.m:
                for r in b.reqs:
                    self.last_ev[r.collab] = ev
        return (ev, host, (ws, x, hole, out))

    def poll(self, handle):
        return handle[0].query()

    def collect(self, handle, b: Batch):
        host = handle[1]
        for i, r in enumerate(b.reqs):
            r.out = host[i]


def make_collaborator_frames(resolutions, frames_per_collab: int = 8, seed: int = 0):
    """Pinned host frames and drifting-blob holes for each collaborator (cycled)."""
    import torch
    from . import synthetic as S
    pool = []
    for c, (H, W) in enumerate(resolutions):
        xs = S.make_frames(frames_per_collab, H, W, seed=seed + 100 * c)
        blobs = S.DriftingBlobs(H, W, seed=seed + 100 * c)
        hs = np.stack([blobs.next() for _ in range(frames_per_collab)])
        pool.append(([torch.from_numpy(xs[i]).pin_memory() for i in range(frames_per_collab)],
                     [torch.from_numpy(hs[i]).pin_memory() for i in range(frames_per_collab)]))
    return pool


def serve(cfg, weights, resolutions=((256, 256), (512, 512), (720, 1280), (720, 1280)), fps: float = 30.0,
          seconds: float = 20.0, slots: int = 4, max_batch: int = 4, hbm_budget: int = 16 << 30, seed: int = 0,
          keep_outputs: bool = False):
    """Run the serving workload in real time on cuda:0 and return (report, finished requests)."""
    import torch
    from . import binding
    inp = binding.Inpainter(cfg, weights)
    try:
        ex = GpuExecutor(inp, slots)
        pool = make_collaborator_frames(resolutions, seed=seed)
        # warm up each resolution once (kernel attributes, allocator)
        for i, (H, W) in enumerate(sorted(set(resolutions))):
            xs, hs = pool[resolutions.index((H, W))]
            # a collaborator id of its own: warm-up frames do not enter a stream's memory
            b = Batch([Request(-1, -1 - i, H, W, 0.0, xs[0], hs[0])], H, W, 0, 0)
            h = ex.launch(b)
            h[0].synchronize()
        reqs = poisson_requests(resolutions, fps, seconds, seed)
        for r in reqs:
            xs, hs = pool[r.collab]
            k = r.rid % len(xs)
            r.x, r.hole = xs[k], hs[k]
        sch = Scheduler(ex, slots=slots, max_batch=max_batch, hbm_budget=hbm_budget, keep_outputs=keep_outputs,
                        one_per_collab=cfg.mem_slots > 0)
        wall0 = time.perf_counter()
        sch.run(reqs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        rep = sch.report()
        done = sum(1 for r in sch.finished if r.status == "done")
        rep["frames_per_s"] = done / wall
        rep["seconds"] = wall
        rep["requests"] = len(reqs)
        return rep, sch.finished
    finally:
        inp.close()
