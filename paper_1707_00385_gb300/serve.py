"""A serving loop over the batch entry point: continuous batching of range
frames of mixed resolutions, admission by free device memory, and latency
accounting (p50 / p99) per request.

Requests arrive over time.  The dispatcher keeps up to `inflight` batches on
the GPU (one stream each).  Whenever a stream is free it forms a batch from
the requests that have arrived and not yet been admitted -- as many as fit the
frame and pixel limits of a batch and the device-memory budget -- and enqueues
host-to-device copies of their ranges, one pc_compute_batch launch over all of
them (one persistent kernel, the frames' own sizes and intrinsics), and
device-to-host copies of k1, k2 and the refined normals.  Requests arriving
while batches run wait only for the next free stream, so their work overlaps
with the batches in flight.  A batch's memory returns to the budget when its
completion event has fired.

Failures stay with the requests that caused them.  A request larger than the
whole budget is refused on arrival.  When a batch cannot be launched (an
argument the library rejects, a host copy that fails), its requests go back to
the head of the queue to be launched one per batch, so that one bad frame does
not fail its neighbours; a request that fails alone is marked failed with the
error.  When a launched batch reports an error on completion, its requests are
marked failed.  Either way its slot and memory return, and serving goes on.

Executors do the device work: GpuExecutor (batched), PlainExecutor (one
pc_compute launch per frame on one stream, the unbatched baseline).  Clock,
sleep and executor are parameters, so the scheduling logic runs on the CPU in
tests with a fake clock and a fake executor.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

# device bytes per pixel held by an admitted frame: range in, k1, k2, normal out
BYTES_PER_PIXEL = 4 + 4 + 4 + 12


@dataclass
class Request:
    rid: int
    depth: object                 # host float32 H x W (torch tensor; page-locked for async copies)
    intrinsics: tuple             # (fx, fy, cx, cy) in pixels
    t_arrival: float              # seconds from the start of the run
    t_admit: float = None
    t_done: float = None
    k1: object = None             # host results, filled when done (when the executor keeps them)
    k2: object = None
    normal: object = None
    error: str = None             # why the request was refused or failed (None: served)
    solo: bool = False            # retried alone after its batch failed to launch

    @property
    def pixels(self) -> int:
        return int(self.depth.shape[0]) * int(self.depth.shape[1])

    @property
    def device_bytes(self) -> int:
        return self.pixels * BYTES_PER_PIXEL

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class _Batch:
    reqs: list
    nbytes: int
    handle: object
    slot: int


@dataclass
class ServeStats:
    requests: int                 # requests served (the rates and latencies are over these)
    seconds: float                # first arrival to last completion
    frames_per_s: float
    mpixel_per_s: float
    p50_ms: float
    p99_ms: float
    mean_batch: float
    batches: int
    peak_device_bytes: int
    budget_bytes: int
    refused: int = 0              # larger than the whole budget
    failed: int = 0               # launch or completion failed
    latencies_ms: list = field(default_factory=list, repr=False)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_ms")
        return d


class Server:
    """Continuous-batching dispatcher.  budget_bytes bounds the device memory
    held by admitted, unfinished frames (BYTES_PER_PIXEL per pixel)."""

    def __init__(self, executor, budget_bytes: int, max_batch_frames: int = 64,
                 max_batch_pixels: int = 16 << 20, inflight: int = 2, poll_s: float = 50e-6):
        if inflight < 1 or max_batch_frames < 1 or budget_bytes <= 0:
            raise ValueError("inflight, max_batch_frames and budget_bytes must be positive")
        self.ex = executor
        self.budget = int(budget_bytes)
        self.max_frames = int(max_batch_frames)
        self.max_pixels = int(max_batch_pixels)
        self.inflight = int(inflight)
        self.poll_s = poll_s

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep) -> ServeStats:
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        n = len(reqs)
        waiting = collections.deque()
        running = []                     # batches on the GPU
        free_slots = list(range(self.inflight))
        used = peak = 0
        nb = nframes = 0
        i = 0
        t0 = clock()

        def fail(batch, err, t):
            for r in batch:
                r.error = f"{type(err).__name__}: {err}"
                r.t_done = t

        while i < n or waiting or running:
            now = clock() - t0
            while i < n and reqs[i].t_arrival <= now:
                r = reqs[i]
                i += 1
                if r.device_bytes > self.budget:
                    r.error = f"refused: needs {r.device_bytes} B, more than the budget of {self.budget} B"
                    r.t_admit = r.t_done = now
                else:
                    waiting.append(r)
            progressed = False
            for b in list(running):
                try:
                    finished = self.ex.done(b.handle)
                    if finished:
                        self.ex.finish(b.handle, b.reqs)
                except Exception as e:   # an error reported by the device work of this batch
                    finished = True
                    fail(b.reqs, e, clock() - t0)
                if finished:
                    t = clock() - t0
                    for r in b.reqs:
                        if r.error is None:
                            r.t_done = t
                    used -= b.nbytes
                    running.remove(b)
                    free_slots.append(b.slot)
                    progressed = True
            if waiting and free_slots:
                batch, nbytes, px = [], 0, 0
                while waiting and len(batch) < self.max_frames:
                    r = waiting[0]
                    if batch and (px + r.pixels > self.max_pixels or r.solo):
                        break
                    if used + nbytes + r.device_bytes > self.budget:
                        break
                    waiting.popleft()
                    batch.append(r)
                    nbytes += r.device_bytes
                    px += r.pixels
                    if r.solo:
                        break
                if batch:
                    slot = free_slots.pop(0)
                    t = clock() - t0
                    for r in batch:
                        r.t_admit = t
                    try:
                        handle = self.ex.launch(batch, slot)
                    except Exception as e:   # nothing of this batch is left running
                        free_slots.append(slot)
                        if len(batch) > 1:
                            for r in reversed(batch):
                                r.solo = True
                                waiting.appendleft(r)
                        else:
                            fail(batch, e, clock() - t0)
                        progressed = True
                        continue
                    running.append(_Batch(batch, nbytes, handle, slot))
                    used += nbytes
                    peak = max(peak, used)
                    nb += 1
                    nframes += len(batch)
                    progressed = True
            if not progressed:
                if running:
                    try:
                        self.ex.wait(running[0].handle, self.poll_s)
                    except Exception:
                        pass                 # the error comes back from done() on the next pass
                else:
                    wait = reqs[i].t_arrival - (clock() - t0) if i < n else 0.0
                    sleep(max(0.0, min(wait, 1e-3)))
        served = [r for r in reqs if r.error is None]
        refused = sum(1 for r in reqs if r.error is not None and r.error.startswith("refused"))
        t_end = max((r.t_done for r in served), default=0.0)
        t_start = served[0].t_arrival if served else 0.0
        lat = np.array([r.latency * 1e3 for r in served]) if served else np.zeros(1)
        secs = max(t_end - t_start, 1e-12)
        return ServeStats(len(served), secs, len(served) / secs, sum(r.pixels for r in served) / secs / 1e6,
                          float(np.percentile(lat, 50)), float(np.percentile(lat, 99)),
                          nframes / max(nb, 1), nb, peak, self.budget, refused,
                          n - len(served) - refused, list(lat))


class GpuExecutor:
    """Device work of a batch: copies of the ranges to the device, one
    pc_compute_batch launch, copies of the results to the host, an event.
    One context and one stream per in-flight slot (a context's batch calls
    stay on one stream)."""

    def __init__(self, window_radius=7, iterations=5, slots=2, keep_results=False, **params):
        import torch
        from .pcurv import Curvature
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.ctx = [Curvature(1.0, 1.0, 0.0, 0.0, window_radius, iterations, **params) for _ in range(slots)]
        self.keep = keep_results
        self._host = collections.defaultdict(list)   # page-locked result buffers by shape

    def _host_buf(self, shape):
        pool = self._host[shape]
        return pool.pop() if pool else self.torch.empty(shape, dtype=self.torch.float32).pin_memory()

    def launch(self, reqs, slot):
        try:
            return self._launch(reqs, slot)
        except Exception:
            # copies of this batch may be in flight: let them end before the
            # buffers they use are released, and take back its host buffers
            for st in self.streams:
                st.synchronize()
            for r in reqs:
                for t in (r.k1, r.k2, r.normal):
                    if t is not None:
                        self._host[tuple(t.shape)].append(t)
                r.k1 = r.k2 = r.normal = None
            raise

    def _launch(self, reqs, slot):
        torch = self.torch
        s = self.streams[slot]
        frames = []
        with torch.cuda.stream(s), torch.cuda.nvtx.range(f"serve batch of {len(reqs)} frames"):
            for r in reqs:
                H, W = r.depth.shape
                d = torch.empty((H, W), dtype=torch.float32, device="cuda")
                d.copy_(r.depth, non_blocking=True)
                k1 = torch.empty((H, W), dtype=torch.float32, device="cuda")
                k2 = torch.empty((H, W), dtype=torch.float32, device="cuda")
                nrm = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
                frames.append((d, r.intrinsics, k1, k2, nrm))
            self.ctx[slot].batch(frames, stream=s)
            for r, (d, _, k1, k2, nrm) in zip(reqs, frames):
                r.k1, r.k2, r.normal = (self._host_buf(tuple(k1.shape)), self._host_buf(tuple(k2.shape)),
                                        self._host_buf(tuple(nrm.shape)))
                r.k1.copy_(k1, non_blocking=True)
                r.k2.copy_(k2, non_blocking=True)
                r.normal.copy_(nrm, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, frames)

    def done(self, handle):
        return handle[0].query()

    def wait(self, handle, timeout_s):
        if not handle[0].query():
            time.sleep(timeout_s)

    def finish(self, handle, reqs):
        if not self.keep:
            for r in reqs:
                for t in (r.k1, r.k2, r.normal):
                    self._host[tuple(t.shape)].append(t)
                r.k1 = r.k2 = r.normal = None

    def close(self):
        for c in self.ctx:
            c.close()


class PlainExecutor(GpuExecutor):
    """The unbatched baseline: each request is its own pc_compute launch
    (with its copies), in arrival order on one stream."""

    def __init__(self, window_radius=7, iterations=5, keep_results=False, **params):
        super().__init__(window_radius, iterations, 1, keep_results, **params)
        from .pcurv import Curvature
        self._curv = {}
        self._args = (window_radius, iterations, params)

    def _launch(self, reqs, slot):
        torch = self.torch
        s = self.streams[0]
        held = []
        with torch.cuda.stream(s):
            for r in reqs:
                if r.intrinsics not in self._curv:
                    from .pcurv import Curvature
                    rr, tt, pp = self._args
                    self._curv[r.intrinsics] = Curvature(*r.intrinsics, window_radius=rr, iterations=tt, **pp)
                H, W = r.depth.shape
                d = torch.empty((H, W), dtype=torch.float32, device="cuda")
                d.copy_(r.depth, non_blocking=True)
                k1, k2, nrm = self._curv[r.intrinsics](d, stream=s)
                r.k1, r.k2, r.normal = (self._host_buf((H, W)), self._host_buf((H, W)), self._host_buf((H, W, 3)))
                r.k1.copy_(k1, non_blocking=True)
                r.k2.copy_(k2, non_blocking=True)
                r.normal.copy_(nrm, non_blocking=True)
                held.append((d, k1, k2, nrm))
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, held)

    def close(self):
        super().close()
        for c in self._curv.values():
            c.close()


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """arrival times (s) of a Poisson process: cumulative exponential gaps"""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def device_budget(fraction: float = 0.5, reserve_bytes: int = 2 << 30) -> int:
    """device-memory budget for admitted frames: a fraction of the free memory
    left after a reserve"""
    import torch
    free, _ = torch.cuda.mem_get_info()
    return max(int((free - reserve_bytes) * fraction), 1 << 20)
