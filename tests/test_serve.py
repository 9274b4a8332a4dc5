"""The serving dispatcher on the CPU: a deterministic arrival trace, a fake
clock and a fake executor that runs batches one after another at a fixed
pixel rate.  Checks continuous batching, admission by the memory budget,
batch limits, order, the latency bookkeeping, and failures injected on the
host (refused frames, launches that raise, batches that report an error)."""
import numpy as np

from paper_1707_00385_gb300.serve import BYTES_PER_PIXEL, Request, Server, poisson_arrivals


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeExecutor:
    """A GPU that runs launched batches in order at `rate` pixels/s, plus a
    fixed cost per launch."""

    def __init__(self, clock, rate=5e8, per_launch=20e-6):
        self.clock, self.rate, self.per_launch = clock, rate, per_launch
        self.busy_until = 0.0
        self.launches = []

    def launch(self, batch, slot):
        start = max(self.clock.t, self.busy_until)
        end = start + self.per_launch + sum(r.pixels for r in batch) / self.rate
        self.busy_until = end
        self.launches.append((slot, [r.rid for r in batch], start, end))
        return end

    def done(self, end):
        return self.clock.t >= end

    def wait(self, end, timeout):
        self.clock.t = min(end, self.clock.t + timeout) if end > self.clock.t else self.clock.t + 1e-6

    def finish(self, end, reqs):
        pass


class Frame:
    def __init__(self, H, W):
        self.shape = (H, W)


SIZES = [(240, 320), (424, 512), (480, 640), (720, 1280)]


def trace(n, rate, seed=0):
    rng = np.random.default_rng(seed)
    t = poisson_arrivals(n, rate, seed)
    return [Request(i, Frame(*SIZES[rng.integers(0, 4)]), (1.0, 1.0, 0.0, 0.0), float(t[i])) for i in range(n)]


def serve(reqs, **kw):
    clk = FakeClock()
    ex = FakeExecutor(clk, rate=kw.pop("rate", 5e8))
    srv = Server(ex, **kw)
    stats = srv.run(reqs, clock=clk, sleep=clk.sleep)
    return stats, ex


def test_every_request_completes_in_order_of_events():
    reqs = trace(300, 1500)
    stats, ex = serve(reqs, budget_bytes=1 << 32)
    assert stats.requests == 300
    for r in reqs:
        assert r.t_arrival <= r.t_admit <= r.t_done
    assert stats.p50_ms <= stats.p99_ms
    # admission is FIFO
    admitted = [rid for _, rids, _, _ in ex.launches for rid in rids]
    assert admitted == sorted(admitted)


def test_continuous_batching_under_load():
    """Above capacity the queue builds up; requests that arrive while batches
    run are admitted together into the next batch."""
    reqs = trace(400, 3000)          # ~3000 frames/s offered, ~1300 frames/s served
    stats, ex = serve(reqs, budget_bytes=1 << 33, max_batch_frames=64)
    assert stats.mean_batch > 4
    assert max(len(rids) for _, rids, _, _ in ex.launches) <= 64
    # two slots alternate, and the GPU is never idle while requests wait
    slots = [s for s, _, _, _ in ex.launches]
    assert set(slots) == {0, 1}
    assert stats.mpixel_per_s > 0.95 * 5e8 / 1e6


def test_light_load_serves_one_frame_per_batch():
    reqs = trace(50, 20)              # far below capacity
    stats, ex = serve(reqs, budget_bytes=1 << 32)
    assert stats.mean_batch == 1.0
    svc = np.array([(e - s) for _, _, s, e in ex.launches]) * 1e3
    assert stats.p99_ms < svc.max() + 1.0


def test_memory_budget_bounds_admission():
    reqs = trace(200, 5000)
    one = 1280 * 720 * BYTES_PER_PIXEL
    stats, ex = serve(reqs, budget_bytes=3 * one)
    assert stats.peak_device_bytes <= 3 * one
    assert stats.requests == 200 and stats.refused == 0 and stats.failed == 0


def test_frames_larger_than_the_budget_are_refused_alone():
    reqs = trace(60, 500, seed=2)
    budget = 640 * 480 * BYTES_PER_PIXEL      # 1280 x 720 frames cannot fit
    big = [r for r in reqs if r.pixels > 640 * 480]
    assert big
    stats, ex = serve(reqs, budget_bytes=budget)
    for r in reqs:
        if r in big:
            assert r.error.startswith("refused") and r.t_done == r.t_admit
        else:
            assert r.error is None and r.t_arrival <= r.t_admit <= r.t_done
    assert stats.refused == len(big) and stats.requests == len(reqs) - len(big) and stats.failed == 0
    launched = {rid for _, rids, _, _ in ex.launches for rid in rids}
    assert not launched & {r.rid for r in big}


class FailingExecutor(FakeExecutor):
    """Launching a batch that holds a bad request raises (as the library does
    for an argument it rejects); a batch holding a request listed in
    `fail_done` reports an error when it completes."""

    def __init__(self, clock, bad=(), fail_done=(), **kw):
        super().__init__(clock, **kw)
        self.bad, self.fail_done = set(bad), set(fail_done)
        self.attempts = []

    def launch(self, batch, slot):
        self.attempts.append([r.rid for r in batch])
        if any(r.rid in self.bad for r in batch):
            raise RuntimeError("pc_compute_batch: PC_ERR_INVALID_ARG (1)")
        end = super().launch(batch, slot)
        return (end, [r.rid for r in batch])

    def done(self, h):
        end, rids = h
        if self.clock.t >= end and any(rid in self.fail_done for rid in rids):
            raise RuntimeError("device work failed")
        return super().done(end)

    def wait(self, h, timeout):
        super().wait(h[0], timeout)


def serve_failing(reqs, **kw):
    clk = FakeClock()
    ex = FailingExecutor(clk, bad=kw.pop("bad", ()), fail_done=kw.pop("fail_done", ()))
    stats = Server(ex, **kw).run(reqs, clock=clk, sleep=clk.sleep)
    return stats, ex


def test_a_bad_request_fails_alone_and_serving_goes_on():
    reqs = trace(300, 3000, seed=5)          # loaded: the bad requests share batches with others
    bad = {17, 150, 151}
    stats, ex = serve_failing(reqs, budget_bytes=1 << 33, bad=bad)
    for r in reqs:
        if r.rid in bad:
            assert "PC_ERR_INVALID_ARG" in r.error and r.t_done >= r.t_admit
        else:
            assert r.error is None and r.t_done is not None
    assert stats.failed == len(bad) and stats.requests == len(reqs) - len(bad)
    # the batches that held a bad request were retried one request per batch
    retried = [a for a in ex.attempts if len(a) == 1 and any(b in a for b in bad)]
    assert len(retried) == len(bad)
    served = [rid for _, rids, _, _ in ex.launches for rid in rids]
    assert sorted(served) == sorted(r.rid for r in reqs if r.rid not in bad)


def test_completion_errors_fail_their_batch_and_return_its_memory():
    reqs = trace(200, 3000, seed=6)
    one = 1280 * 720 * BYTES_PER_PIXEL
    stats, ex = serve_failing(reqs, budget_bytes=4 * one, fail_done={40})
    hit = next(rids for _, rids, _, _ in ex.launches if 40 in rids)
    for r in reqs:
        if r.rid in hit:
            assert r.error == "RuntimeError: device work failed"
        else:
            assert r.error is None
    assert stats.failed == len(hit) and stats.requests == len(reqs) - len(hit)
    assert stats.peak_device_bytes <= 4 * one   # the failed batch's memory came back


def test_pixel_limit_per_batch():
    reqs = trace(200, 5000)
    stats, ex = serve(reqs, budget_bytes=1 << 33, max_batch_pixels=1_000_000)
    for _, rids, _, _ in ex.launches:
        px = sum(reqs[i].depth.shape[0] * reqs[i].depth.shape[1] for i in rids)
        assert len(rids) == 1 or px <= 1_000_000


def test_deterministic_for_a_trace():
    a, _ = serve(trace(150, 2000, seed=4), budget_bytes=1 << 32)
    b, _ = serve(trace(150, 2000, seed=4), budget_bytes=1 << 32)
    assert a.as_dict() == b.as_dict()


def test_poisson_arrivals_rate():
    t = poisson_arrivals(20000, 2000.0, 1)
    assert np.all(np.diff(t) > 0)
    assert abs(20000 / t[-1] - 2000.0) < 60
