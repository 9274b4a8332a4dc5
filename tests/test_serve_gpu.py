"""The serving loop on the GPU: frames of four resolutions arriving faster
than they are served are batched continuously; every result is the same as
the frame computed alone (bit for bit, hence within any tolerance), with the
batched executor and with the one-launch-per-frame baseline; a request the
library rejects fails alone while the others are served."""
import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_00385_gb300 import build
    build.build()
    import paper_1707_00385_gb300 as pc
    pc.load()
    return pc


@pytest.fixture(scope="module")
def pool():
    import torch
    sizes = [(240, 320, "kinect"), (424, 512, "tof"), (480, 640, "kinect"), (720, 1280, "kinect")]
    frames = []
    for j, (h, w, noise) in enumerate(sizes):
        s = synth.kinect_scene(500 + j, H=h, W=w, noise=noise, nprims=8)
        frames.append((torch.from_numpy(s.depth).pin_memory(), s.intrinsics))
    return frames


def make_trace(pool, n, rate, seed):
    from paper_1707_00385_gb300.serve import Request, poisson_arrivals
    rng = np.random.default_rng(seed)
    t = poisson_arrivals(n, rate, seed)
    return [Request(i, *pool[rng.integers(0, len(pool))], float(t[i])) for i in range(n)]


def alone(gpu, r):
    import torch
    c = gpu.Curvature(*r.intrinsics, window_radius=7, iterations=5)
    k1, k2, n = c(r.depth.cuda())
    torch.cuda.synchronize()
    c.close()
    return k1.cpu().numpy(), k2.cpu().numpy(), n.cpu().numpy()


@pytest.mark.parametrize("plain", [False, True])
def test_results_same_alone_and_in_the_mix(gpu, pool, plain):
    from paper_1707_00385_gb300.serve import GpuExecutor, PlainExecutor, Server
    reqs = make_trace(pool, 40, 4000.0, seed=3)
    if plain:
        ex = PlainExecutor(keep_results=True)
        srv = Server(ex, budget_bytes=1 << 31, max_batch_frames=1, inflight=64)
    else:
        ex = GpuExecutor(keep_results=True)
        srv = Server(ex, budget_bytes=1 << 31, max_batch_frames=16)
    stats = srv.run(reqs)
    print(stats.as_dict())
    assert stats.requests == 40 and stats.p50_ms <= stats.p99_ms
    if not plain:
        assert stats.mean_batch > 1.5       # arrivals during batches were batched together
    ref = {}
    for r in reqs:
        key = id(r.depth)
        if key not in ref:
            ref[key] = alone(gpu, r)
        a1, a2, an = ref[key]
        assert np.array_equal(r.k1.numpy(), a1, equal_nan=True)
        assert np.array_equal(r.k2.numpy(), a2, equal_nan=True)
        assert np.array_equal(r.normal.numpy(), an, equal_nan=True)
    ex.close()


@pytest.mark.parametrize("plain", [False, True])
def test_a_rejected_request_fails_alone(gpu, pool, plain):
    """Request 7 carries intrinsics the library rejects (fx = 0): its batch
    fails to launch, its requests are retried one per batch, request 7 fails
    with the library's status and every other result equals the frame alone."""
    from paper_1707_00385_gb300.serve import GpuExecutor, PlainExecutor, Request, Server
    reqs = make_trace(pool, 24, 4000.0, seed=8)
    bad = reqs[7]
    reqs[7] = Request(bad.rid, bad.depth, (0.0,) + tuple(bad.intrinsics[1:]), bad.t_arrival)
    if plain:
        ex = PlainExecutor(keep_results=True)
        srv = Server(ex, budget_bytes=1 << 31, max_batch_frames=1, inflight=64)
    else:
        ex = GpuExecutor(keep_results=True)
        srv = Server(ex, budget_bytes=1 << 31, max_batch_frames=16)
    stats = srv.run(reqs)
    print(stats.as_dict())
    assert reqs[7].error is not None and "invalid argument (1)" in reqs[7].error, reqs[7].error
    assert stats.failed == 1 and stats.refused == 0 and stats.requests == 23
    for r in reqs:
        if r is reqs[7]:
            continue
        assert r.error is None
        a1, a2, an = alone(gpu, r)
        assert np.array_equal(r.k1.numpy(), a1, equal_nan=True)
        assert np.array_equal(r.k2.numpy(), a2, equal_nan=True)
        assert np.array_equal(r.normal.numpy(), an, equal_nan=True)
    ex.close()


def test_budget_from_free_memory(gpu):
    from paper_1707_00385_gb300.serve import device_budget
    import torch
    b = device_budget(0.5)
    free, _ = torch.cuda.mem_get_info()
    assert 0 < b <= free
