"""Behaviour of the C ABI on the GPU: edge cases of the input, the
host-memory entry point, streams, determinism, and argument errors."""

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


def run(pc, depth, intr, r, T, **kw):
    import torch
    c = pc.Curvature(*intr, window_radius=r, iterations=T, **kw)
    k1, k2, n = c(torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda())
    torch.cuda.synchronize()
    c.close()
    return k1.cpu().numpy(), k2.cpu().numpy(), n.cpu().numpy()


@pytest.mark.parametrize("H,W", [(1, 1), (2, 3), (4, 5), (13, 17), (9, 33), (8, 32)])
def test_tiny_images_vs_oracle(gpu, orc, H, W):
    """Images smaller than a tile, or exactly one tile, with holes."""
    rng = np.random.default_rng(H * 100 + W)
    d = (1.2 + 0.02 * rng.standard_normal((H, W))).astype(np.float32)
    d[rng.random((H, W)) < 0.15] = 0.0
    intr = (60.0, 60.0, W / 2.0, H / 2.0)
    k1, k2, n = run(gpu, d, intr, 3, 3)
    from oracle import parity
    ref = parity.reference(d, orc.params(*intr, r=3, T=3, pivot_tol=1e-5))
    rep = parity.compare(k1, k2, n, ref, pivot_tol=1e-5)
    assert rep.ok(), rep.summary()
    f = ref.field
    assert np.all(np.isnan(k1[f.status == orc.INVALID_CENTRE]))
    assert np.all(np.isnan(k1[f.status == orc.FEW_POINTS]))


def test_invalid_ranges(gpu):
    """0, negative, NaN and infinite ranges are all "no measurement"."""
    d = np.full((24, 40), 1.5, np.float32)
    d[5, 5], d[6, 6], d[7, 7], d[8, 8] = 0.0, -1.0, np.nan, np.inf
    k1, k2, n = run(gpu, d, (50.0, 50.0, 20.0, 12.0), 3, 2)
    for v, u in ((5, 5), (6, 6), (7, 7), (8, 8)):
        assert np.isnan(k1[v, u]) and np.isnan(k2[v, u]) and np.isnan(n[v, u]).all()
    # the plane around them is still exact
    assert np.abs(k1[15:20, 15:30]).max() < 1e-3
    assert np.allclose(n[15:20, 15:30], [0, 0, 1], atol=1e-5)


def test_all_invalid_image(gpu):
    k1, k2, n = run(gpu, np.zeros((20, 50), np.float32), (50.0, 50.0, 25.0, 10.0), 7, 5)
    assert np.isnan(k1).all() and np.isnan(k2).all() and np.isnan(n).all()


def test_empty_image(gpu):
    import torch
    c = gpu.Curvature(50.0, 50.0, 0.0, 0.0, 3, 2)
    d = torch.zeros((0, 10), device="cuda")
    k1, k2, n = c(d)
    assert k1.shape == (0, 10)
    c.close()


@pytest.mark.parametrize("H,W", [(8, 16384), (16384, 4)])
def test_maximum_dimensions(gpu, orc, H, W):
    """The largest allowed side (PC_MAX_DIM): sampled pixels against the oracle."""
    rng = np.random.default_rng(0)
    d = (2.0 + 0.001 * rng.standard_normal((H, W))).astype(np.float32)
    intr = (525.0, 525.0, W / 2.0, H / 2.0)
    k1, k2, n = run(gpu, d, intr, 3, 3)
    uv = np.stack([rng.integers(0, W, 200), rng.integers(0, H, 200)], 1).astype(np.int32)
    uv = np.concatenate([uv, [[0, 0], [W - 1, H - 1], [W - 1, 0]]]).astype(np.int32)
    from oracle import parity
    ref = parity.reference(d, orc.params(*intr, r=3, T=3, pivot_tol=1e-5), uv=uv)
    rep = parity.compare(k1[uv[:, 1], uv[:, 0]], k2[uv[:, 1], uv[:, 0]], n[uv[:, 1], uv[:, 0]], ref,
                         pivot_tol=1e-5)
    assert rep.ok() and rep.n_well_posed > 0.5 * len(uv), rep.summary()


def test_host_entry_matches_device_entry(gpu):
    import torch
    s = synth.crop(synth.kinect_scene(2), 100, 100, 64, 96)
    c = gpu.Curvature(*s.intrinsics, window_radius=7, iterations=5)
    k1, k2, n = c(torch.from_numpy(s.depth).cuda())
    hd = torch.from_numpy(s.depth).pin_memory()
    hk1, hk2 = torch.empty(64, 96).pin_memory(), torch.empty(64, 96).pin_memory()
    hn = torch.empty(64, 96, 3).pin_memory()
    c.compute_host(hd, hk1, hk2, hn)
    torch.cuda.synchronize()
    assert np.array_equal(hk1.numpy(), k1.cpu().numpy(), equal_nan=True)
    assert np.array_equal(hk2.numpy(), k2.cpu().numpy(), equal_nan=True)
    assert np.array_equal(hn.numpy(), n.cpu().numpy(), equal_nan=True)
    # pageable host memory and a larger image (staging buffers grow)
    s2 = synth.kinect_scene(2, H=120, W=160)
    hk1b, hk2b = torch.empty(120, 160), torch.empty(120, 160)
    c.compute_host(torch.from_numpy(s2.depth), hk1b, hk2b, None)
    torch.cuda.synchronize()
    c2 = gpu.Curvature(*s.intrinsics, window_radius=7, iterations=5)   # same parameters as c
    ref1, ref2, _ = c2(torch.from_numpy(s2.depth).cuda(), want_normal=False)
    torch.cuda.synchronize()
    assert np.array_equal(hk1b.numpy(), ref1.cpu().numpy(), equal_nan=True)
    assert np.array_equal(hk2b.numpy(), ref2.cpu().numpy(), equal_nan=True)
    c.close()
    c2.close()


@pytest.mark.parametrize("H,W,r,params", [(480, 640, 7, {}), (720, 1280, 7, {}), (480, 640, 7, {"lanes_per_pixel": 2}),
                                          (2000, 160, 7, {}), (480, 640, 12, {}), (480, 640, 3, {"tile_height": 4})])
def test_host_entry_in_bands_matches_device_entry(gpu, H, W, r, params):
    """Frames of several waves of CTAs go through pc_compute_host in bands of
    tile rows (copies overlapping the kernels): the same bits as pc_compute,
    for two frames enqueued back to back on one stream (the second reuses the
    staging buffers the first is still copying out of) and without normals."""
    import torch
    frames = [synth.kinect_scene(40 + j, H=H, W=W) for j in range(2)]
    c = gpu.Curvature(*frames[0].intrinsics, window_radius=r, iterations=5, **params)
    ref = []
    for s in frames:
        k1, k2, n = c(torch.from_numpy(s.depth).cuda())
        ref.append((k1.cpu().numpy(), k2.cpu().numpy(), n.cpu().numpy()))
    hd = [torch.from_numpy(s.depth).pin_memory() for s in frames]
    out = [(torch.empty(H, W).pin_memory(), torch.empty(H, W).pin_memory(), torch.empty(H, W, 3).pin_memory())
           for _ in frames]
    stream = torch.cuda.Stream()
    for d, (hk1, hk2, hn) in zip(hd, out):
        c.compute_host(d, hk1, hk2, hn, stream=stream)
    stream.synchronize()
    for (a1, a2, an), (hk1, hk2, hn) in zip(ref, out):
        assert np.array_equal(hk1.numpy(), a1, equal_nan=True)
        assert np.array_equal(hk2.numpy(), a2, equal_nan=True)
        assert np.array_equal(hn.numpy(), an, equal_nan=True)
    hk1, hk2 = torch.full((H, W), 3.0).pin_memory(), torch.full((H, W), 3.0).pin_memory()
    c.compute_host(hd[1], hk1, hk2, None, stream=stream)
    stream.synchronize()
    assert np.array_equal(hk1.numpy(), ref[1][0], equal_nan=True)
    assert np.array_equal(hk2.numpy(), ref[1][1], equal_nan=True)
    c.close()


def test_without_normals_and_determinism(gpu):
    import torch
    s = synth.crop(synth.kinect_scene(4), 200, 300, 40, 64)
    c = gpu.Curvature(*s.intrinsics, window_radius=7, iterations=5)
    d = torch.from_numpy(s.depth).cuda()
    a1, a2, an = c(d)
    b1, b2, bn = c(d, want_normal=False)
    assert bn is None
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        c1, c2_, cn = c(d, stream=side)
    side.synchronize()
    torch.cuda.synchronize()
    for x, y in ((a1, b1), (a2, b2), (a1, c1), (a2, c2_), (an, cn)):
        assert torch.equal(torch.nan_to_num(x, 7.0), torch.nan_to_num(y, 7.0))
    c.close()


def test_argument_errors_leave_outputs_untouched(gpu):
    import torch
    c = gpu.Curvature(525.0, 525.0, 10.0, 10.0, 3, 2)
    d = torch.ones((16, 16), device="cuda")
    k1 = torch.full((16, 16), 3.0, device="cuda")
    k2 = torch.full((16, 16), 3.0, device="cuda")
    host = torch.ones((16, 16))
    # a host pointer where device memory is required
    st = gpu.pc_compute(c.ctx, host.data_ptr(), 16, 16, None, k1.data_ptr(), k2.data_ptr(), None)
    assert st == gpu.PC_ERR_INVALID_ARG
    # misaligned device pointer
    st = gpu.pc_compute(c.ctx, d.data_ptr() + 2, 16, 16, None, k1.data_ptr(), k2.data_ptr(), None)
    assert st == gpu.PC_ERR_INVALID_ARG
    # NULL output
    st = gpu.pc_compute(c.ctx, d.data_ptr(), 16, 16, None, None, k2.data_ptr(), None)
    assert st == gpu.PC_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((k1 == 3.0).all()) and bool((k2 == 3.0).all())
    with pytest.raises(ValueError):
        c(torch.ones((16, 16), device="cuda", dtype=torch.float64))
    c.close()


def test_contexts_on_concurrent_streams(gpu):
    """Four contexts on four streams, each with per-frame, batch and host-batch
    calls in flight at once, give the bits of the same calls run one after
    another on the default stream."""
    import torch
    scenes = [synth.kinect_scene(60 + i, H=h, W=w) for i, (h, w) in
              enumerate([(240, 320), (480, 640), (424, 512), (120, 160)])]

    def work(c, s, stream):
        d = torch.from_numpy(s.depth).cuda()
        a = c(d, stream=stream)
        frames = [(d, s.intrinsics, torch.empty_like(d), torch.empty_like(d),
                   torch.empty(d.shape + (3,), device="cuda")) for _ in range(2)]
        c.batch(frames, stream=stream)
        hf = [(torch.from_numpy(s.depth).pin_memory(), s.intrinsics, torch.empty(d.shape).pin_memory(),
               torch.empty(d.shape).pin_memory(), torch.empty(d.shape + (3,)).pin_memory())]
        c.host_batch(hf, stream=stream)
        return d, a, frames, hf

    def results(out):
        d, a, frames, hf = out
        return ([t.cpu().numpy() for t in a] + [t.cpu().numpy() for f in frames for t in f[2:]] +
                [t.numpy().copy() for t in hf[0][2:]])

    ctxs = [gpu.Curvature(*s.intrinsics, window_radius=7, iterations=5) for s in scenes]
    seq = []
    for c, s in zip(ctxs, scenes):
        out = work(c, s, None)
        torch.cuda.synchronize()
        seq.append(results(out))
    streams = [torch.cuda.Stream() for _ in scenes]
    outs = [work(c, s, st) for c, s, st in zip(ctxs, scenes, streams)]
    torch.cuda.synchronize()
    for out, ref in zip(outs, seq):
        for x, y in zip(results(out), ref):
            assert np.array_equal(x, y, equal_nan=True)
    for c in ctxs:
        c.close()
