"""Tile shapes (32x8 and 32x4 pixels per CTA, one thread per pixel) and the
autotuner: the shape is a performance choice only, results are the same bits
(lane groups, which the autotuner may also choose: tests/test_lanes_gpu.py)."""
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


def run(gpu, s, th, r=7, **kw):
    import torch
    c = gpu.Curvature(*s.intrinsics, window_radius=r, iterations=5, tile_height=th, **kw)
    out = c(torch.from_numpy(s.depth).cuda())
    torch.cuda.synchronize()
    c.close()
    return [o.cpu().numpy() for o in out]


@pytest.mark.parametrize("H,W,r,kw", [(480, 640, 7, {}), (61, 77, 3, {}), (120, 160, 11, {}),
                                      (100, 90, 7, {"stride": 2}), (50, 70, 5, {"reject": 1})])
def test_tile_shapes_give_the_same_bits(gpu, H, W, r, kw):
    s = synth.kinect_scene(31, H=H, W=W) if H >= 100 and W >= 100 else \
        synth.crop(synth.kinect_scene(31), 100, 100, H, W)
    a, b = run(gpu, s, 8, r, **kw), run(gpu, s, 4, r, **kw)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)


def test_batch_with_either_tile_shape(gpu):
    import torch
    scenes = [synth.kinect_scene(40 + i, H=h, W=w) for i, (h, w) in enumerate([(240, 320), (480, 640), (120, 160)])]
    outs = {}
    for th in (8, 4):
        c = gpu.Curvature(1.0, 1.0, 0.0, 0.0, window_radius=7, iterations=5, tile_height=th)
        args = []
        for s in scenes:
            d = torch.from_numpy(s.depth).cuda()
            args.append((d, s.intrinsics, torch.empty_like(d), torch.empty_like(d), torch.empty(d.shape + (3,), device="cuda")))
        c.batch(args)
        torch.cuda.synchronize()
        outs[th] = [[t.cpu().numpy() for t in a[2:]] for a in args]
        c.close()
    for fa, fb in zip(outs[8], outs[4]):
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y, equal_nan=True)


def test_plan_heuristic_and_autotune(gpu):
    import torch
    s = synth.kinect_scene(3, H=480, W=640)
    c = gpu.Curvature(*s.intrinsics, window_radius=7, iterations=5)
    assert c.tile_height(480, 640) == 8      # 1200 tiles of 32x8: plenty per SM
    assert c.tile_height(60, 80) == 4        # 24 tiles: too few
    assert c.lanes_per_pixel(60, 80) == 1    # the heuristic keeps one lane per pixel
    small = synth.crop(s, 0, 0, 60, 80)
    # the autotuner may also pick a lane group (32 x 8/lanes tiles)
    variants = ((1, 8), (1, 4), (2, 4), (4, 2), (8, 1))
    th = c.autotune(torch.from_numpy(small.depth).cuda())
    assert (c.lanes_per_pixel(60, 80), th) in variants and c.tile_height(60, 80) == th
    th2 = c.autotune(torch.from_numpy(s.depth).cuda())
    assert (c.lanes_per_pixel(480, 640), th2) in variants and c.tile_height(480, 640) == th2
    print("autotuned: 60x80 ->", th, c.lanes_per_pixel(60, 80), "640x480 ->", th2, c.lanes_per_pixel(480, 640))
    c.close()
