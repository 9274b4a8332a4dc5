"""pc_compute_batch_static, the batch entry point for callers that cannot
allocate device memory (their host program owns all device memory, or a
latency-bound loop cannot afford cudaMalloc).  Its scratch is a fixed array
inside the library.  Called through the C ABI, it must give what
pc_compute_batch gives on the same frames, on two calls in a row (the array
is shared by every call and keeps the previous call's contents).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
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


def make_frames(torch, scenes):
    out = []
    for s in scenes:
        d = torch.from_numpy(s.depth).cuda()
        out.append((d, s.intrinsics, torch.full(d.shape, 9.0, device="cuda"),
                    torch.full(d.shape, 9.0, device="cuda"), torch.full(d.shape + (3,), 9.0, device="cuda")))
    return out


def table(pc, frames):
    arr = (pc.pc_frame * len(frames))()
    for i, (d, intr, a, b, n) in enumerate(frames):
        arr[i] = pc.pc_frame(d.data_ptr(), d.shape[0], d.shape[1], *map(float, intr), a.data_ptr(),
                             b.data_ptr(), n.data_ptr())
    return arr


def same_bits(a, b):
    """equal element by element, NaN where the other is NaN"""
    import torch
    return torch.equal(torch.isnan(a), torch.isnan(b)) and torch.equal(torch.nan_to_num(a, 3.0),
                                                                       torch.nan_to_num(b, 3.0))


@pytest.mark.parametrize("lanes", [0, 4])
def test_no_alloc_batch_matches_batch_on_two_calls(gpu, lanes):
    """lanes = 4 forces a lane group of 4 threads per pixel (the moment sums
    in another order): both entry points must run that variant."""
    import torch
    sets = [
        [synth.kinect_scene(7, H=120, W=160), synth.kinect_scene(8, H=240, W=320, noise="tof"),
         synth.crop(synth.kinect_scene(9), 100, 200, 37, 53)],
        [synth.kinect_scene(10, H=480, W=640), synth.crop(synth.kinect_scene(11), 0, 0, 9, 31)],
    ]
    prm = gpu.pcurv.pc_params_default()
    prm.lanes_per_pixel = lanes
    st, ctx = gpu.pc_create(525.0, 525.0, 0.0, 0.0, 7, 5, prm)
    assert st == gpu.PC_OK
    try:
        for scenes in sets:                      # two calls in a row, different frames
            ref = make_frames(torch, scenes)
            new = make_frames(torch, scenes)
            assert gpu.pc_compute_batch(ctx, table(gpu, ref), len(ref), None) == gpu.PC_OK
            st = gpu.pc_compute_batch_static(ctx, table(gpu, new), len(new), None)
            assert st == gpu.PC_OK, gpu.pc_last_error(ctx)
            torch.cuda.synchronize()
            for (_, _, a1, a2, an), (_, _, b1, b2, bn) in zip(ref, new):
                assert same_bits(a1, b1) and same_bits(a2, b2) and same_bits(an, bn)
                assert torch.isfinite(a1).float().mean() > 0.5     # the frames were computed
    finally:
        gpu.pc_destroy(ctx)


def test_no_alloc_batch_rejects_too_many_frames(gpu):
    import torch
    st, ctx = gpu.pc_create(525.0, 525.0, 0.0, 0.0, 3, 2)
    try:
        d = torch.ones((8, 8), device="cuda")
        k = torch.empty((8, 8), device="cuda")
        n = gpu.pcurv.PC_STATIC_MAX_FRAMES + 1
        arr = (gpu.pc_frame * n)()
        for i in range(n):
            arr[i] = gpu.pc_frame(d.data_ptr(), 8, 8, 50.0, 50.0, 4.0, 4.0, k.data_ptr(), k.data_ptr(), None)
        assert gpu.pc_compute_batch_static(ctx, arr, n, None) == gpu.PC_ERR_INVALID_ARG
        assert "exceed" in gpu.pc_last_error(ctx)
        assert gpu.pc_compute_batch_static(ctx, None, 0, None) == gpu.PC_OK
    finally:
        gpu.pc_destroy(ctx)
