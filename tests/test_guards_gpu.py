"""Guard bands: every store of every entry point stays inside its buffer.

compute-sanitizer is not available on this machine, so each output is written
into the middle of a larger buffer whose words before and after hold a
sentinel, and the sentinels are checked after the call -- over odd image
shapes (1x1 up to several ragged tiles), window radii (unrolled and run-time),
strides, rejection, every kernel variant (32x8 and 32x4 tiles, 2, 4 and 8
lanes per pixel, compensated sums, 16-bit storage one frame at a time and in
a batch) and every entry point that writes device or host memory."""
import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

GUARD = 256          # elements on each side (1 KB for floats: keeps 16-byte alignment)
SENTINEL = 7.25
SHAPES = [(1, 1), (3, 3), (13, 17), (9, 33), (8, 32), (37, 45), (70, 100)]


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
def frames():
    k = synth.kinect_scene(2)
    return {hw: synth.crop(k, 200, 300, *hw) for hw in SHAPES}


class Guarded:
    """n elements in the middle of a buffer with GUARD sentinels on each side
    (device or pinned host memory)."""

    def __init__(self, n, dtype=None, device="cuda", sentinel=SENTINEL):
        import torch
        dtype = dtype or torch.float32
        self.n, self.sentinel = n, sentinel
        self.buf = torch.full((n + 2 * GUARD,), sentinel, dtype=dtype, device=device)
        if device == "cpu":
            self.buf = self.buf.pin_memory()

    @property
    def ptr(self):
        return self.buf[GUARD:].data_ptr()

    def intact(self):
        b = self.buf.cpu()
        return bool((b[:GUARD] == self.sentinel).all()) and bool((b[GUARD + self.n:] == self.sentinel).all())

    def written(self):
        return not bool((self.buf[GUARD:GUARD + self.n] == self.sentinel).all()) if self.n else True


def ctx(gpu, s, r, **params):
    p = gpu.pc_params_default()
    for k, v in params.items():
        setattr(p, k, v)
    st, c = gpu.pc_create(*map(float, s.intrinsics), r, 5, p)
    assert st == gpu.PC_OK
    return c


def outputs(H, W, device="cuda"):
    return Guarded(H * W, device=device), Guarded(H * W, device=device), Guarded(3 * H * W, device=device)


CONFIGS = [(7, {}), (7, {"tile_height": 4}), (7, {"lanes_per_pixel": 2}), (7, {"lanes_per_pixel": 4}),
           (7, {"lanes_per_pixel": 8}), (1, {}), (12, {}), (15, {}), (7, {"stride": 3}), (5, {"reject": 1}),
           (18, {"stride": 3}), (3, {"kahan": 1}), (7, {"fp64_solve_cond": 1e6, "pivot_tol": 1e-7})]


@pytest.mark.parametrize("r,params", CONFIGS, ids=[f"r{r}-" + "-".join(f"{k}{v}" for k, v in p.items())
                                                  for r, p in CONFIGS])
def test_compute_stays_in_bounds(gpu, frames, r, params):
    import torch
    for (H, W), s in frames.items():
        c = ctx(gpu, s, r, **params)
        d = torch.from_numpy(s.depth).cuda()
        k1, k2, n = outputs(H, W)
        assert gpu.pc_compute(c, d.data_ptr(), H, W, None, k1.ptr, k2.ptr, n.ptr) == gpu.PC_OK
        torch.cuda.synchronize()
        gpu.pc_destroy(c)
        assert k1.intact() and k2.intact() and n.intact(), (H, W)
        assert k1.written() and n.written(), (H, W)


@pytest.mark.parametrize("params", [{}, {"lanes_per_pixel": 4}, {"tile_height": 4}])
@pytest.mark.parametrize("static", [False, True])
def test_batches_stay_in_bounds(gpu, frames, params, static):
    import torch
    c = ctx(gpu, next(iter(frames.values())), 7, **params)
    arr = (gpu.pc_frame * len(frames))()
    held = []
    for i, ((H, W), s) in enumerate(frames.items()):
        d = torch.from_numpy(s.depth).cuda()
        k1, k2, n = outputs(H, W)
        held.append((d, k1, k2, n))
        arr[i] = gpu.pc_frame(d.data_ptr(), H, W, *map(float, s.intrinsics), k1.ptr, k2.ptr, n.ptr)
    call = gpu.pc_compute_batch_static if static else gpu.pc_compute_batch
    assert call(c, arr, len(frames), None) == gpu.PC_OK
    torch.cuda.synchronize()
    gpu.pc_destroy(c)
    for (d, k1, k2, n), hw in zip(held, frames):
        assert k1.intact() and k2.intact() and n.intact(), hw
        assert k1.written() and n.written(), hw


def test_host_entry_points_stay_in_bounds(gpu, frames):
    import torch
    c = ctx(gpu, next(iter(frames.values())), 7)
    arr = (gpu.pc_frame * len(frames))()
    held = []
    for i, ((H, W), s) in enumerate(frames.items()):
        d = torch.from_numpy(s.depth).pin_memory()
        k1, k2, n = outputs(H, W, device="cpu")
        held.append((d, k1, k2, n))
        arr[i] = gpu.pc_frame(d.data_ptr(), H, W, *map(float, s.intrinsics), k1.ptr, k2.ptr, n.ptr)
    assert gpu.pc_compute_host_batch(c, arr, len(frames), None) == gpu.PC_OK
    torch.cuda.synchronize()
    for (d, k1, k2, n), hw in zip(held, frames):
        assert k1.intact() and k2.intact() and n.intact(), hw
    # one small frame (one launch) and frames of several waves (bands of tile rows)
    for s in (list(frames.values())[-1], synth.kinect_scene(5, H=480, W=640), synth.kinect_scene(6, H=1003, W=517)):
        H, W = s.depth.shape
        d = torch.from_numpy(s.depth).pin_memory()
        k1, k2, n = outputs(H, W, device="cpu")
        assert gpu.pc_compute_host(c, d.data_ptr(), H, W, None, k1.ptr, k2.ptr, n.ptr) == gpu.PC_OK
        torch.cuda.synchronize()
        assert k1.intact() and k2.intact() and n.intact(), (H, W)
        assert k1.written() and n.written(), (H, W)
    gpu.pc_destroy(c)


@pytest.mark.parametrize("fmt", [1, 2])
def test_packed_storage_stays_in_bounds(gpu, frames, fmt):
    import torch
    for (H, W), s in frames.items():
        c = ctx(gpu, s, 7)
        d = torch.from_numpy(s.depth).cuda()
        tiles = ((W + 31) // 32) * ((H + 7) // 8)
        packed = Guarded(H * W, dtype=torch.int16, sentinel=12345)
        base = Guarded(tiles)
        assert gpu.pc_pack_depth(c, d.data_ptr(), H, W, fmt, None, packed.ptr, base.ptr) == gpu.PC_OK
        k1, k2, n = outputs(H, W)
        assert gpu.pc_compute_packed(c, packed.ptr, base.ptr, fmt, H, W, None, k1.ptr, k2.ptr, n.ptr) == gpu.PC_OK
        torch.cuda.synchronize()
        gpu.pc_destroy(c)
        assert packed.intact() and base.intact(), (H, W)
        assert k1.intact() and k2.intact() and n.intact(), (H, W)


@pytest.mark.parametrize("r", [3, 5, 11])
@pytest.mark.parametrize("fmt", [1, 2])
def test_packed_batch_stays_in_bounds(gpu, frames, fmt, r):
    """pc_compute_packed_batch over every shape at once (unrolled radii 3 and
    11, run-time radius 5)."""
    import torch
    c = ctx(gpu, next(iter(frames.values())), r)
    arr = (gpu.pc_packed_frame * len(frames))()
    held = []
    for i, ((H, W), s) in enumerate(frames.items()):
        d = torch.from_numpy(s.depth).cuda()
        tiles = ((W + 31) // 32) * ((H + 7) // 8)
        packed = Guarded(H * W, dtype=torch.int16, sentinel=12345)
        base = Guarded(tiles)
        assert gpu.pc_pack_depth(c, d.data_ptr(), H, W, fmt, None, packed.ptr, base.ptr) == gpu.PC_OK
        k1, k2, n = outputs(H, W)
        held.append((packed, base, k1, k2, n))
        arr[i] = gpu.pc_packed_frame(packed.ptr, base.ptr, H, W, *map(float, s.intrinsics), k1.ptr, k2.ptr, n.ptr)
    assert gpu.pc_compute_packed_batch(c, arr, len(frames), fmt, None) == gpu.PC_OK
    torch.cuda.synchronize()
    gpu.pc_destroy(c)
    for (packed, base, k1, k2, n), hw in zip(held, frames):
        assert packed.intact() and base.intact(), hw
        assert k1.intact() and k2.intact() and n.intact(), hw
        assert k1.written() and n.written(), hw


def test_organised_outputs_stay_in_bounds(gpu, frames):
    import torch
    for (H, W), s in frames.items():
        c = ctx(gpu, s, 7)
        d = torch.from_numpy(s.depth).cuda()
        xyz, nrm = Guarded(3 * H * W), Guarded(3 * H * W)
        assert gpu.pc_backproject(c, d.data_ptr(), H, W, None, xyz.ptr) == gpu.PC_OK
        assert gpu.pc_initial_normals(c, d.data_ptr(), H, W, None, nrm.ptr) == gpu.PC_OK
        torch.cuda.synchronize()
        gpu.pc_destroy(c)
        assert xyz.intact() and nrm.intact(), (H, W)
        assert xyz.written() and nrm.written(), (H, W)
