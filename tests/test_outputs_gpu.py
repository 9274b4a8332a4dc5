"""The organised outputs on the GPU (point cloud, initial-normal field) and the
pipelined host-memory batch, through the C ABI, against the FP64 oracle and
against the device path."""
import types

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
def scene():
    return synth.kinect_scene(8)


def holes(depth, seed):
    """the same range image with NaN, infinite and negative ranges sprinkled in"""
    rng = np.random.default_rng(seed)
    d = depth.copy()
    m = rng.random(d.shape)
    d[m < 0.01] = np.nan
    d[(m >= 0.01) & (m < 0.015)] = np.inf
    d[(m >= 0.015) & (m < 0.02)] = -0.5
    return d


# ---- organised point cloud ---------------------------------------------------

def backproject(pc, depth, intr, offset=0):
    """pc_backproject; offset > 0 places the output 4*offset bytes into a larger buffer
    (breaks 16-byte alignment, so the scalar form runs)"""
    import torch
    H, W = depth.shape
    c = pc.Curvature(*intr)
    d = torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda()
    buf = torch.full((H * W * 3 + offset,), 7.0, device="cuda")
    xyz = buf[offset:].view(H, W, 3)
    c.backproject(d, xyz)
    torch.cuda.synchronize()
    c.close()
    out = buf.cpu().numpy()
    assert np.all(out[:offset] == 7.0)
    return out[offset:].reshape(H, W, 3)


def check_points(xyz, ref):
    bad = np.isnan(ref)
    assert np.array_equal(np.isnan(xyz), bad)
    # three correctly rounded operations: within 2 ulp of the exact coordinate
    err = np.abs(xyz[~bad].astype(np.float64) - ref[~bad])
    assert np.all(err <= 2.0 ** -22 * np.abs(ref[~bad]) + 1e-30)


@pytest.mark.parametrize("shape", [(480, 640), (37, 53), (1, 1), (3, 4), (5, 7), (0, 9)])
def test_backproject_matches_oracle(gpu, orc, scene, shape):
    H, W = shape
    d = holes(scene.depth, H * 1000 + W)[:H, :W] if H else np.zeros((0, W), np.float32)
    xyz = backproject(gpu, d, scene.intrinsics)
    assert xyz.shape == (H, W, 3)
    if H * W:
        check_points(xyz, orc.backproject_image(d, orc.params(*scene.intrinsics, r=3, T=0)))


def test_backproject_vector_and_scalar_forms_agree(gpu, scene):
    d = holes(scene.depth, 5)
    a = backproject(gpu, d, scene.intrinsics)          # 16-byte aligned, W % 4 == 0: vector form
    b = backproject(gpu, d, scene.intrinsics, offset=1)  # scalar form
    assert np.array_equal(a, b, equal_nan=True)


# ---- initial-normal field ------------------------------------------------------

def initial_normals(pc, depth, intr, **kw):
    import torch
    c = pc.Curvature(*intr, **kw)
    n = c.initial_normals(torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda())
    torch.cuda.synchronize()
    c.close()
    return n.cpu().numpy()


@pytest.mark.parametrize("nr", [1, 3, 5, 8])
def test_initial_normals_match_oracle(gpu, orc, scene, nr):
    from oracle import parity
    d = holes(scene.depth, 11)
    n = initial_normals(gpu, d, scene.intrinsics, normal_radius=nr)
    ref = parity.normal_reference(d, orc.params(*scene.intrinsics, r=3, T=0, rn=nr))
    rep = parity.compare_normals(n, ref)
    print(rep.summary())
    assert rep.ok(), rep.summary()
    assert rep.n_well_posed > 0.95 * rep.n_valid_oracle
    assert np.isnan(n).all(-1).sum() + np.isfinite(n).all(-1).sum() == n.shape[0] * n.shape[1]


@pytest.mark.parametrize("shape", [(37, 53), (1, 1), (2, 9), (9, 2), (8, 32)])
def test_initial_normals_ragged_and_tiny(gpu, orc, scene, shape):
    from oracle import parity
    H, W = shape
    d = holes(scene.depth[200:200 + H, 300:300 + W], H + W)
    n = initial_normals(gpu, d, scene.intrinsics)
    ref = parity.normal_reference(d, orc.params(*scene.intrinsics, r=3, T=0))
    rep = parity.compare_normals(n, ref)
    assert rep.ok(), rep.summary()


def test_initial_normals_are_where_the_iterations_start(gpu, scene):
    """pc_compute with no iterations returns the initial normal as its normal
    wherever its window is valid: the same bits as pc_initial_normals."""
    import torch
    d = holes(scene.depth, 12)
    n0 = initial_normals(gpu, d, scene.intrinsics)
    c = gpu.Curvature(*scene.intrinsics, window_radius=3, iterations=0)
    _, _, n = c(torch.from_numpy(d).cuda())
    torch.cuda.synchronize()
    c.close()
    n = n.cpu().numpy()
    fin = np.isfinite(n).all(-1)
    assert fin.mean() > 0.9
    assert np.array_equal(n[fin], n0[fin])
    # where pc_compute gives NaN but the field does not, the window check failed:
    # fewer than 6 valid points in the 7 x 7 window
    extra = ~fin & np.isfinite(n0).all(-1)
    valid = np.isfinite(d) & (d > 0)
    pad = np.pad(valid, 3)
    cnt = sum(pad[3 + dv:3 + dv + d.shape[0], 3 + du:3 + du + d.shape[1]] for dv in range(-3, 4)
              for du in range(-3, 4))
    assert np.all(cnt[extra] < 6)


@pytest.mark.parametrize("H,W", [(720, 1280), (1200, 1600), (1600, 2560)])
def test_initial_normals_every_tile_height(gpu, H, W):
    """Larger images take taller tiles (two, four, eight pixels per thread on
    a 152-SM GPU): the field keeps the same bits as the normals pc_compute
    starts from (T = 0), which the oracle checks."""
    import torch
    s = synth.kinect_scene(21, H=H, W=W)
    d = holes(s.depth, 13)
    n0 = initial_normals(gpu, d, s.intrinsics)
    c = gpu.Curvature(*s.intrinsics, window_radius=3, iterations=0)
    _, _, n = c(torch.from_numpy(d).cuda())
    torch.cuda.synchronize()
    c.close()
    n = n.cpu().numpy()
    fin = np.isfinite(n).all(-1)
    assert fin.mean() > 0.9
    assert np.array_equal(n[fin], n0[fin])
    assert np.isnan(n0).all(-1).sum() + np.isfinite(n0).all(-1).sum() == H * W


# ---- pipelined host-memory batch --------------------------------------------------

def host_frames(scene_list, with_normal):
    import torch
    out = []
    for i, s in enumerate(scene_list):
        H, W = s.depth.shape
        out.append((torch.from_numpy(s.depth).pin_memory(), s.intrinsics, torch.empty((H, W)).pin_memory(),
                    torch.empty((H, W)).pin_memory(),
                    torch.empty((H, W, 3)).pin_memory() if with_normal[i] else None))
    return out


def device_results(pc, s, r=7, T=5):
    import torch
    c = pc.Curvature(*s.intrinsics, window_radius=r, iterations=T)
    k1, k2, n = c(torch.from_numpy(s.depth).cuda())
    torch.cuda.synchronize()
    c.close()
    return k1.cpu().numpy(), k2.cpu().numpy(), n.cpu().numpy()


def test_host_batch_equals_the_device_path(gpu):
    """Mixed sizes, an empty frame and frames without normals: every result
    equals pc_compute's bit for bit."""
    import torch
    rng = np.random.default_rng(4)
    sizes = [(240, 320), (424, 512), (480, 640), (0, 0), (720, 1280), (37, 53), (480, 640)]
    sc = [synth.kinect_scene(20 + i, H=H, W=W) if H else None for i, (H, W) in enumerate(sizes)]
    live = [s for s in sc if s is not None]
    with_normal = [bool(rng.random() < 0.7) for _ in live]
    fr = host_frames(live, with_normal)
    empty = (torch.zeros((0, 0)), (525.0, 525.0, 0.0, 0.0), torch.zeros((0, 0)), torch.zeros((0, 0)), None)
    fr.insert(3, empty)
    c = gpu.Curvature(525.0, 525.0, 319.5, 239.5, window_radius=7, iterations=5)
    stream = torch.cuda.Stream()
    c.host_batch(fr, stream=stream)
    stream.synchronize()
    c.close()
    fr.pop(3)
    for s, (d, intr, k1, k2, n), wn in zip(live, fr, with_normal):
        e1, e2, en = device_results(gpu, s)
        assert np.array_equal(k1.numpy(), e1, equal_nan=True)
        assert np.array_equal(k2.numpy(), e2, equal_nan=True)
        if wn:
            assert np.array_equal(n.numpy(), en, equal_nan=True)


def test_host_batch_many_chunks_and_repeated_calls(gpu):
    """More pixels than one chunk (several chunks through both staging slots),
    a frame larger than a chunk, and the same context called again."""
    import torch
    base = synth.kinect_scene(31)
    # 1920 x 3200 = 6.1 Mpx, more than a chunk: a chunk of its own (the tiled
    # ranges need no geometric meaning for a bit-for-bit comparison)
    big = types.SimpleNamespace(depth=np.ascontiguousarray(np.tile(base.depth, (4, 5))),
                                intrinsics=base.intrinsics)
    sc = [base] * 20 + [big] + [base] * 6
    fr = host_frames(sc, [True] * len(sc))
    c = gpu.Curvature(525.0, 525.0, 319.5, 239.5, window_radius=5, iterations=3)
    stream = torch.cuda.Stream()
    for _ in range(2):
        for _, _, k1, _, _ in fr:
            k1.fill_(0.0)
        c.host_batch(fr, stream=stream)
        stream.synchronize()
        e1, _, en = device_results(gpu, base, r=5, T=3)
        b1, _, bn = device_results(gpu, big, r=5, T=3)
        for i, (_, _, k1, _, n) in enumerate(fr):
            want1, wantn = (b1, bn) if i == 20 else (e1, en)
            assert np.array_equal(k1.numpy(), want1, equal_nan=True), i
            assert np.array_equal(n.numpy(), wantn, equal_nan=True), i
    c.close()


def test_host_batch_is_ordered_on_the_callers_stream(gpu):
    """The results are on the host once the caller's stream is synchronised,
    and the call starts after work already queued on that stream."""
    import torch
    s = synth.kinect_scene(33)
    stream = torch.cuda.Stream()
    dev = torch.from_numpy(s.depth).cuda()
    host = torch.empty_like(dev, device="cpu").pin_memory()
    with torch.cuda.stream(stream):
        torch.cuda._sleep(50_000_000)                       # keep the stream busy first
        host.copy_(dev, non_blocking=True)                  # the input arrives through the stream
    k1 = torch.empty(s.depth.shape).pin_memory()
    k2 = torch.empty(s.depth.shape).pin_memory()
    c = gpu.Curvature(*s.intrinsics, window_radius=7, iterations=5)
    c.host_batch([(host, s.intrinsics, k1, k2, None)], stream=stream)
    stream.synchronize()
    c.close()
    e1, e2, _ = device_results(gpu, s)
    assert np.array_equal(k1.numpy(), e1, equal_nan=True)
    assert np.array_equal(k2.numpy(), e2, equal_nan=True)
