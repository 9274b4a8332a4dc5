"""Python binding of the C ABI in include/pcurv.h (ctypes; argument marshalling only).

The functions keep the C names (pc_create, pc_compute, pc_compute_host,
pc_destroy, pc_status_string, pc_params_default, pc_last_error) and take raw
addresses.  `Curvature` wraps them for torch tensors: torch supplies device
memory and the CUDA stream, every step of the method runs in the library's
kernels.  There is no fallback: if libpcurv.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libpcurv.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pcurv.h")

PC_OK, PC_ERR_INVALID_ARG, PC_ERR_CUDA, PC_ERR_OOM, PC_ERR_TIMEOUT, PC_ERR_UNSUPPORTED = range(6)
PC_MAX_RADIUS, PC_MAX_NORMAL_RADIUS, PC_MAX_ITERATIONS, PC_MAX_DIM, PC_MAX_BATCH = 24, 8, 64, 16384, 4096
PC_STATIC_MAX_FRAMES = 256
PC_HOST_CHUNK_PIXELS = 4 << 20
PC_DEPTH_F16, PC_DEPTH_BF16 = 1, 2
PC_PACK_TILE_W, PC_PACK_TILE_H = 32, 8


class pc_params(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_float),
        ("reject", ctypes.c_int),
        ("reject_ratio", ctypes.c_float),
        ("normal_radius", ctypes.c_int),
        ("stride", ctypes.c_int),
        ("det_tol", ctypes.c_float),
        ("pivot_tol", ctypes.c_float),
        ("min_window", ctypes.c_int),
        ("batch_graph", ctypes.c_int),
        ("kahan", ctypes.c_int),
        ("fp64_solve_cond", ctypes.c_float),
        ("tile_height", ctypes.c_int),
        ("lanes_per_pixel", ctypes.c_int),
    ]


class pc_frame(ctypes.Structure):
    _fields_ = [
        ("depth", ctypes.c_void_p),
        ("H", ctypes.c_int), ("W", ctypes.c_int),
        ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
        ("k1", ctypes.c_void_p), ("k2", ctypes.c_void_p), ("normal", ctypes.c_void_p),
    ]


class pc_packed_frame(ctypes.Structure):
    _fields_ = [
        ("packed", ctypes.c_void_p), ("tile_base", ctypes.c_void_p),
        ("H", ctypes.c_int), ("W", ctypes.c_int),
        ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
        ("k1", ctypes.c_void_p), ("k2", ctypes.c_void_p), ("normal", ctypes.c_void_p),
    ]


class PcError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what}: {pc_status_string(status)} ({status})"
        super().__init__(msg + (f": {detail}" if detail else ""))


_lib = None
_vp = ctypes.c_void_p


def load() -> ctypes.CDLL:
    """Loads libpcurv.so (built by __graft_entry__.build() or
    `python -m paper_1707_00385_gb300.build`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.pc_params_default.argtypes = [ctypes.POINTER(pc_params)]
        L.pc_params_default.restype = None
        L.pc_create.argtypes = [ctypes.c_float] * 4 + [ctypes.c_int, ctypes.c_int,
                                                       ctypes.POINTER(pc_params), ctypes.POINTER(_vp)]
        L.pc_compute.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.pc_compute_host.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.pc_compute_batch.argtypes = [_vp, ctypes.POINTER(pc_frame), ctypes.c_int, _vp]
        L.pc_compute_batch_static.argtypes = [_vp, ctypes.POINTER(pc_frame), ctypes.c_int, _vp]
        L.pc_pack_depth.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        L.pc_autotune.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.pc_plan_tile_height.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
        L.pc_plan_tile_height.restype = ctypes.c_int
        L.pc_plan_lanes_per_pixel.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
        L.pc_plan_lanes_per_pixel.restype = ctypes.c_int
        _ip = ctypes.POINTER(ctypes.c_int)
        L.pc_plans_export.argtypes = [_vp, _ip, _ip, _ip, _ip, ctypes.c_int]
        L.pc_plans_export.restype = ctypes.c_int
        L.pc_plans_import.argtypes = [_vp, _ip, _ip, _ip, _ip, ctypes.c_int]
        L.pc_plans_import.restype = ctypes.c_int
        L.pc_compute_packed.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                        _vp, _vp, _vp]
        L.pc_compute_host_batch.argtypes = [_vp, ctypes.POINTER(pc_frame), ctypes.c_int, _vp]
        L.pc_compute_packed_batch.argtypes = [_vp, ctypes.POINTER(pc_packed_frame), ctypes.c_int, ctypes.c_int, _vp]
        L.pc_backproject.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
        L.pc_initial_normals.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
        L.pc_destroy.argtypes = [_vp]
        L.pc_status_string.argtypes = [ctypes.c_int]
        L.pc_status_string.restype = ctypes.c_char_p
        L.pc_last_error.argtypes = [_vp]
        L.pc_last_error.restype = ctypes.c_char_p
        L.pc_fp32_peak_kernel.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_longlong, _vp,
                                          ctypes.POINTER(ctypes.c_double)]
        L.pc_fp32_peak_kernel.restype = ctypes.c_int
        L.pc_moments_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_longlong, _vp,
                                       ctypes.POINTER(ctypes.c_int)]
        L.pc_moments_probe.restype = ctypes.c_int
        for f in ("pc_create", "pc_compute", "pc_compute_host", "pc_compute_batch",
                  "pc_compute_batch_static", "pc_pack_depth", "pc_compute_packed", "pc_autotune", "pc_destroy",
                  "pc_compute_host_batch", "pc_backproject", "pc_initial_normals", "pc_compute_packed_batch"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


# ---- the C functions, same names --------------------------------------------

def pc_params_default() -> pc_params:
    p = pc_params()
    load().pc_params_default(ctypes.byref(p))
    return p


def pc_create(fx, fy, cx, cy, window_radius, iterations, params: pc_params | None = None):
    """Returns (status, ctx handle or None)."""
    out = _vp()
    st = load().pc_create(fx, fy, cx, cy, window_radius, iterations,
                          ctypes.byref(params) if params is not None else None, ctypes.byref(out))
    return st, (out.value if st == PC_OK else None)


def pc_compute(ctx, depth, H, W, stream, k1_out, k2_out, normal_out) -> int:
    return load().pc_compute(ctx, depth, H, W, stream, k1_out, k2_out, normal_out)


def pc_compute_host(ctx, depth_host, H, W, stream, k1_host, k2_host, normal_host) -> int:
    return load().pc_compute_host(ctx, depth_host, H, W, stream, k1_host, k2_host, normal_host)


def pc_compute_batch(ctx, frames, n, stream) -> int:
    """frames: a ctypes array of pc_frame (or None when n == 0)."""
    return load().pc_compute_batch(ctx, frames, n, stream)


def pc_compute_batch_static(ctx, frames, n, stream) -> int:
    """The batch entry point that allocates no device memory (fixed scratch)."""
    return load().pc_compute_batch_static(ctx, frames, n, stream)


def pc_compute_host_batch(ctx, frames, n, stream) -> int:
    """frames: a ctypes array of pc_frame whose buffers are host addresses."""
    return load().pc_compute_host_batch(ctx, frames, n, stream)


def pc_backproject(ctx, depth, H, W, stream, xyz) -> int:
    return load().pc_backproject(ctx, depth, H, W, stream, xyz)


def pc_initial_normals(ctx, depth, H, W, stream, normal) -> int:
    return load().pc_initial_normals(ctx, depth, H, W, stream, normal)


def pc_pack_depth(ctx, depth, H, W, fmt, stream, packed, tile_base) -> int:
    return load().pc_pack_depth(ctx, depth, H, W, fmt, stream, packed, tile_base)


def pc_compute_packed(ctx, packed, tile_base, fmt, H, W, stream, k1_out, k2_out, normal_out) -> int:
    return load().pc_compute_packed(ctx, packed, tile_base, fmt, H, W, stream, k1_out, k2_out, normal_out)


def pc_compute_packed_batch(ctx, frames, n, fmt, stream) -> int:
    """frames: a ctypes array of pc_packed_frame (or None when n == 0)."""
    return load().pc_compute_packed_batch(ctx, frames, n, fmt, stream)


def pc_autotune(ctx, depth, H, W, stream, k1_out, k2_out, normal_out) -> int:
    return load().pc_autotune(ctx, depth, H, W, stream, k1_out, k2_out, normal_out)


def pc_plan_tile_height(ctx, H, W) -> int:
    return load().pc_plan_tile_height(ctx, H, W)


def pc_plan_lanes_per_pixel(ctx, H, W) -> int:
    return load().pc_plan_lanes_per_pixel(ctx, H, W)


def pc_plans_export(ctx):
    """Returns the plans of ctx as a list of (H, W, tile_height, lanes_per_pixel),
    oldest first (None for a NULL ctx)."""
    L = load()
    n = L.pc_plans_export(ctx, None, None, None, None, 0)
    if n < 0:
        return None
    arrs = [(ctypes.c_int * max(n, 1))() for _ in range(4)]
    n = L.pc_plans_export(ctx, *arrs, n)
    return [tuple(int(a[i]) for a in arrs) for i in range(n)]


def pc_plans_import(ctx, plans) -> int:
    """Adds plans given as (H, W, tile_height, lanes_per_pixel) tuples."""
    n = len(plans)
    arrs = [(ctypes.c_int * max(n, 1))(*[p[k] for p in plans]) for k in range(4)]
    return load().pc_plans_import(ctx, *arrs, n)


def pc_destroy(ctx) -> int:
    return load().pc_destroy(ctx)


def pc_status_string(status: int) -> str:
    return load().pc_status_string(status).decode()


def pc_last_error(ctx) -> str:
    return load().pc_last_error(ctx).decode()


def pc_moments_probe(mode, pixels, iters, sink, sink_len, stream):
    """Design measurement (not the method): returns (status, CTAs launched)."""
    blocks = ctypes.c_int(0)
    st = load().pc_moments_probe(mode, pixels, iters, sink, sink_len, stream, ctypes.byref(blocks))
    return st, blocks.value


def pc_fp32_peak_kernel(blocks, iters, packed, sink, sink_len, stream):
    """Measurement utility (not the method): returns (status, FLOP of the launch)."""
    flop = ctypes.c_double(0.0)
    st = load().pc_fp32_peak_kernel(blocks, iters, packed, sink, sink_len, stream, ctypes.byref(flop))
    return st, flop.value


# ---- torch convenience wrapper ----------------------------------------------

def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Curvature:
    """A pc_ctx for one camera and one parameter set.

    c = Curvature(fx, fy, cx, cy, window_radius=7, iterations=5)
    k1, k2, normal = c(depth)          # depth: CUDA float32 H x W tensor
    """

    def __init__(self, fx, fy, cx, cy, window_radius=7, iterations=5, **params):
        p = pc_params_default()
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        st, ctx = pc_create(fx, fy, cx, cy, window_radius, iterations, p)
        if st != PC_OK:
            raise PcError(st, "pc_create")
        self.ctx = ctx
        self.params = p
        self.window_radius, self.iterations = window_radius, iterations

    def close(self):
        if self.ctx is not None:
            pc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __call__(self, depth, k1=None, k2=None, normal=None, want_normal=True, stream=None):
        """Enqueues the method on `stream` (default: torch's current stream)
        and returns (k1, k2, normal); normal is None when want_normal is False."""
        import torch
        if depth.dtype != torch.float32 or not depth.is_cuda or depth.dim() != 2:
            raise ValueError("depth must be a 2-D float32 CUDA tensor")
        depth = depth.contiguous()
        H, W = depth.shape
        if k1 is None:
            k1 = torch.empty((H, W), dtype=torch.float32, device=depth.device)
        if k2 is None:
            k2 = torch.empty((H, W), dtype=torch.float32, device=depth.device)
        if want_normal and normal is None:
            normal = torch.empty((H, W, 3), dtype=torch.float32, device=depth.device)
        for t in (k1, k2) + ((normal,) if normal is not None else ()):
            if not t.is_contiguous() or t.dtype != torch.float32:
                raise ValueError("outputs must be contiguous float32")
        st = pc_compute(self.ctx, depth.data_ptr(), H, W, _stream_handle(stream), k1.data_ptr(),
                        k2.data_ptr(), normal.data_ptr() if normal is not None else None)
        if st != PC_OK:
            raise PcError(st, "pc_compute", pc_last_error(self.ctx))
        return k1, k2, normal

    def autotune(self, depth, stream=None):
        """pc_autotune on this image: times the kernel variants (tile shapes,
        lanes per pixel), remembers the fastest for its size; returns the tile
        height now planned (lanes_per_pixel(H, W) gives the lanes)."""
        import torch
        H, W = depth.shape
        k1 = torch.empty((H, W), device=depth.device)
        k2 = torch.empty((H, W), device=depth.device)
        n = torch.empty((H, W, 3), device=depth.device)
        st = pc_autotune(self.ctx, depth.contiguous().data_ptr(), H, W, _stream_handle(stream), k1.data_ptr(),
                         k2.data_ptr(), n.data_ptr())
        if st != PC_OK:
            raise PcError(st, "pc_autotune", pc_last_error(self.ctx))
        return pc_plan_tile_height(self.ctx, H, W)

    def tile_height(self, H, W):
        return pc_plan_tile_height(self.ctx, H, W)

    def lanes_per_pixel(self, H, W):
        return pc_plan_lanes_per_pixel(self.ctx, H, W)

    def _plan_key(self, device_name):
        p = self.params
        return {"device": device_name, "window_radius": self.window_radius, "iterations": self.iterations,
                "stride": p.stride, "normal_radius": p.normal_radius, "reject": p.reject, "kahan": p.kahan,
                "lanes_per_pixel": p.lanes_per_pixel}

    def save_plans(self, path, device_name=None):
        """Writes this context's plans (pc_plans_export) to a JSON file, with
        the GPU model and the parameters they were tuned for."""
        import json
        import torch
        name = device_name or torch.cuda.get_device_name()
        with open(path, "w") as f:
            json.dump({"key": self._plan_key(name), "plans": pc_plans_export(self.ctx)}, f)

    def load_plans(self, path, device_name=None) -> bool:
        """Adds the plans of a file written by save_plans when they were tuned
        for this GPU model and these parameters; returns whether it did."""
        import json
        import torch
        name = device_name or torch.cuda.get_device_name()
        with open(path) as f:
            d = json.load(f)
        if d.get("key") != self._plan_key(name):
            return False
        st = pc_plans_import(self.ctx, [tuple(p) for p in d["plans"]])
        if st != PC_OK:
            raise PcError(st, "pc_plans_import", pc_last_error(self.ctx))
        return True

    def batch(self, frames, stream=None):
        """pc_compute_batch over a list of (depth, (fx, fy, cx, cy), k1, k2, normal)
        tuples of CUDA tensors (normal may be None); enqueues one persistent launch."""
        arr = (pc_frame * max(len(frames), 1))()
        for i, (d, intr, a, b, n) in enumerate(frames):
            H, W = d.shape
            arr[i] = pc_frame(d.data_ptr(), H, W, *map(float, intr), a.data_ptr(), b.data_ptr(),
                              n.data_ptr() if n is not None else None)
        st = pc_compute_batch(self.ctx, arr if frames else None, len(frames), _stream_handle(stream))
        if st != PC_OK:
            raise PcError(st, "pc_compute_batch", pc_last_error(self.ctx))

    def pack(self, depth, fmt, stream=None):
        """pc_pack_depth: returns (packed int16 tensor H x W, tile_base float tensor)."""
        import torch
        H, W = depth.shape
        packed = torch.empty((H, W), dtype=torch.int16, device=depth.device)
        base = torch.empty(((H + 7) // 8, (W + 31) // 32), dtype=torch.float32, device=depth.device)
        st = pc_pack_depth(self.ctx, depth.contiguous().data_ptr(), H, W, fmt, _stream_handle(stream),
                           packed.data_ptr(), base.data_ptr())
        if st != PC_OK:
            raise PcError(st, "pc_pack_depth", pc_last_error(self.ctx))
        return packed, base

    def compute_packed(self, packed, base, fmt, stream=None, want_normal=True):
        """pc_compute_packed on the storage made by pack(); returns (k1, k2, normal)."""
        import torch
        H, W = packed.shape
        k1 = torch.empty((H, W), device=packed.device)
        k2 = torch.empty((H, W), device=packed.device)
        normal = torch.empty((H, W, 3), device=packed.device) if want_normal else None
        st = pc_compute_packed(self.ctx, packed.data_ptr(), base.data_ptr(), fmt, H, W, _stream_handle(stream),
                               k1.data_ptr(), k2.data_ptr(), normal.data_ptr() if normal is not None else None)
        if st != PC_OK:
            raise PcError(st, "pc_compute_packed", pc_last_error(self.ctx))
        return k1, k2, normal

    def batch_packed(self, frames, fmt, stream=None):
        """pc_compute_packed_batch over a list of (packed, tile_base, (fx, fy, cx, cy),
        k1, k2, normal) tuples of CUDA tensors (the storage of pack(), all in
        format fmt; normal may be None); enqueues one persistent launch."""
        arr = (pc_packed_frame * max(len(frames), 1))()
        for i, (q, base, intr, a, b, n) in enumerate(frames):
            H, W = q.shape
            arr[i] = pc_packed_frame(q.data_ptr(), base.data_ptr(), H, W, *map(float, intr), a.data_ptr(),
                                     b.data_ptr(), n.data_ptr() if n is not None else None)
        st = pc_compute_packed_batch(self.ctx, arr if frames else None, len(frames), fmt, _stream_handle(stream))
        if st != PC_OK:
            raise PcError(st, "pc_compute_packed_batch", pc_last_error(self.ctx))

    def host_batch(self, frames, stream=None):
        """pc_compute_host_batch over a list of (depth, (fx, fy, cx, cy), k1, k2,
        normal) tuples of CPU float32 tensors (pinned for the copies to overlap;
        normal may be None).  Synchronise the stream before reading the outputs."""
        arr = (pc_frame * max(len(frames), 1))()
        for i, (d, intr, a, b, n) in enumerate(frames):
            H, W = d.shape
            arr[i] = pc_frame(d.data_ptr(), H, W, *map(float, intr), a.data_ptr(), b.data_ptr(),
                              n.data_ptr() if n is not None else None)
        st = pc_compute_host_batch(self.ctx, arr if frames else None, len(frames), _stream_handle(stream))
        if st != PC_OK:
            raise PcError(st, "pc_compute_host_batch", pc_last_error(self.ctx))

    def backproject(self, depth, xyz=None, stream=None):
        """pc_backproject: the organised point cloud (H x W x 3) of a CUDA range image."""
        import torch
        H, W = depth.shape
        depth = depth.contiguous()
        if xyz is None:
            xyz = torch.empty((H, W, 3), dtype=torch.float32, device=depth.device)
        st = pc_backproject(self.ctx, depth.data_ptr(), H, W, _stream_handle(stream), xyz.data_ptr())
        if st != PC_OK:
            raise PcError(st, "pc_backproject", pc_last_error(self.ctx))
        return xyz

    def initial_normals(self, depth, normal=None, stream=None):
        """pc_initial_normals: the (2 normal_radius + 1)^2 regression normals (H x W x 3)."""
        import torch
        H, W = depth.shape
        depth = depth.contiguous()
        if normal is None:
            normal = torch.empty((H, W, 3), dtype=torch.float32, device=depth.device)
        st = pc_initial_normals(self.ctx, depth.data_ptr(), H, W, _stream_handle(stream), normal.data_ptr())
        if st != PC_OK:
            raise PcError(st, "pc_initial_normals", pc_last_error(self.ctx))
        return normal

    def compute_host(self, depth, k1, k2, normal=None, stream=None):
        """Host-memory form (pc_compute_host): depth, k1, k2, normal are CPU
        float32 tensors (pinned for asynchronous copies).  Enqueues the copies
        and the kernel; synchronise the stream before reading the outputs."""
        H, W = depth.shape
        st = pc_compute_host(self.ctx, depth.data_ptr(), H, W, _stream_handle(stream), k1.data_ptr(),
                             k2.data_ptr(), normal.data_ptr() if normal is not None else None)
        if st != PC_OK:
            raise PcError(st, "pc_compute_host", pc_last_error(self.ctx))
