"""FP64 CPU oracle for per-pixel principal curvature from range images.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path (the CUDA library
and its binding) never imports it, and the oracle never imports the product.

The arithmetic lives in ``pc_oracle.c`` (plain C, double precision, one pixel
at a time, in the order of Sec. 3.2 of Spek, Li and Drummond, arXiv
1707.00385).  This module compiles it with gcc and exposes each step through
ctypes so that the tests can pin every step separately.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, INVALID_CENTRE, BAD_NORMAL, FEW_POINTS, SINGULAR = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile pc_oracle.c into liboracle.so next to it (OpenMP when available).

    -ffp-contract=off keeps every double operation separately rounded, so the
    x86 and Arm builds give the same numbers.  PC_ORACLE_LIB names another
    build to load instead (the test that plants mistakes in a copy of the
    source runs the pins against that copy)."""
    override = os.environ.get("PC_ORACLE_LIB")
    if override:
        return override
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-D_DEFAULT_SOURCE",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("r", ctypes.c_int), ("rn", ctypes.c_int), ("T", ctypes.c_int), ("stride", ctypes.c_int),
        ("k", ctypes.c_double), ("reject", ctypes.c_int), ("reject_ratio", ctypes.c_double),
        ("det_tol", ctypes.c_double), ("pivot_tol", ctypes.c_double), ("min_window", ctypes.c_int),
        ("perturb", ctypes.c_double), ("perturb_points", ctypes.c_double), ("perturb_seed", ctypes.c_ulonglong),
        ("f32_sums", ctypes.c_int),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iters", ctypes.c_int), ("npts", ctypes.c_int),
        ("k1", ctypes.c_double), ("k2", ctypes.c_double),
        ("normal", ctypes.c_double * 3), ("n0", ctypes.c_double * 3),
        ("A", ctypes.c_double), ("B", ctypes.c_double), ("C", ctypes.c_double), ("tz", ctypes.c_double),
        ("R", ctypes.c_double * 9), ("min_pivot", ctypes.c_double), ("last_b", ctypes.c_double * 6),
        ("cond", ctypes.c_double),
    ]


# validity thresholds of the method as this repository reads it (both the
# oracle and the CUDA path use the same values, each from its own source)
DET_TOL = 1e-6
PIVOT_TOL = 1e-5
MIN_WINDOW = 6


def params(fx, fy, cx, cy, r, T, *, rn=3, k=1e-4, stride=1, reject=0, reject_ratio=2.0,
           det_tol=DET_TOL, pivot_tol=PIVOT_TOL, min_window=MIN_WINDOW, perturb=0.0,
           perturb_points=0.0, perturb_seed=0, f32_sums=0) -> Params:
    """f32_sums = 1 is the probe's calibration mode, not the method: p' and
    every sum of the normal equations and of the initial-normal regression
    rounded to single precision (plain loop order)."""
    return Params(float(fx), float(fy), float(cx), float(cy), int(r), int(rn), int(T), int(stride),
                  float(k), int(reject), float(reject_ratio), float(det_tol), float(pivot_tol),
                  int(min_window), float(perturb), float(perturb_points), int(perturb_seed), int(f32_sums))


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int)
_P = ctypes.POINTER(Params)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.or_backproject.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
        L.or_initial_normal.argtypes = [_D, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _D]
        L.or_regression_sums.argtypes = [_D, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _D]
        L.or_frame_from_normal.argtypes = [_D, _D]
        L.or_rotation_exp.argtypes = [_D, _D]
        L.or_residual.argtypes = [_D] + [ctypes.c_double] * 4 + [_D, _D, _D]
        L.or_weight.argtypes = [_P, ctypes.c_double, ctypes.c_double]
        L.or_weight.restype = ctypes.c_double
        L.or_irls_step.argtypes = [_D, ctypes.c_int, _P, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.or_principal.argtypes = [ctypes.c_double] * 3 + [_D, _D]
        L.or_window.argtypes = [_D, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int]
        L.or_fit_pixel.argtypes = [_D, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(Result)]
        L.or_backproject_image.argtypes = [_F, ctypes.c_int, ctypes.c_int, _P, _D]
        L.or_initial_normal_image.argtypes = [_F, ctypes.c_int, ctypes.c_int, _P, _D, _I, ctypes.c_int]
        L.or_fit_pixel_f32.argtypes = [_F, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(Result)]
        for name, dp in (("or_curvature_image", _F), ("or_curvature_image_f64", _D)):
            getattr(L, name).argtypes = [dp, ctypes.c_int, ctypes.c_int, _P, _D, _D, _D, _I, _D, _D, _D,
                                         ctypes.c_int]
        for name, dp in (("or_curvature_pixels", _F), ("or_curvature_pixels_f64", _D)):
            getattr(L, name).argtypes = [dp, ctypes.c_int, ctypes.c_int, _P, _I, ctypes.c_int,
                                         _D, _D, _D, _I, _D, _D, _D, ctypes.c_int]
        L.or_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def max_threads() -> int:
    return int(lib().or_max_threads())


# ---- single steps ---------------------------------------------------------

def backproject(p: Params, u: int, v: int, z: float) -> np.ndarray:
    P = np.zeros(3)
    lib().or_backproject(ctypes.byref(p), u, v, z, _dp(P))
    return P


def _as_f64(depth):
    return np.ascontiguousarray(depth, dtype=np.float64)


def initial_normal(depth, p: Params, u0: int, v0: int):
    d = _as_f64(depth)
    n = np.zeros(3)
    st = lib().or_initial_normal(_dp(d), d.shape[0], d.shape[1], ctypes.byref(p), u0, v0, _dp(n))
    return st, n


def regression_sums(depth, p: Params, u0: int, v0: int):
    """(count, sums) of the initial-normal regression of one pixel without the
    probe: sums = (M00, M01, M11, v0, v1, sum of squared centred heights);
    single precision when p.f32_sums (the probe's calibration)."""
    d = _as_f64(depth)
    sums = np.zeros(6)
    cnt = lib().or_regression_sums(_dp(d), d.shape[0], d.shape[1], ctypes.byref(p), u0, v0, _dp(sums))
    return cnt, sums


def frame_from_normal(n) -> np.ndarray:
    n = np.ascontiguousarray(n, dtype=np.float64)
    R = np.zeros(9)
    lib().or_frame_from_normal(_dp(n), _dp(R))
    return R.reshape(3, 3)


def rotation_exp(w) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    R = np.zeros(9)
    lib().or_rotation_exp(_dp(w), _dp(R))
    return R.reshape(3, 3)


def residual(R, tz, A, B, C, pp):
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(9)
    pp = np.ascontiguousarray(pp, dtype=np.float64)
    e = ctypes.c_double()
    j = np.zeros(6)
    lib().or_residual(_dp(R), tz, A, B, C, _dp(pp), ctypes.byref(e), _dp(j))
    return e.value, j


def weight(p: Params, eps: float, mse: float = 0.0) -> float:
    return lib().or_weight(ctypes.byref(p), eps, mse)


def irls_step(pts, p: Params, R, tz, A, B, C):
    """One re-weighted update; returns dict(status, R, tz, A, B, C, N, rhs, b, w, min_pivot)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    m = pts.shape[0]
    Rm = np.ascontiguousarray(R, dtype=np.float64).reshape(9).copy()
    st = [ctypes.c_double(v) for v in (tz, A, B, C)]
    mp = ctypes.c_double(1.0)
    N, rhs, b, w = np.zeros(36), np.zeros(6), np.zeros(6), np.zeros(max(m, 1))
    status = lib().or_irls_step(_dp(pts), m, ctypes.byref(p), _dp(Rm), *[ctypes.byref(s) for s in st],
                                ctypes.byref(mp), _dp(N), _dp(rhs), _dp(b), _dp(w))
    return dict(status=status, R=Rm.reshape(3, 3), tz=st[0].value, A=st[1].value, B=st[2].value,
                C=st[3].value, N=N.reshape(6, 6), rhs=rhs, b=b, w=w[:m], min_pivot=mp.value)


def principal(A, B, C):
    k1, k2 = ctypes.c_double(), ctypes.c_double()
    lib().or_principal(A, B, C, ctypes.byref(k1), ctypes.byref(k2))
    return k1.value, k2.value


def window(depth, p: Params, u0: int, v0: int) -> np.ndarray:
    d = _as_f64(depth)
    side = 2 * p.r + 1
    uv = np.zeros(2 * side * side, dtype=np.int32)
    n = lib().or_window(_dp(d), d.shape[0], d.shape[1], ctypes.byref(p), u0, v0, _ip(uv), side * side)
    return uv[: 2 * n].reshape(-1, 2)


def fit_pixel(depth, p: Params, u0: int, v0: int) -> Result:
    res = Result()
    if np.asarray(depth).dtype == np.float32:
        d = np.ascontiguousarray(depth, dtype=np.float32)
        lib().or_fit_pixel_f32(d.ctypes.data_as(_F), d.shape[0], d.shape[1], ctypes.byref(p), u0, v0,
                               ctypes.byref(res))
    else:
        d = _as_f64(depth)
        lib().or_fit_pixel(_dp(d), d.shape[0], d.shape[1], ctypes.byref(p), u0, v0, ctypes.byref(res))
    return res


# ---- whole images / pixel lists --------------------------------------------

@dataclass
class Field:
    k1: np.ndarray
    k2: np.ndarray
    normal: np.ndarray
    status: np.ndarray
    min_pivot: np.ndarray
    last_b: np.ndarray      # update b of the last iteration, (..., 6)
    cond: np.ndarray = None  # largest max/min scaled-pivot ratio of one iteration (inf: singular)

    def converged(self, step_k=1e-5, step_theta=1e-6):
        """Pixels whose last Gauss-Newton update is below step_k * (1 + |k1|)
        for A, B, C and below step_theta (rad) for the frame: the fixed-count
        iteration has settled, so its output no longer depends on the path."""
        kk = np.abs(self.last_b[..., 3:]).max(-1)
        th = np.hypot(self.last_b[..., 0], self.last_b[..., 1])
        with np.errstate(invalid="ignore"):
            return (self.status == OK) & (kk <= step_k * (1 + np.abs(self.k1))) & (th <= step_theta)


def backproject_image(depth, p: Params) -> np.ndarray:
    """Organised point cloud (H x W x 3) of a float32 range image: the
    back-projection of every pixel, NaN where the range is not valid."""
    d = np.ascontiguousarray(depth, dtype=np.float32)
    H, W = d.shape
    xyz = np.zeros((H, W, 3))
    lib().or_backproject_image(d.ctypes.data_as(_F), H, W, ctypes.byref(p), _dp(xyz))
    return xyz


def initial_normal_image(depth, p: Params, nthreads: int = 0):
    """Initial normal (H x W x 3, NaN unless OK) and status (H x W) of every
    pixel of a float32 range image."""
    d = np.ascontiguousarray(depth, dtype=np.float32)
    H, W = d.shape
    n = np.zeros((H, W, 3))
    st = np.zeros((H, W), dtype=np.int32)
    lib().or_initial_normal_image(d.ctypes.data_as(_F), H, W, ctypes.byref(p), _dp(n), _ip(st), nthreads)
    return n, st


def curvature_image(depth, p: Params, nthreads: int = 0) -> Field:
    """The method at every pixel.  float32 depth is widened exactly; float64
    depth is used as given."""
    depth = np.asarray(depth)
    H, W = depth.shape
    k1, k2 = np.zeros((H, W)), np.zeros((H, W))
    nrm, st, mp = np.zeros((H, W, 3)), np.zeros((H, W), dtype=np.int32), np.zeros((H, W))
    lb, cd = np.zeros((H, W, 6)), np.zeros((H, W))
    if depth.dtype == np.float32:
        d = np.ascontiguousarray(depth)
        lib().or_curvature_image(d.ctypes.data_as(_F), H, W, ctypes.byref(p), _dp(k1), _dp(k2), _dp(nrm),
                                 _ip(st), _dp(mp), _dp(lb), _dp(cd), nthreads)
    else:
        d = _as_f64(depth)
        lib().or_curvature_image_f64(_dp(d), H, W, ctypes.byref(p), _dp(k1), _dp(k2), _dp(nrm), _ip(st),
                                     _dp(mp), _dp(lb), _dp(cd), nthreads)
    return Field(k1, k2, nrm, st, mp, lb, cd)


def curvature_pixels(depth, p: Params, uv, nthreads: int = 0) -> Field:
    """The method at the listed pixels uv (n x 2 array of (u, v))."""
    depth = np.asarray(depth)
    H, W = depth.shape
    uv = np.ascontiguousarray(uv, dtype=np.int32).reshape(-1, 2)
    n = uv.shape[0]
    k1, k2 = np.zeros(n), np.zeros(n)
    nrm, st, mp = np.zeros((n, 3)), np.zeros(n, dtype=np.int32), np.zeros(n)
    lb, cd = np.zeros((n, 6)), np.zeros(n)
    if depth.dtype == np.float32:
        d = np.ascontiguousarray(depth)
        lib().or_curvature_pixels(d.ctypes.data_as(_F), H, W, ctypes.byref(p), _ip(uv), n, _dp(k1), _dp(k2),
                                  _dp(nrm), _ip(st), _dp(mp), _dp(lb), _dp(cd), nthreads)
    else:
        d = _as_f64(depth)
        lib().or_curvature_pixels_f64(_dp(d), H, W, ctypes.byref(p), _ip(uv), n, _dp(k1), _dp(k2), _dp(nrm),
                                      _ip(st), _dp(mp), _dp(lb), _dp(cd), nthreads)
    return Field(k1, k2, nrm, st, mp, lb, cd)
