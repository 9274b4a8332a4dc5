"""Seeded synthetic range images with analytic ground truth.

This module only makes inputs: it ray-casts analytic primitives (planes,
spheres, finite open cylinders, parabolic saddle patches) through a pinhole
camera in float64, keeps the nearest hit, adds depth noise and zeroes random
blobs of pixels.  It holds none of the curvature method's arithmetic (no
back-projection of ranges, no fitting), so the oracle and the CUDA path can
both be fed from it.

Conventions shared with the method: pixel (u, v) is column u, row v, with its
centre at integer coordinates; the ray through it is ((u-cx)/fx, (v-cy)/fy, 1),
so the ray parameter of a hit is its depth Z.  Ground-truth normals point away
from the camera; a surface that is convex towards the camera has positive
curvature (a sphere of radius rho gives (1/rho, 1/rho)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Camera:
    H: int
    W: int
    fx: float
    fy: float
    cx: float
    cy: float

    def rays(self) -> np.ndarray:
        v, u = np.mgrid[0:self.H, 0:self.W].astype(np.float64)
        d = np.empty((self.H, self.W, 3))
        d[..., 0] = (u - self.cx) / self.fx
        d[..., 1] = (v - self.cy) / self.fy
        d[..., 2] = 1.0
        return d


def kinect_camera(H: int = 480, W: int = 640) -> Camera:
    """Kinect-like intrinsics: fx = fy = 525 at 640 px wide, scaled with the
    width, principal point at the image centre (525 / 319.5 / 239.5 at 640x480)."""
    f = 525.0 * W / 640.0
    return Camera(H, W, f, f, (W - 1) / 2.0, (H - 1) / 2.0)


# ---------------------------------------------------------------------------
# primitives: each returns (t, k1, k2, normal) per ray, t = inf where missed

def _no_hit(shape):
    return (np.full(shape, np.inf), np.full(shape, np.nan), np.full(shape, np.nan),
            np.full(shape + (3,), np.nan))


def _away(nrm, d):
    """orient normals to point away from the camera (n . ray > 0)"""
    s = np.sign(np.einsum("...i,...i->...", nrm, d))
    s[s == 0] = 1.0
    return nrm * s[..., None]


@dataclass
class Plane:
    n: np.ndarray  # unit normal
    d: float       # plane {P : n . P = d}

    def hit(self, rays):
        nd = rays @ self.n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(np.abs(nd) > 1e-12, self.d / nd, np.inf)
        t = np.where(t > 0, t, np.inf)
        k = np.where(np.isfinite(t), 0.0, np.nan)
        nrm = _away(np.broadcast_to(self.n, rays.shape).copy(), rays)
        return t, k, k.copy(), nrm


@dataclass
class Sphere:
    c: np.ndarray
    rho: float

    def hit(self, rays):
        dd = np.einsum("...i,...i->...", rays, rays)
        dc = rays @ self.c
        disc = dc * dc - dd * (self.c @ self.c - self.rho ** 2)
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t = np.where(ok, (dc - sq) / dd, np.inf)
        t = np.where(t > 0, t, np.inf)
        P = rays * np.where(np.isfinite(t), t, 0.0)[..., None]
        nrm = _away((P - self.c) / self.rho, rays)
        kk = np.where(np.isfinite(t), 1.0 / self.rho, np.nan)
        return t, kk, kk.copy(), nrm


@dataclass
class Cylinder:
    """finite open cylinder: axis through a along unit e, radius rho, |axial| <= L"""
    a: np.ndarray
    e: np.ndarray
    rho: float
    L: float

    def hit(self, rays):
        e = self.e
        dpar = rays @ e
        dperp = rays - dpar[..., None] * e
        aperp = self.a - (self.a @ e) * e
        qa = np.einsum("...i,...i->...", dperp, dperp)
        qb = -2.0 * (dperp @ aperp)
        qc = aperp @ aperp - self.rho ** 2
        disc = qb * qb - 4 * qa * qc
        ok = (disc >= 0) & (qa > 1e-15)
        sq = np.sqrt(np.where(ok, disc, 0.0))
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = np.where(ok, (-qb - sq) / (2 * qa), np.inf)
            t2 = np.where(ok, (-qb + sq) / (2 * qa), np.inf)

        def axial_ok(t):
            s = t * dpar - self.a @ e
            return np.isfinite(t) & (t > 0) & (np.abs(s) <= self.L)

        o1, o2 = axial_ok(t1), axial_ok(t2)
        t = np.where(o1, t1, np.where(o2, t2, np.inf))
        P = rays * np.where(np.isfinite(t), t, 0.0)[..., None]
        Q = P - self.a
        radial = (Q - (Q @ e)[..., None] * e) / self.rho
        nrm = _away(radial, rays)
        # outer wall: convex towards the camera (1/rho, 0); inner wall seen
        # through an open end: concave (0, -1/rho)
        k1 = np.where(o1, 1.0 / self.rho, np.where(o2, 0.0, np.nan))
        k2 = np.where(o1, 0.0, np.where(o2, -1.0 / self.rho, np.nan))
        return t, k1, k2, nrm


@dataclass
class Saddle:
    """graph z_l = a x_l^2 - c y_l^2 over |x_l|, |y_l| <= s in a local frame:
    camera point = o + Rs @ (x_l, y_l, z_l); Rs's third column points away
    from the camera."""
    o: np.ndarray
    Rs: np.ndarray
    a: float
    c: float
    s: float

    def hit(self, rays):
        dl = rays @ self.Rs          # R_s^T d for every ray
        ol = self.Rs.T @ self.o
        a, c = self.a, self.c
        al = a * dl[..., 0] ** 2 - c * dl[..., 1] ** 2
        be = -2 * a * dl[..., 0] * ol[0] + 2 * c * dl[..., 1] * ol[1] - dl[..., 2]
        ga = a * ol[0] ** 2 - c * ol[1] ** 2 + ol[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            disc = be * be - 4 * al * ga
            sq = np.sqrt(np.where(disc >= 0, disc, np.nan))
            lin = np.abs(al) < 1e-14
            r_lin = -ga / be
            # cancellation-free pair of roots
            qq = -0.5 * (be + np.copysign(sq, be))
            ra, rb = qq / al, ga / qq
            ra = np.where(lin, r_lin, ra)
            rb = np.where(lin, np.inf, rb)

        def valid(t):
            q = t[..., None] * dl - ol
            return (np.isfinite(t) & (t > 0) & (np.abs(q[..., 0]) <= self.s)
                    & (np.abs(q[..., 1]) <= self.s))

        lo, hi = np.minimum(ra, rb), np.maximum(ra, rb)
        lo = np.where(np.isnan(lo), np.inf, lo)
        hi = np.where(np.isnan(hi), np.inf, hi)
        t = np.where(valid(lo), lo, np.where(valid(hi), hi, np.inf))
        q = np.where(np.isfinite(t), t, 0.0)[..., None] * dl - ol
        x, y = q[..., 0], q[..., 1]
        fx_, fy_ = 2 * a * x, -2 * c * y
        fxx, fyy = 2 * a, -2 * c
        g = 1.0 + fx_ ** 2 + fy_ ** 2
        # shape operator of the graph with the normal along +z_l
        E, F, G = 1 + fx_ ** 2, fx_ * fy_, 1 + fy_ ** 2
        Lf, Nf = fxx / np.sqrt(g), fyy / np.sqrt(g)
        det1 = E * G - F * F
        S11 = (G * Lf) / det1
        S12 = (-F * Nf) / det1
        S21 = (-F * Lf) / det1
        S22 = (E * Nf) / det1
        tr = S11 + S22
        dt = S11 * S22 - S12 * S21
        root = np.sqrt(np.maximum(tr * tr / 4 - dt, 0.0))
        hit = np.isfinite(t)
        k1 = np.where(hit, tr / 2 + root, np.nan)
        k2 = np.where(hit, tr / 2 - root, np.nan)
        nl = np.stack([-fx_, -fy_, np.ones_like(x)], -1) / np.sqrt(g)[..., None]
        nrm = _away(nl @ self.Rs.T, rays)
        # seen from the +z_l side the surface bends the other way
        facing = np.einsum("...i,...i->...", nl @ self.Rs.T, rays) > 0
        k1, k2 = np.where(facing, k1, -k2), np.where(facing, k2, -k1)
        return t, k1, k2, nrm


@dataclass
class Torus:
    """torus around axis e (unit) through centre c: ring radius R, tube radius rho"""
    c: np.ndarray
    e: np.ndarray
    R: float
    rho: float

    def _parts(self, P):
        q = P - self.c
        s = q @ self.e
        radial = q - s[..., None] * self.e
        dr = np.linalg.norm(radial, axis=-1)
        return q, s, radial, dr

    def hit(self, rays):
        d = rays / np.linalg.norm(rays, axis=-1, keepdims=True)
        scale = np.linalg.norm(rays, axis=-1)
        bound = self.R + self.rho
        # start at the bounding sphere, march by the exact distance (sphere tracing)
        dc = d @ self.c
        disc = dc * dc - (self.c @ self.c - bound * bound)
        t = np.where(disc > 0, dc - np.sqrt(np.maximum(disc, 0.0)), np.inf)
        t = np.maximum(t, 0.0)
        t_far = np.where(disc > 0, dc + np.sqrt(np.maximum(disc, 0.0)), -np.inf)
        alive = np.isfinite(t)
        for _ in range(400):
            P = d * np.where(alive, t, 0.0)[..., None]
            _, s_, _, dr = self._parts(P)
            sdf = np.sqrt((dr - self.R) ** 2 + s_ ** 2) - self.rho
            step = np.where(alive, sdf, 0.0)
            t = t + step
            alive &= (np.abs(sdf) > 1e-12) & (t <= t_far)
        P = d * np.where(np.isfinite(t), t, 0.0)[..., None]
        _, s_, _, dr = self._parts(P)
        sdf = np.sqrt((dr - self.R) ** 2 + s_ ** 2) - self.rho
        found = np.isfinite(t) & (np.abs(sdf) < 1e-9) & (t <= t_far + 1e-9)
        # Newton on the quartic F = (|q|^2 + R^2 - rho^2)^2 - 4 R^2 (|q|^2 - s^2) along the ray
        for _ in range(3):
            P = d * np.where(found, t, 0.0)[..., None]
            q, s_, _, _ = self._parts(P)
            qq = np.einsum("...i,...i->...", q, q)
            g = qq + self.R ** 2 - self.rho ** 2
            F = g * g - 4 * self.R ** 2 * (qq - s_ * s_)
            dqq = 2 * (q @ np.eye(3) * d).sum(-1)
            ds = d @ self.e
            dF = 2 * g * dqq - 4 * self.R ** 2 * (dqq - 2 * s_ * ds)
            t = np.where(found & (dF != 0), t - F / np.where(dF != 0, dF, 1.0), t)
        z = np.where(found, t / scale, np.inf)     # ray parameter of the unnormalised ray = depth
        P = rays * np.where(found, z, 0.0)[..., None]
        q, s_, radial, dr = self._parts(P)
        cosphi = (dr - self.R) / self.rho
        ring_dir = radial / np.maximum(dr, 1e-300)[..., None]
        outward = ((dr - self.R)[..., None] * ring_dir + s_[..., None] * self.e) / self.rho
        nrm = _away(outward, rays)
        kt = np.full(z.shape, 1.0 / self.rho)
        kr = cosphi / (self.R + self.rho * cosphi)
        # seen from outside: convex towards the camera is positive
        k1 = np.where(found, np.maximum(kt, kr), np.nan)
        k2 = np.where(found, np.minimum(kt, kr), np.nan)
        return z, k1, k2, nrm


# ---------------------------------------------------------------------------

@dataclass
class Scene:
    depth: np.ndarray        # float32 H x W, metres, 0 = no range
    cam: Camera
    gt_k1: np.ndarray        # float64 H x W, m^-1, NaN where undefined
    gt_k2: np.ndarray
    gt_normal: np.ndarray    # float64 H x W x 3
    label: np.ndarray        # int32 H x W, index of the primitive hit, -1 none
    clean: np.ndarray        # float64 noise-free depth (inf where no hit)
    prims: list = field(default_factory=list)

    @property
    def intrinsics(self):
        return (self.cam.fx, self.cam.fy, self.cam.cx, self.cam.cy)


def render(cam: Camera, prims, noise=None, rng=None, invalid_frac=0.0, blob_radius=(2, 8)) -> Scene:
    """Ray-cast prims (nearest hit wins), then add noise(z, rng) to the depth
    and zero random disks until invalid_frac of the pixels are zero."""
    rays = cam.rays()
    shape = (cam.H, cam.W)
    t, k1, k2, nrm = _no_hit(shape)
    label = np.full(shape, -1, dtype=np.int32)
    for i, pr in enumerate(prims):
        ti, a, b, n = pr.hit(rays)
        closer = ti < t
        t = np.where(closer, ti, t)
        k1 = np.where(closer, a, k1)
        k2 = np.where(closer, b, k2)
        nrm = np.where(closer[..., None], n, nrm)
        label = np.where(closer, i, label)
    clean = t.copy()
    z = np.where(np.isfinite(t), t, 0.0)
    if noise is not None:
        z = np.where(z > 0, z + noise(z, rng), 0.0)
        z = np.where(z > 0, z, 0.0)
    depth = z.astype(np.float32)
    if invalid_frac > 0:
        target = invalid_frac * cam.H * cam.W
        vv, uu = np.mgrid[0:cam.H, 0:cam.W]
        mask = np.zeros(shape, dtype=bool)
        while mask.sum() < target:
            cu, cv = rng.uniform(0, cam.W), rng.uniform(0, cam.H)
            rad = rng.uniform(*blob_radius)
            mask |= (uu - cu) ** 2 + (vv - cv) ** 2 <= rad * rad
        depth[mask] = 0.0
    return Scene(depth, cam, k1, k2, nrm, label, clean, list(prims))


def kinect_noise(z, rng):
    """sigma(z) = 0.0012 + 0.0019 (z - 0.4)^2 metres (structured-light model)"""
    return rng.standard_normal(z.shape) * (0.0012 + 0.0019 * (z - 0.4) ** 2)


def tof_noise(z, rng):
    """sigma(z) = 0.8 mm + 0.1 % of z (time-of-flight model)"""
    return rng.standard_normal(z.shape) * (0.0008 + 0.001 * z)


def const_noise(sigma):
    def f(z, rng):
        return rng.standard_normal(z.shape) * sigma
    return f


def _rand_rotation(rng, max_tilt):
    """rotation whose third column is within max_tilt of +z (away from camera)"""
    axis = rng.normal(size=3)
    axis[2] = 0.0
    axis /= np.linalg.norm(axis) + 1e-300
    ang = rng.uniform(0, max_tilt)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R1 = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
    spin = rng.uniform(0, 2 * np.pi)
    Rz = np.array([[np.cos(spin), -np.sin(spin), 0], [np.sin(spin), np.cos(spin), 0], [0, 0, 1]])
    return R1 @ Rz


def sphere_scene(seed: int = 0) -> Scene:
    """64 x 48 image, fx = fy = 57.5, principal point (32, 24); a sphere of
    radius 0.10 m centred 0.80 m ahead in front of a plane at 1.5 m; Gaussian
    depth noise of 1 mm."""
    cam = Camera(48, 64, 57.5, 57.5, 32.0, 24.0)
    prims = [Sphere(np.array([0.0, 0.0, 0.8]), 0.10), Plane(np.array([0.0, 0.0, 1.0]), 1.5)]
    rng = np.random.default_rng(seed)
    return render(cam, prims, noise=const_noise(0.001), rng=rng)


def kinect_scene(seed: int = 0, H: int = 480, W: int = 640, noise: str = "kinect",
                 invalid_frac: float = 0.02, nprims=None) -> Scene:
    """Kinect-like scene: a wall at 2.5-3.5 m, a tilted floor, and 10-20
    primitives at 0.5-3.5 m -- spheres (r 0.03-0.3 m), open cylinders
    (r 0.02-0.2 m, random axes) and saddles z = a x^2 - c y^2 (a, c in
    [1, 20] m^-1, |x|, |y| <= 0.1 m, tilt <= 45 deg); depth noise (kinect:
    0.0012 + 0.0019 (z-0.4)^2 m; tof: 0.8 mm + 0.1 % z); invalid_frac of the
    pixels zeroed in disks of radius 2-8 px."""
    rng = np.random.default_rng(seed)
    cam = kinect_camera(H, W)
    prims = []
    # wall, slightly tilted
    wn = np.array([rng.uniform(-0.15, 0.15), rng.uniform(-0.15, 0.15), 1.0])
    wn /= np.linalg.norm(wn)
    prims.append(Plane(wn, rng.uniform(2.5, 3.5)))
    # floor below the camera (camera y points down), tilted towards the camera
    tilt = rng.uniform(0.05, 0.35)
    fn = np.array([0.0, np.cos(tilt), -np.sin(tilt)])
    prims.append(Plane(fn, rng.uniform(0.6, 1.2)))
    n = int(rng.integers(10, 21)) if nprims is None else int(nprims)
    for _ in range(n):
        kind = rng.integers(0, 3)
        u, v = rng.uniform(0.05, 0.95) * W, rng.uniform(0.05, 0.95) * H
        Z = rng.uniform(0.5, 3.5)
        c = np.array([(u - cam.cx) / cam.fx * Z, (v - cam.cy) / cam.fy * Z, Z])
        if kind == 0:
            rho = rng.uniform(0.03, 0.3)
            c = c * (max(Z, rho + 0.3) / Z)
            prims.append(Sphere(c, rho))
        elif kind == 1:
            rho = rng.uniform(0.02, 0.2)
            e = rng.normal(size=3)
            e /= np.linalg.norm(e)
            c = c * (max(Z, rho + 0.4) / Z)
            prims.append(Cylinder(c, e, rho, rng.uniform(0.05, 0.3)))
        else:
            a, cc = rng.uniform(1, 20), rng.uniform(1, 20)
            prims.append(Saddle(c, _rand_rotation(rng, np.deg2rad(45)), a, cc, 0.1))
    nf = {"kinect": kinect_noise, "tof": tof_noise, "none": None}[noise]
    return render(cam, prims, noise=nf, rng=rng, invalid_frac=invalid_frac)


def crop(scene: Scene, v0: int, u0: int, H: int, W: int) -> Scene:
    """The H x W window of a scene starting at row v0, column u0, with the
    principal point moved so that every pixel keeps its ray."""
    c = scene.cam
    cam = Camera(H, W, c.fx, c.fy, c.cx - u0, c.cy - v0)
    sl = (slice(v0, v0 + H), slice(u0, u0 + W))
    return Scene(np.ascontiguousarray(scene.depth[sl]), cam, scene.gt_k1[sl], scene.gt_k2[sl],
                 scene.gt_normal[sl], scene.label[sl], scene.clean[sl], scene.prims)
