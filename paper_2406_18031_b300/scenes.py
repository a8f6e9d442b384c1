"""Seeded synthetic input sequences for the structure-flow filter.

This module only makes inputs: grayscale images and range maps rendered by a
small CPU ray-caster, plus the analytic ground truth of each synthetic scene.
It holds none of the filter's arithmetic and is shared by the tests (oracle
and CUDA sides alike) and the benchmark.

The paper evaluates on Blender renders (Urban Canyon, 512x512 at 300 Hz) and
on ZED stereo driving video (1024x1024); neither is available, so these
scenes stand in for their shapes, rates and flow magnitudes:

* ``plane64``  64x64, one level, a fronto-parallel textured plane at 5 m, camera
  translating at (0.5, 0.2, 1.0) m/s, 600 Hz -- closed-form structure flow.
* ``scene512`` 512x512, two levels, 8 textured planes and 4 spheres at 1-20 m,
  smooth random-walk camera motion scaled to about 8 px/frame, 600 Hz.
* ``drive``    384x1248, three levels, ground plane 1.5 m below the camera and
  20 boxes at 3-60 m, forward 10-25 m/s, yaw within +/-0.3 rad/s, 100 Hz,
  1% range noise, sky without a depth measurement.
* ``batch``    many independent ``plane64``-style streams of mixed sizes.

Camera model: pinhole rays through pixel centres, x right, y down, z forward.
Structure flow ground truth is w = -Omega x eta - v_c / lambda (static scene,
rad/s), the paper's Eq. 10 with a zero point velocity.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Sequence:
    name: str
    image: np.ndarray          # [F, H, W] float32 in [0, 1]
    range: np.ndarray          # [F, H, W] float32, metres along the ray (inf: none)
    dt: float                  # seconds per frame
    fx: float
    fy: float
    cx: float
    cy: float
    levels: int
    iters: list                # propagation sub-iterations per level (bottom first)
    smooth: list               # smoothing passes per level (bottom first)
    v: np.ndarray              # [F, 3] camera linear velocity, camera frame, m/s
    omega: np.ndarray          # [F, 3] camera angular velocity, camera frame, rad/s
    meta: dict = field(default_factory=dict)

    @property
    def frames(self):
        return self.image.shape[0]

    @property
    def shape(self):
        return self.image.shape[1:]

    def rays(self):
        return camera_rays(self.shape[0], self.shape[1], self.fx, self.fy, self.cx, self.cy)

    def gt_flow(self, k):
        """Ground-truth structure flow of frame k, [3, H, W] rad/s (Eq. 10, v_x = 0)."""
        eta = self.rays()
        lam = self.range[k].astype(np.float64)
        om = self.omega[k]
        rot = -np.cross(np.broadcast_to(om, eta.shape), eta)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = np.where(np.isfinite(lam) & (lam > 0), 1.0 / lam, 0.0)
        w = rot - self.v[k][None, None, :] * inv[..., None]
        return np.moveaxis(w, -1, 0)


def camera_rays(H, W, fx, fy, cx, cy):
    """Unit rays through pixel centres, [H, W, 3] float64."""
    j = (np.arange(W) + 0.5 - cx) / fx
    i = (np.arange(H) + 0.5 - cy) / fy
    x, y = np.meshgrid(j, i)
    d = np.stack([x, y, np.ones_like(x)], -1)
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def _rodrigues(axis_angle):
    th = np.linalg.norm(axis_angle)
    if th < 1e-15:
        return np.eye(3)
    k = axis_angle / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def _integrate(v, omega, dt, substeps=8):
    """World-from-camera poses (R, p) at every frame for body-frame (v, omega)."""
    F = v.shape[0]
    R = np.eye(3); p = np.zeros(3)
    Rs, ps = [], []
    h = dt / substeps
    for k in range(F):
        Rs.append(R.copy()); ps.append(p.copy())
        for _ in range(substeps):
            p = p + R @ v[k] * h
            R = R @ _rodrigues(omega[k] * h)
    return np.array(Rs), np.array(ps)


# ---------------------------------------------------------------------------
# textures (world-attached, so brightness is conserved along motion)
# ---------------------------------------------------------------------------

class _Blobs2D:
    """Sum of isotropic Gaussian blobs on a plane's (s, t) coordinates."""

    def __init__(self, rng, n, extent, sigma_range):
        self.c = rng.uniform(-extent, extent, size=(n, 2))
        self.s = rng.uniform(*sigma_range, size=n)
        self.a = rng.uniform(0.0, 1.0, size=n)

    def __call__(self, st):
        out = np.zeros(st.shape[:-1])
        for c, s, a in zip(self.c, self.s, self.a):
            d2 = ((st - c) ** 2).sum(-1)
            out += a * np.exp(-0.5 * d2 / (s * s))
        return out


class _Waves3D:
    """Smooth value texture: a few random 3D sinusoids, range [0, 1]."""

    def __init__(self, rng, n, k_range, base):
        d = rng.normal(size=(n, 3))
        self.k = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(*k_range, size=(n, 1))
        self.ph = rng.uniform(0, 2 * np.pi, size=n)
        self.a = rng.uniform(0.3, 1.0, size=n)
        self.a /= self.a.sum()
        self.base = base

    def __call__(self, X):
        out = np.zeros(X.shape[:-1])
        for k, ph, a in zip(self.k, self.ph, self.a):
            out += a * np.sin(X @ k + ph)
        return np.clip(self.base + 0.35 * out, 0.0, 1.0)


# ---------------------------------------------------------------------------
# scenes
# ---------------------------------------------------------------------------

def plane64(frames=20, seed=1000, H=64, W=64, depth=5.0, v=(0.5, 0.2, 1.0), rate=600.0,
            n_blobs=200, iters=None, levels=1, smooth=None):
    """Fronto-parallel plane at ``depth`` m textured with Gaussian blobs."""
    rng = np.random.default_rng(seed)
    f = W / 2.0  # 90 degree horizontal field of view
    fx = fy = f
    cx, cy = W / 2.0, H / 2.0
    dt = 1.0 / rate
    # blob sigma 1..6 px at the plane, in metres
    px_m = depth / f
    tex = _Blobs2D(rng, n_blobs, extent=1.2 * depth * (W / 2) / f + 0.5, sigma_range=(1.0 * px_m, 6.0 * px_m))
    eta = camera_rays(H, W, fx, fy, cx, cy)
    vv = np.asarray(v, dtype=np.float64)
    imgs, rngs = [], []
    for k in range(frames):
        c = vv * (k * dt)                     # camera position (no rotation)
        lam = (depth - c[2]) / eta[..., 2]    # range along the ray to the plane
        X = c[None, None, :] + lam[..., None] * eta
        imgs.append(tex(X[..., :2])); rngs.append(lam)
    imgs = np.array(imgs)
    scale = 1.0 / max(imgs[0].max(), 1e-12)
    imgs = np.clip(imgs * scale, 0.0, 1.0)
    F = frames
    return Sequence("plane64", imgs.astype(np.float32), np.array(rngs).astype(np.float32), dt,
                    fx, fy, cx, cy, levels, list(iters or [2] * levels),
                    list(smooth or ([2] + [4] * (levels - 1))),
                    np.tile(vv, (F, 1)), np.zeros((F, 3)), meta=dict(depth=depth))


def _ray_plane(o, d, n, c):
    """Distance along rays (o + t d) to the plane n.(X - c) = 0 (inf if none)."""
    den = d @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        t = ((c - o) @ n) / den
    return np.where((np.abs(den) > 1e-9) & (t > 1e-6), t, np.inf)


def _ray_sphere(o, d, c, r):
    oc = o - c
    b = d @ oc
    q = b * b - (oc @ oc - r * r)
    sq = np.sqrt(np.maximum(q, 0.0))
    t0 = -b - sq
    t1 = -b + sq
    t = np.where(t0 > 1e-6, t0, t1)
    return np.where((q > 0) & (t > 1e-6), t, np.inf)


def _ray_box(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (lo - o) * inv
        t2 = (hi - o) * inv
    tmin = np.nanmax(np.minimum(t1, t2), axis=-1)
    tmax = np.nanmin(np.maximum(t1, t2), axis=-1)
    hit = (tmax >= tmax * 0 + np.maximum(tmin, 1e-6))
    t = np.where(tmin > 1e-6, tmin, tmax)
    return np.where(hit & (t > 1e-6), t, np.inf)


def _map_frames(fn, frames):
    """[fn(0), ..., fn(frames - 1)] on a pool of threads (numpy releases the
    interpreter lock inside its array operations, so the frames render in
    parallel); fn must not draw random numbers."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    workers = max(1, min(frames, os.cpu_count() or 1, 32))
    if workers == 1:
        return [fn(k) for k in range(frames)]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, range(frames)))


def _random_walk(rng, F, sigma, vmax, start=None):
    x = np.zeros((F, 3)) if start is None else np.tile(start, (F, 1)).astype(np.float64)
    cur = x[0].copy()
    vel = np.zeros(3)
    for k in range(F):
        vel = 0.95 * vel + sigma * rng.normal(size=3)
        cur = cur + vel
        n = np.linalg.norm(cur)
        if n > vmax:
            cur *= vmax / n
        x[k] = cur
    return x


def scene512(frames=300, seed=1001, H=512, W=512, rate=600.0, max_flow=8.0, levels=2,
             iters=(8, 4), smooth=(2, 4)):
    """Eight textured planes and four spheres at 1-20 m; random-walk camera."""
    rng = np.random.default_rng(seed)
    f = W / 2.0
    fx = fy = f
    cx, cy = W / 2.0, H / 2.0
    dt = 1.0 / rate
    objs = []
    # background plane (one of the eight) facing the camera at 20 m
    objs.append(("plane", np.array([0.0, 0.0, -1.0]), np.array([0.0, 0.0, 20.0]), None,
                 _Waves3D(rng, 6, (0.5, 2.5), 0.5)))
    for _ in range(7):
        z = rng.uniform(1.0, 20.0)
        ang = np.arctan2(W / 2, f) * 0.8
        cxy = np.tan(rng.uniform(-ang, ang, size=2)) * z
        ctr = np.array([cxy[0], cxy[1], z])
        nrm = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), -1.0])
        nrm /= np.linalg.norm(nrm)
        half = rng.uniform(0.15, 0.45) * z
        k0 = 256.0 / (z * rng.uniform(6.0, 20.0))
        objs.append(("rect", nrm, ctr, half, _Waves3D(rng, 6, (0.5 * k0, 2.0 * k0), rng.uniform(0.3, 0.7))))
    for _ in range(4):
        z = rng.uniform(1.5, 20.0)
        ang = np.arctan2(W / 2, f) * 0.7
        cxy = np.tan(rng.uniform(-ang, ang, size=2)) * z
        r = rng.uniform(0.08, 0.25) * z
        k0 = 256.0 / (z * rng.uniform(6.0, 20.0))
        objs.append(("sphere", None, np.array([cxy[0], cxy[1], z + r]), r,
                     _Waves3D(rng, 6, (0.5 * k0, 2.0 * k0), rng.uniform(0.3, 0.7))))
    # camera motion: smooth random walk, mostly lateral translation
    v = _random_walk(rng, frames, 0.05, 3.0, start=rng.normal(size=3))
    v[:, 2] *= 0.3
    om = _random_walk(rng, frames, 0.01, 0.5, start=0.2 * rng.normal(size=3))
    eta = camera_rays(H, W, fx, fy, cx, cy)

    def render(R, p):
        d = eta.reshape(-1, 3) @ R.T
        o = p
        best = np.full(d.shape[0], np.inf)
        val = np.zeros(d.shape[0])
        for kind, nrm, ctr, size, tex in objs:
            if kind == "plane":
                t = _ray_plane(o, d, nrm, ctr)
            elif kind == "rect":
                t = _ray_plane(o, d, nrm, ctr)
                X = o + np.where(np.isfinite(t), t, 0.0)[:, None] * d
                rel = X - ctr
                a1 = np.cross(nrm, [0.0, 1.0, 0.0]); a1 /= np.linalg.norm(a1)
                a2 = np.cross(nrm, a1)
                inside = (np.abs(rel @ a1) < size) & (np.abs(rel @ a2) < size)
                t = np.where(inside, t, np.inf)
            else:
                t = _ray_sphere(o, d, ctr, size)
            m = t < best
            if m.any():
                best[m] = t[m]
                val[m] = tex(o + t[m, None] * d[m])
        return val.reshape(H, W), best.reshape(H, W)

    # scale the velocity so the largest image flow over the sequence is
    # ``max_flow`` px/frame (estimated on a coarse subset of the rays, then
    # checked again after the rescale changes the trajectory)
    sub = eta[::8, ::8]

    def peak_flow(Rs_, ps_, v_, om_):
        peak = 0.0
        for k in range(0, frames, max(1, frames // 32)):
            d = sub.reshape(-1, 3) @ Rs_[k].T
            best = np.full(d.shape[0], np.inf)
            for kind, nrm, ctr, size, tex in objs:
                if kind == "sphere":
                    t = _ray_sphere(ps_[k], d, ctr, size)
                else:
                    t = _ray_plane(ps_[k], d, nrm, ctr)
                    if kind == "rect":
                        X = ps_[k] + np.where(np.isfinite(t), t, 0.0)[:, None] * d
                        rel = X - ctr
                        a1 = np.cross(nrm, [0.0, 1.0, 0.0]); a1 /= np.linalg.norm(a1)
                        a2 = np.cross(nrm, a1)
                        t = np.where((np.abs(rel @ a1) < size) & (np.abs(rel @ a2) < size), t, np.inf)
                best = np.minimum(best, t)
            e = sub.reshape(-1, 3)
            w = -np.cross(np.broadcast_to(om_[k], e.shape), e) - v_[k][None, :] / best[:, None]
            tang = w - e * (w * e).sum(-1, keepdims=True)
            peak = max(peak, (np.linalg.norm(tang, axis=-1) * f * dt).max())
        return peak

    s = 1.0
    for _ in range(3):
        Rs, ps = _integrate(v * s, om * s, dt)
        s *= max_flow / max(peak_flow(Rs, ps, v * s, om * s), 1e-12)
    v *= s
    om *= s
    Rs, ps = _integrate(v, om, dt)
    out = _map_frames(lambda k: render(Rs[k], ps[k]), frames)
    imgs = [y for y, _ in out]
    rngs = [lam for _, lam in out]
    return Sequence("scene512", np.array(imgs, np.float32), np.array(rngs, np.float32), dt,
                    fx, fy, cx, cy, levels, list(iters), list(smooth), v, om,
                    meta=dict(velocity_scale=s))


def drive(frames=500, seed=1002, H=384, W=1248, rate=100.0, levels=3, iters=(32, 16, 8),
          smooth=(2, 4, 4), noise=0.01):
    """Driving-shaped scene: ground plane, 20 boxes, forward motion with yaw, sky."""
    rng = np.random.default_rng(seed)
    fx = fy = (W / 2.0) / np.tan(np.deg2rad(40.0))  # 80 degree horizontal FOV
    cx, cy = W / 2.0, H / 2.0
    dt = 1.0 / rate
    ground = _Waves3D(rng, 8, (0.5, 4.0), 0.45)
    boxes = []
    for _ in range(20):
        z = rng.uniform(3.0, 60.0)
        x = rng.uniform(-0.6, 0.6) * z
        sx, sy, sz = rng.uniform(0.5, 2.5), rng.uniform(1.0, 3.0), rng.uniform(0.5, 4.0)
        lo = np.array([x - sx, 1.5 - sy, z])
        hi = np.array([x + sx, 1.5, z + sz])
        boxes.append((lo, hi, _Waves3D(rng, 6, (0.5, 3.0), rng.uniform(0.3, 0.7))))
    speed = rng.uniform(10.0, 25.0)
    v = np.zeros((frames, 3)); v[:, 2] = speed
    yaw = np.clip(np.cumsum(rng.normal(scale=0.01, size=frames)), -0.3, 0.3)
    om = np.zeros((frames, 3)); om[:, 1] = yaw
    Rs, ps = _integrate(v, om, dt)
    eta = camera_rays(H, W, fx, fy, cx, cy)

    def render(k):
        d = eta.reshape(-1, 3) @ Rs[k].T
        o = ps[k]
        best = _ray_plane(o, d, np.array([0.0, -1.0, 0.0]), np.array([0.0, 1.5, 0.0]))
        val = np.full(d.shape[0], 0.85)                  # sky brightness
        m = np.isfinite(best)
        val[m] = ground(o + best[m, None] * d[m])
        for lo, hi, tex in boxes:
            t = _ray_box(o, d, lo, hi)
            mm = t < best
            if mm.any():
                best[mm] = t[mm]
                val[mm] = tex(o + t[mm, None] * d[mm])
        return val.reshape(H, W), best.reshape(H, W)

    out = _map_frames(render, frames)
    imgs, rngs = [], []
    for k in range(frames):                              # range noise drawn in frame order
        val, lam = out[k]
        lam = np.where(np.isfinite(lam), lam * (1.0 + noise * rng.normal(size=lam.shape)), np.inf)
        imgs.append(val); rngs.append(lam)
    return Sequence("drive", np.array(imgs, np.float32), np.array(rngs, np.float32), dt, fx, fy, cx, cy,
                    levels, list(iters), list(smooth), v, om, meta=dict(speed=speed))


class _Waves2D:
    """Cheap plane texture: a few random 2-D sinusoids, range [0, 1]."""

    def __init__(self, rng, n, k_range):
        d = rng.normal(size=(n, 2))
        self.k = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(*k_range, size=(n, 1))
        self.ph = rng.uniform(0, 2 * np.pi, size=n)
        self.a = rng.uniform(0.3, 1.0, size=n)
        self.a /= self.a.sum()

    def __call__(self, st):
        out = np.zeros(st.shape[:-1], np.float32)
        for k, ph, a in zip(self.k, self.ph, self.a):
            out += np.float32(a) * np.sin((st @ k + ph).astype(np.float32))
        return np.clip(0.5 + 0.4 * out, 0.0, 1.0)


def plane_stream(frames, seed, H, W, depth, v, rate, levels, iters, smooth, period=None):
    """A fronto-parallel textured plane under camera translation (config-1
    style) with a sinusoidal texture.

    Without ``period`` the camera moves at constant velocity v.  With it the
    camera oscillates, c(t) = v T / (2 pi) sin(2 pi t / T) with T = period
    frames, so its velocity is v cos(2 pi t / T), never faster than v, and
    frame k + period equals frame k: the sequence cycles without a jump.

    The plane's world point seen by pixel (i, j) is separable in the pixel
    coordinates, so each sinusoid of the texture is rendered as
    sin(a_j + b_i) = sin a_j cos b_i + cos a_j sin b_i from per-column and
    per-row values (one [H, 16] x [16, W] product per frame)."""
    rng = np.random.default_rng(seed)
    f = W / 2.0
    dt = 1.0 / rate
    px_m = depth / f
    tex = _Waves2D(rng, 8, (2 * np.pi / (40 * px_m), 2 * np.pi / (6 * px_m)))
    xj = (np.arange(W) + 0.5 - W / 2.0) / f          # ray direction (x_j, y_i, 1) of pixel (i, j)
    yi = (np.arange(H) + 0.5 - H / 2.0) / f
    norm = np.sqrt(1.0 + xj[None, :] ** 2 + yi[:, None] ** 2)
    vv = np.asarray(v, dtype=np.float64)
    imgs, rngs, vel = [], [], []
    for k in range(frames):
        if period:
            ph = 2.0 * np.pi * k / period
            c = vv * (period * dt / (2.0 * np.pi)) * np.sin(ph)
            vel.append(vv * np.cos(ph))
        else:
            c = vv * (k * dt)
            vel.append(vv)
        z = depth - c[2]                             # distance to the plane along the optical axis
        X = c[0] + z * xj                            # world x of the point seen by column j
        Y = c[1] + z * yi                            # world y of the point seen by row i
        aj = tex.k[:, 0:1] * X[None, :] + tex.ph[:, None]                  # [waves, W]
        bi = tex.k[:, 1:2] * Y[None, :]                                     # [waves, H]
        rows = np.concatenate([np.cos(bi), np.sin(bi)]).T                   # [H, 2 waves]
        cols = np.concatenate([tex.a[:, None] * np.sin(aj), tex.a[:, None] * np.cos(aj)])
        imgs.append(np.clip(0.5 + 0.4 * (rows @ cols), 0.0, 1.0)); rngs.append(z * norm)
    return Sequence("plane_stream", np.array(imgs, np.float32), np.array(rngs, np.float32), dt, f, f, W / 2.0,
                    H / 2.0, levels, list(iters), list(smooth), np.array(vel), np.zeros((frames, 3)),
                    meta=dict(depth=depth, period=period))


def batch(frames=2, seed=1003, sizes=((256, 16), (512, 32), (1024, 16)), max_flow=4.0, rate=600.0, period=None):
    """Independent config-1-style streams of mixed sizes (list of Sequences).

    Each stream is a textured plane with its own depth and camera velocity,
    chosen so the largest per-axis flow at level 1 is just below ``max_flow``
    px/frame (so N_1 = max_flow sub-iterations satisfy the CFL bound); 256x256
    streams use two pyramid levels, larger ones three, with
    N_h = ceil(max_flow / 2^(h-1)) and smoothing [2, 4, 4].  ``period``: the
    cameras oscillate with that many frames per cycle (see plane_stream).
    """
    rng = np.random.default_rng(seed)
    out = []
    for size, count in sizes:
        levels = 2 if size <= 256 else 3
        iters = [int(np.ceil(max_flow / 2 ** h)) for h in range(levels)]
        smooth = [2] + [4] * (levels - 1)
        for _ in range(count):
            depth = rng.uniform(3.0, 8.0)
            direction = rng.normal(size=3)
            direction[2] = abs(direction[2])
            direction /= np.linalg.norm(direction)
            # image flow of a fronto-parallel plane, per axis: (x v_z - f v_xy) / depth / rate
            # (px/frame, f = size / 2, |x| <= f), at most f (|v_xy| + sqrt(2) v_z) / depth / rate
            # over the image: the largest per-axis flow stays below max_flow (CFL-safe at N_1)
            vmag = 0.95 * max_flow * depth * rate / (size / 2.0) / (np.linalg.norm(direction[:2]) +
                                                                     np.sqrt(2.0) * direction[2])
            out.append(plane_stream(frames, int(rng.integers(1 << 30)), size, size, depth, direction * vmag, rate,
                                    levels, iters, smooth, period))
    return out


CONFIGS = {
    "plane64": plane64,
    "scene512": scene512,
    "drive": drive,
}
