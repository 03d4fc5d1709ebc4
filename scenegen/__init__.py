"""Seeded synthetic inputs shared by the oracle tests and the GPU benchmark.

This module only makes inputs: raw Gaussian attributes in the layout of the
3DGS PLY export (Kerbl et al.) and camera paths.  It holds none of the
method's arithmetic (no decoding, paging, LOD, proxy, projection or
blending); both the oracle and the CUDA library consume what it returns.

The per-element random numbers come from ``gen.c`` (counter-based SplitMix64),
compiled on first use into ``libscenegen.so`` next to this file.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libscenegen.so")
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", src, "-o", _SO, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class RawGaussians:
    """Raw Kerbl-format attributes.  f_rest is channel-major [n][3][K-1]."""
    pos: np.ndarray        # [n,3] f32
    log_scale: np.ndarray  # [n,3] f32
    rot: np.ndarray        # [n,4] f32, (w,x,y,z), not necessarily unit
    op_logit: np.ndarray   # [n]   f32
    f_dc: np.ndarray       # [n,3] f32
    f_rest: np.ndarray     # [n,3,K-1] f32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def subset(self, idx) -> "RawGaussians":
        return RawGaussians(self.pos[idx], self.log_scale[idx], self.rot[idx], self.op_logit[idx],
                            self.f_dc[idx], self.f_rest[idx], self.sh_degree)


def _alloc(n, sh_degree):
    k1 = (sh_degree + 1) ** 2 - 1
    return (np.empty((n, 3), np.float32), np.empty((n, 3), np.float32), np.empty((n, 4), np.float32),
            np.empty((n,), np.float32), np.empty((n, 3), np.float32), np.empty((n, 3, k1), np.float32))


def uniform_scene(n=16384, seed=1001, lo=-5.0, hi=5.0, ls_mu=-4.0, ls_sd=0.5, op_mu=0.0, op_sd=1.0,
                  sh_degree=0, rest_sd=0.1) -> RawGaussians:
    """Positions uniform in [lo,hi]^3 (the 16,384-Gaussian 10 m cube scene)."""
    lib = _load()
    a = _alloc(n, sh_degree)
    lib.sg_uniform(ctypes.c_int64(n), ctypes.c_uint64(seed), ctypes.c_double(lo), ctypes.c_double(hi),
                   ctypes.c_double(ls_mu), ctypes.c_double(ls_sd), ctypes.c_double(op_mu), ctypes.c_double(op_sd),
                   ctypes.c_int(sh_degree), ctypes.c_double(rest_sd), *[_p(x) for x in a])
    return RawGaussians(*a, sh_degree)


def blob_scene(n=1_000_000, seed=1002, n_blobs=200, blob_sigma=0.5, lo=0.0, hi=50.0, ls_mu=-4.0, ls_sd=0.5,
               op_mu=0.0, op_sd=1.0, sh_degree=3, rest_sd=0.1) -> RawGaussians:
    """n Gaussians in n_blobs isotropic clusters (std blob_sigma) in [lo,hi]^3."""
    lib = _load()
    a = _alloc(n, sh_degree)
    lib.sg_blobs(ctypes.c_int64(n), ctypes.c_uint64(seed), ctypes.c_int(n_blobs), ctypes.c_double(blob_sigma),
                 ctypes.c_double(lo), ctypes.c_double(hi), ctypes.c_double(ls_mu), ctypes.c_double(ls_sd),
                 ctypes.c_double(op_mu), ctypes.c_double(op_sd), ctypes.c_int(sh_degree), ctypes.c_double(rest_sd),
                 *[_p(x) for x in a])
    return RawGaussians(*a, sh_degree)


def city_scene(n=50_000_000, seed=1003, n_boxes=5000, extent=2000.0, ground_frac=0.3, op_mu=2.0, op_sd=1.0,
               sh_degree=3, rest_sd=0.1) -> RawGaussians:
    """Ground plane plus axis-aligned boxes (the 2 km x 2 km city scene), world z up."""
    lib = _load()
    a = _alloc(n, sh_degree)
    cdf = np.empty(n_boxes, np.float64)
    lib.sg_city(ctypes.c_int64(n), ctypes.c_uint64(seed), ctypes.c_int(n_boxes), ctypes.c_double(extent),
                ctypes.c_double(ground_frac), ctypes.c_double(op_mu), ctypes.c_double(op_sd), ctypes.c_int(sh_degree),
                ctypes.c_double(rest_sd), _p(cdf), *[_p(x) for x in a])
    return RawGaussians(*a, sh_degree)


def city_boxes(seed=1003, n_boxes=5000, extent=2000.0) -> np.ndarray:
    out = np.empty((n_boxes, 5), np.float64)
    _load().sg_city_boxes(ctypes.c_uint64(seed), ctypes.c_int(n_boxes), ctypes.c_double(extent), _p(out))
    return out


def u01(seed, stream, n) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().sg_u01(ctypes.c_uint64(seed), ctypes.c_uint64(stream), ctypes.c_int64(n), _p(out))
    return out


# ----------------------------------------------------------------------------- cameras

@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (+x right, +y down, +z forward).

    view is the 3x4 world-to-camera matrix [R | t]; campos the centre in world
    coordinates.  All values are the float32 numbers both sides consume."""
    view: np.ndarray   # [3,4] f32
    campos: np.ndarray  # [3] f32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    tile_w: int = 16
    tile_h: int = 16


def look_at(eye, target, up, width, height, fov_y_deg, tile=(16, 16)) -> Camera:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    fy = 0.5 * height / math.tan(math.radians(fov_y_deg) / 2)
    view = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    return Camera(view, eye.astype(np.float32), np.float32(fy), np.float32(fy), np.float32(width / 2),
                  np.float32(height / 2), width, height, tile[0], tile[1])


def tiny_camera(width=256, height=256, fov_y_deg=60.0, dist=15.0, tile=(16, 16)) -> Camera:
    """Camera at distance `dist` on the -z axis looking at the origin."""
    return look_at((0, 0, -dist), (0, 0, 0), (0, -1, 0), width, height, fov_y_deg, tile)


def _catmull_rom(pts, t):
    n = len(pts) - 1
    s = min(max(t, 0.0), 1.0) * (n - 1e-9)
    i = int(s)
    u = s - i
    p0 = pts[max(i - 1, 0)]
    p1, p2 = pts[i], pts[i + 1]
    p3 = pts[min(i + 2, n)]
    return 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)


def orbit_fly_path(n_frames=300, seed=2002, centre=(25.0, 25.0, 25.0), radius=60.0, height=25.0, lo=0.0, hi=50.0,
                   width=1920, height_px=1080, fov_y_deg=90.0 * 1080 / 1920, tile=(16, 16)):
    """Half orbit around the blob cube, half Catmull-Rom flythrough of 6 seeded points.

    The vertical FoV default gives a 90 degree horizontal FoV at 16:9."""
    c = np.asarray(centre, np.float64)
    cams = []
    n_orbit = n_frames // 2
    for k in range(n_orbit):
        a = 2 * math.pi * k / n_orbit
        eye = c + np.array([radius * math.cos(a), radius * math.sin(a), height])
        cams.append(look_at(eye, c, (0, 0, 1), width, height_px, fov_y_deg, tile))
    u = u01(seed, 1, 18).reshape(6, 3)
    pts = [c + np.array([radius * math.cos(0), 0.0, height])] + [lo + (hi - lo) * u[i] for i in range(6)]
    pts = np.array(pts)
    n_fly = n_frames - n_orbit
    for k in range(n_fly):
        t = k / max(n_fly - 1, 1)
        eye = _catmull_rom(pts, t)
        ahead = _catmull_rom(pts, min(t + 0.02, 1.0))
        if np.linalg.norm(ahead - eye) < 1e-6:
            ahead = eye + (eye - _catmull_rom(pts, t - 0.02))
        cams.append(look_at(eye, ahead, (0, 0, 1), width, height_px, fov_y_deg, tile))
    return cams


def city_walk_path(n_frames=1000, seed=2003, scene_seed=1003, n_boxes=5000, extent=2000.0, eye_h=1.7, step=0.05,
                   width=1920, height_px=1080, fov_y_deg=90.0 * 1080 / 1920, tile=(16, 16)):
    """Walking-speed street-level flythrough (5 cm per frame) with a slowly sweeping yaw.

    The start is the free point nearest the centre of the city (not inside a box)."""
    boxes = city_boxes(scene_seed, n_boxes, extent)

    def inside(p):
        return np.any((p[0] >= boxes[:, 0] - 1) & (p[0] <= boxes[:, 0] + boxes[:, 2] + 1) &
                      (p[1] >= boxes[:, 1] - 1) & (p[1] <= boxes[:, 1] + boxes[:, 3] + 1))

    u = u01(seed, 2, 4096)
    start = None
    for k in range(2048):
        p = np.array([extent * (0.4 + 0.2 * u[2 * k]), extent * (0.4 + 0.2 * u[2 * k + 1])])
        if not inside(p):
            start = p
            break
    if start is None:
        start = np.array([extent / 2, extent / 2])
    yaw0 = 2 * math.pi * u01(seed, 3, 1)[0]
    cams = []
    p = start.copy()
    for k in range(n_frames):
        heading = yaw0 + 0.3 * math.sin(2 * math.pi * k / 500.0)
        look = heading + 0.5 * math.sin(2 * math.pi * k / 170.0)
        eye = np.array([p[0], p[1], eye_h])
        tgt = eye + np.array([math.cos(look), math.sin(look), -0.02])
        cams.append(look_at(eye, tgt, (0, 0, 1), width, height_px, fov_y_deg, tile))
        p = p + step * np.array([math.cos(heading), math.sin(heading)])
    return cams


def random_fly_path(n_frames, seed, lo=0.0, hi=50.0, speed=0.25, turn_every=0, width=1920, height_px=1080,
                    fov_y_deg=90.0 * 1080 / 1920, tile=(16, 16), margin=10.0):
    """Seeded flythrough around the blob cube.

    With turn_every > 0 the heading jumps by +-90 degrees every turn_every frames
    (the abrupt-turn held-out trajectories); otherwise it drifts smoothly."""
    u = u01(seed, 4, 8 + 4 * n_frames)
    c = 0.5 * (lo + hi)
    eye = np.array([lo - margin + (hi - lo + 2 * margin) * u[0], lo - margin + (hi - lo + 2 * margin) * u[1],
                    c + (hi - lo) * (u[2] - 0.5) * 0.5])
    yaw = 2 * math.pi * u[3]
    pitch = 0.2 * (u[4] - 0.5)
    cams = []
    for k in range(n_frames):
        if turn_every > 0 and k > 0 and k % turn_every == 0:
            yaw += (math.pi / 2) * (1 if u[8 + 4 * k] < 0.5 else -1)
        elif turn_every == 0:
            yaw += 0.05 * (u[8 + 4 * k] - 0.5)
        # steer back towards the cube when leaving it
        to_c = np.array([c, c, c]) - eye
        if np.linalg.norm(to_c[:2]) > 0.9 * (hi - lo) and turn_every == 0:
            yaw = 0.9 * yaw + 0.1 * math.atan2(to_c[1], to_c[0])
        d = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
        cams.append(look_at(eye, eye + d, (0, 0, 1), width, height_px, fov_y_deg, tile))
        eye = eye + speed * d
    return cams


def batched_views(n_views=64, seed=2005, centre=(25.0, 25.0, 25.0), radius=60.0, tile=(16, 16)):
    """Cameras of uneven resolution (log-uniform between 512x512 and 1920x1080 pixels),
    vertical FoV U[40, 90] degrees, placed on a sphere around the blob cube."""
    u = u01(seed, 5, 6 * n_views)
    c = np.asarray(centre, np.float64)
    cams = []
    lo_px, hi_px = math.log(512 * 512), math.log(1920 * 1080)
    for k in range(n_views):
        area = math.exp(lo_px + (hi_px - lo_px) * u[6 * k])
        aspect = 1.0 + (1920 / 1080 - 1.0) * u[6 * k + 1]
        h = int(round(math.sqrt(area / aspect) / 8)) * 8
        w = int(round(h * aspect / 8)) * 8
        w, h = min(max(w, 512), 1920), min(max(h, 512 if w < 1920 else 512), 1080)
        fov = 40.0 + 50.0 * u[6 * k + 2]
        az = 2 * math.pi * u[6 * k + 3]
        el = math.asin(2 * u[6 * k + 4] - 1) * 0.6
        eye = c + radius * np.array([math.cos(az) * math.cos(el), math.sin(az) * math.cos(el), math.sin(el)])
        cams.append(look_at(eye, c, (0, 0, 1), w, h, fov, tile))
    return cams
