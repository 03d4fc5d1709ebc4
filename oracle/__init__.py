"""ORACLE — plain, slow, obviously correct CPU reference of the virtual-memory
3DGS per-frame path.  TEST INFRASTRUCTURE ONLY: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import, call or link anything here.  It shares no code with the CUDA library
and never imports it; only the seeded input generator (``scenegen``) serves
both.

Layout
  build.py      offline scene preparation (numpy, FP64)
  feedback.c    visibility-buffer raster, reduction, request compaction (C)
  residency.py  LOD choice, page table, LOD controller (Python, fp32 spec)
  render.c      projection, tile binning + sort, tile ranges, blending (C, FP64)
  mlp.py        prefetcher network forward/backward/Adam (numpy, FP64)

The C files are compiled with gcc -O2 -ffp-contract=off -fno-fast-math, so
every float32 operation of a discrete decision is a single correctly rounded
IEEE operation, in the written order.  Their per-Gaussian, per-tile and
per-triangle loops may run on several OpenMP threads (set_threads; one by
default): the iterations are independent, so the results are the same.

Parity pins (tests/test_oracle_*.py) tie every function to something other
than itself: closed-form images, finite differences, quadrature, brute force,
exact format arithmetic printed in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import build as build_mod  # noqa: F401
from . import mlp, residency  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = [os.path.join(_HERE, f) for f in ("render.c", "feedback.c")]
_lib = None


def compile_oracle(force=False):
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
                               *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        compile_oracle()
        _lib = ctypes.CDLL(_SO)
        _lib.vo_bin_sort.restype = ctypes.c_int64
        _lib.vo_compact.restype = ctypes.c_int
        _lib.vo_float_bits.restype = ctypes.c_uint32
        _lib.vo_float_bits.argtypes = [ctypes.c_float]
        _lib.vo_tile_kept.restype = ctypes.c_int
        _lib.vo_set_threads(1)
    return _lib


class VoCamera(ctypes.Structure):
    _fields_ = [("view", ctypes.c_float * 12), ("campos", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32)]


def vo_camera(cam):
    c = VoCamera()
    c.view[:] = [float(v) for v in np.asarray(cam.view, np.float32).reshape(-1)]
    c.campos[:] = [float(v) for v in np.asarray(cam.campos, np.float32)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.tile_w, c.tile_h = cam.width, cam.height, cam.tile_w, cam.tile_h
    return c


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dt)


# --------------------------------------------------------------------------- render
def project(g, cam, rect_binning=False):
    """g: dict pos[n,3] scale[n,3] rot[n,4] opacity[n] sh[n,K,3] (fp32).
    ctr32/con32 are the FP32 centre and conic the tile rule reads;
    rect_binning keeps every tile of a splat's rectangle instead."""
    n = len(g["opacity"])
    K = g["sh"].shape[1]
    pos, scale, rot = _c(g["pos"], np.float32), _c(g["scale"], np.float32), _c(g["rot"], np.float32)
    op, sh = _c(g["opacity"], np.float32), _c(g["sh"], np.float32)
    out = dict(vis=np.zeros(n, np.uint8), radius=np.zeros(n, np.float32), rect=np.zeros((n, 4), np.int32),
               depth=np.zeros(n, np.float32), touched=np.zeros(n, np.int32), ctr32=np.zeros((n, 2), np.float32),
               con32=np.zeros((n, 3), np.float32), centre=np.zeros((n, 2)), conic=np.zeros((n, 3)),
               rgb=np.zeros((n, 3)), rect_binning=bool(rect_binning))
    c = vo_camera(cam)
    lib().vo_project(ctypes.c_int64(n), _p(pos), _p(scale), _p(rot), _p(op), _p(sh), ctypes.c_int(K), ctypes.byref(c),
                     _p(out["vis"]), _p(out["radius"]), _p(out["rect"]), _p(out["depth"]), _p(out["touched"]),
                     _p(out["ctr32"]), _p(out["con32"]), ctypes.c_int(1 if rect_binning else 0), _p(out["centre"]),
                     _p(out["conic"]), _p(out["rgb"]))
    return out


def tile_kept(pr, i, cam, tx, ty):
    """Is tile (tx, ty) of its rectangle one of splat i's tiles (the row rule
    of the tile binning, FP32 spec)?"""
    c = vo_camera(cam)
    u, w = pr["ctr32"][i], pr["con32"][i]
    return bool(lib().vo_tile_kept(ctypes.c_float(u[0]), ctypes.c_float(u[1]), ctypes.c_float(w[0]),
                                   ctypes.c_float(w[1]), ctypes.c_float(w[2]), ctypes.byref(c), ctypes.c_int(int(tx)),
                                   ctypes.c_int(int(ty))))


def splat_tiles(pr, i, cam):
    """Tiles (tx, ty) of splat i in row-major order."""
    if not pr["vis"][i]:
        return []
    x0, y0, x1, y1 = (int(t) for t in pr["rect"][i])
    return [(tx, ty) for ty in range(y0, y1) for tx in range(x0, x1)
            if pr["rect_binning"] or tile_kept(pr, i, cam, tx, ty)]


def set_threads(n):
    """OpenMP threads of the oracle's C loops (results do not depend on it);
    returns the count now in effect."""
    lib().vo_set_threads(int(n))
    return int(lib().vo_max_threads())


def grid_dims(cam):
    return (cam.width + cam.tile_w - 1) // cam.tile_w, (cam.height + cam.tile_h - 1) // cam.tile_h


def bin_sort(pr, vid, cam):
    M = int(pr["touched"][pr["vis"] != 0].astype(np.int64).sum())
    keys = np.zeros(max(M, 1), np.uint64)
    idx = np.zeros(max(M, 1), np.int64)
    vid = _c(vid, np.int64)
    c = vo_camera(cam)
    m = lib().vo_bin_sort(ctypes.c_int64(len(vid)), _p(pr["vis"]), _p(pr["rect"]), _p(pr["touched"]), _p(pr["ctr32"]),
                          _p(pr["con32"]), ctypes.c_int(1 if pr["rect_binning"] else 0), _p(pr["depth"]), _p(vid),
                          ctypes.byref(c), _p(keys), _p(idx), ctypes.c_int64(len(keys)))
    assert m == M, (m, M)
    return keys[:M], idx[:M]


def ranges(keys, cam):
    gx, gy = grid_dims(cam)
    r = np.zeros((gx * gy, 2), np.int64)
    lib().vo_ranges(ctypes.c_int64(len(keys)), _p(_c(keys, np.uint64)), ctypes.c_int(gx * gy), _p(r))
    return r


def blend(cam, rng, idx, pr, opacity, bg=(0.0, 0.0, 0.0)):
    img = np.zeros((3, cam.height, cam.width))
    flag = np.zeros((cam.height, cam.width), np.uint8)
    nc = np.zeros((cam.height, cam.width), np.int32)
    bgv = np.asarray(bg, np.float64)
    c = vo_camera(cam)
    lib().vo_blend(ctypes.byref(c), _p(_c(rng, np.int64)), _p(_c(idx, np.int64)), _p(pr["centre"]), _p(pr["conic"]),
                   _p(_c(opacity, np.float32)), _p(pr["rgb"]), _p(bgv), _p(img), _p(flag), _p(nc))
    return img, flag, nc


def render(g, vid, cam, bg=(0.0, 0.0, 0.0), rect_binning=False):
    """Full splat pipeline over the given Gaussians (vid = virtual ids for ties)."""
    pr = project(g, cam, rect_binning)
    keys, idx = bin_sort(pr, vid, cam)
    rng = ranges(keys, cam)
    img, flag, nc = blend(cam, rng, idx, pr, g["opacity"], bg)
    return dict(proj=pr, keys=keys, idx=idx, ranges=rng, image=img, flag=flag, n_contrib=nc)


def sh_basis(dirs):
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((len(dirs), 16))
    lib().vo_sh_basis(ctypes.c_int64(len(dirs)), _p(dirs), _p(out))
    return out


# --------------------------------------------------------------------------- feedback
def feedback_raster(verts, tris, face_page, cam, ds):
    Wf, Hf = (cam.width + ds - 1) // ds, (cam.height + ds - 1) // ds
    buf = np.full(Wf * Hf, np.iinfo(np.uint64).max, np.uint64)
    c = vo_camera(cam)
    lib().vo_feedback_raster(ctypes.c_int64(len(tris)), _p(_c(verts, np.float32)), _p(_c(tris, np.int32)),
                             _p(_c(face_page, np.int32)), ctypes.byref(c), ctypes.c_int(ds), _p(buf))
    return buf.reshape(Hf, Wf)


def feedback_reduce(buf, n_vp, link_ptr, link_col, use_links=True):
    req = np.zeros(n_vp, np.uint32)
    direct = np.zeros(n_vp, np.uint8)
    b = _c(buf, np.uint64).reshape(-1)
    lp = _c(link_ptr, np.int64)
    lc = _c(link_col, np.int32) if len(link_col) else np.zeros(1, np.int32)
    lib().vo_feedback_reduce(ctypes.c_int64(len(b)), _p(b), ctypes.c_int(n_vp), _p(lp), _p(lc),
                             ctypes.c_int(1 if use_links else 0), _p(req), _p(direct))
    return req, direct


def compact(req, direct):
    n = len(req)
    pg = np.zeros(max(n, 1), np.int32)
    en = np.zeros(max(n, 1), np.uint32)
    di = np.zeros(max(n, 1), np.uint8)
    m = lib().vo_compact(ctypes.c_int(n), _p(_c(req, np.uint32)), _p(_c(direct, np.uint8)), _p(pg), _p(en), _p(di))
    return pg[:m], en[:m], di[:m]


def float_bits(f):
    return lib().vo_float_bits(float(f))


# --------------------------------------------------------------------------- frame
def gather_draw(scene, draw, weights=None):
    """Gaussians of the draw list [(p, l, e, s)] in draw order, with virtual
    ids 2 p page_size + k page_size + slot (k: the item's rank among the
    page's items, 1 for the old level of a cross-fade); weights (optional,
    float32 per item) scale the opacities in float32."""
    ps = scene.params.page_size
    parts = {k: [] for k in ("pos", "scale", "rot", "opacity", "sh")}
    vids = []
    prev = None
    for i, (p, l, e, s) in enumerate(draw):
        lv = scene.levels[l]
        for k in parts:
            parts[k].append(lv[k][p])
        if weights is not None and weights[i] != np.float32(1):
            parts["opacity"][-1] = (lv["opacity"][p] * np.float32(weights[i])).astype(np.float32)
        k = 1 if prev == p else 0
        prev = p
        vids.append((2 * p + k) * ps + np.arange(lv["opacity"].shape[1], dtype=np.int64))
    if not draw:
        K = scene.levels[0]["sh"].shape[2]
        return dict(pos=np.zeros((0, 3), np.float32), scale=np.zeros((0, 3), np.float32),
                    rot=np.zeros((0, 4), np.float32), opacity=np.zeros(0, np.float32),
                    sh=np.zeros((0, K, 3), np.float32)), np.zeros(0, np.int64)
    return {k: np.concatenate(v, 0) for k, v in parts.items()}, np.concatenate(vids)


def full_scene(scene):
    """Every page at level 0 in page order (the no-virtual-memory reference)."""
    draw = [(p, 0, p, 0) for p in range(scene.n_pages)]
    return gather_draw(scene, draw)


def frame(scene, pt, cam, ds=4, links=True, render_image=True):
    """One virtual-memory frame: feedback -> reduce -> compact -> LOD -> page
    table -> render of the drawn pages -> controller."""
    buf = feedback_raster(scene.verts, scene.tris, scene.face_page, cam, ds)
    req, direct = feedback_reduce(buf, scene.n_pages, scene.link_ptr, scene.link_col, links)
    pages, enc, di = compact(req, direct)
    lv = residency.lod_select(pages, enc, scene.err, cam.fy, pt.tau, pt.rp.lod)
    up = residency.update(pt, pages, enc, di, lv)
    out = dict(buf=buf, req=req, direct=direct, pages=pages, enc=enc, levels=lv, update=up, tau=pt.tau)
    if render_image:
        g, vid = gather_draw(scene, up["draw"], up["draw_w"])
        out["render"] = render(g, vid, cam)
    residency.control(pt, up["usage"], up["draw"])
    return out
