"""Helpers shared by the GPU parity tests: oracle-prepared scenes imported
into the library, image comparison with the FP32/FP64 threshold carve-out."""
import numpy as np

import oracle
import scenegen
from oracle import build as ob

IMG_TOL = 1e-3  # max abs per channel (FP32 kernel vs FP64 oracle)


def flag_tol(ref):
    """Tolerance of a flagged pixel (one where an alpha came within rounding
    of the 1/255 skip threshold, or the transmittance within rounding of the
    1e-4 stop).  A splat j whose skip decision flips adds or removes its own
    term alpha_j T_j c_j, at most T_j c_max / 255, and scales the
    transmittance of every later splat by (1 - alpha_j), which moves their
    sum, itself at most T_j c_max, by at most alpha_j T_j c_max: together
    2 c_max / 255 with T_j <= 1 (a flipped stop only drops terms below
    1e-4 c_max).  c_max is the largest colour of the view's splats (colours
    are not clamped above 1); 1e-3 is added for the unflagged FP32 error."""
    rgb = ref["proj"]["rgb"]
    c_max = max(1.0, float(rgb.max()) if rgb.size else 1.0)
    return IMG_TOL + 2.0 * c_max / 255.0


def tiny_scene(links=True):
    raw = scenegen.uniform_scene()
    bp = ob.BuildParams(page_size=256, paging="morton", lo=(-5, -5, -5), hi=(5, 5, 5), voxel=10 / 32, kappa=0.5,
                        link_samples=8, links=links)
    return raw, ob.build_scene(raw, bp)


def city_scene(n=60000, n_boxes=20, extent=160.0, levels=3, fanout=8, page_size=512, sh=3, lod_method="moment"):
    raw = scenegen.city_scene(n=n, n_boxes=n_boxes, extent=extent, sh_degree=sh)
    bp = ob.BuildParams(page_size=page_size, paging="octree", lod_levels=levels, lod_fanout=fanout, lo=(-4, -4, -4),
                        hi=(extent + 4, extent + 4, 84), voxel=4.0, kappa=0.5, link_samples=4, lod_method=lod_method,
                        kmeans_iters=6)
    return raw, ob.build_scene(raw, bp)


def round16_scene(sc):
    """The scene as an fp16 pool stores it: scale, rotation and SH rounded to
    half precision (round to nearest even), position and opacity kept fp32."""
    import dataclasses
    levels = []
    for L in sc.levels:
        L = dict(L)
        for k in ("scale", "rot", "sh"):
            L[k] = L[k].astype(np.float16).astype(np.float32)
        levels.append(L)
    return dataclasses.replace(sc, levels=levels)


def import_scene(v, raw, sc, fp16=False):
    return v.vm3dgs_scene_import(sc.levels, sc.err, sc.count, sc.verts, sc.tris, sc.face_page, sc.link_ptr,
                                 sc.link_col, sc.params.page_size, sc.params.lod_fanout, raw.sh_degree, fp16=fp16)


def compare_image(gpu_img, ref):
    """gpu_img [3,H,W] float32 vs oracle render dict; returns (max_err_unflagged, n_flagged)."""
    d = np.abs(gpu_img.astype(np.float64) - ref["image"])
    flag = ref["flag"].astype(bool)
    unfl = d[:, ~flag]
    e0 = float(unfl.max()) if unfl.size else 0.0
    e1 = float(d[:, flag].max()) if flag.any() else 0.0
    assert e0 <= IMG_TOL, "max abs error %.3g on unflagged pixels" % e0
    tol = flag_tol(ref)
    assert e1 <= tol, "max abs error %.3g on flagged pixels (bound %.3g)" % (e1, tol)
    return e0, int(flag.sum())


def expected_tmask(pr, cam):
    """The kernel's per-splat tile mask as the oracle's tile rule gives it:
    the kept tiles of a rectangle of at most 64 tiles as row-major bits of
    the rectangle, 0 for culled splats and larger rectangles."""
    out = np.zeros(len(pr["vis"]), np.uint64)
    for i in np.nonzero(pr["vis"])[0]:
        x0, y0, x1, y1 = (int(t) for t in pr["rect"][i])
        w = x1 - x0
        if w * (y1 - y0) > 64:
            continue
        m = 0
        for tx, ty in oracle.splat_tiles(pr, i, cam):
            m |= 1 << ((ty - y0) * w + (tx - x0))
        out[i] = m
    return out


def city_cam(extent, k=0, width=320, height=180, tile=(16, 16)):
    """Street-level camera looking along the city from one corner."""
    eye = np.array([0.35 * extent + 3.0 * k, 0.2 * extent, 1.7 + 0.3 * k])
    tgt = eye + np.array([np.cos(0.6 + 0.05 * k), np.sin(0.6 + 0.05 * k), -0.05])
    return scenegen.look_at(eye, tgt, (0, 0, 1), width, height, 60.0, tile)
