"""Pins of the page-determination oracle: exact coverage of pixel-aligned
quads, a brute-force (every pixel, Python integers) rasteriser, the
perspective-correct depth of a plane, near-plane clipping and a dictionary
recount of the reduction."""
import math
import struct

import numpy as np

import oracle
import scenegen


def _cam(w=64, h=48, f=40.0):
    return scenegen.Camera(view=np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32),
                           campos=np.zeros(3, np.float32), fx=np.float32(f), fy=np.float32(f),
                           cx=np.float32(w / 2), cy=np.float32(h / 2), width=w, height=h)


def _quad_at_depth(x0, y0, x1, y1, z, f, cx, cy):
    """World quad at depth z whose projection is the pixel rectangle [x0,x1) x [y0,y1)
    (edges half a pixel outside the covered centres)."""
    def back(u, v):
        return ((u - cx) * z / f, (v - cy) * z / f, z)
    v = [back(x0, y0), back(x1, y0), back(x1, y1), back(x0, y1)]
    return np.array(v, np.float32), np.array([[0, 1, 2], [0, 2, 3]], np.int32)


def test_quad_covers_rectangle_exactly_once():
    cam = _cam()
    verts, tris = _quad_at_depth(10.25, 5.25, 30.75, 20.75, 2.0, 40.0, 32.0, 24.0)
    b = [oracle.feedback_raster(verts, tris[i:i + 1], np.array([7], np.int32), cam, 1) for i in range(2)]
    cov = (b[0] != np.iinfo(np.uint64).max).astype(int) + (b[1] != np.iinfo(np.uint64).max).astype(int)
    yy, xx = np.mgrid[0:48, 0:64] + 0.5
    inside = (xx > 10.25) & (xx < 30.75) & (yy > 5.25) & (yy < 20.75)
    np.testing.assert_array_equal(cov, inside.astype(int))
    both = oracle.feedback_raster(verts, tris, np.array([7, 7], np.int32), cam, 1)
    # page id + 1 in the low word, depth = 2.0 (within 2 ulp) in the high word
    z = (both[inside] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert np.all(np.abs(z - 2.0) <= 2 * np.spacing(np.float32(2.0)))
    assert np.all((both[inside] & np.uint64(0xFFFFFFFF)) == 8)


def _snap(v):
    return int(np.rint(np.float32(v) * np.float32(256.0)))


def _bruteforce_raster(verts, tris, face_page, cam, ds):
    """Every pixel of the buffer against every (unclipped, in-front) triangle,
    edge functions in Python integers, same ownership rule stated in words: a
    pixel exactly on an edge belongs to the triangle for which the edge runs
    upwards (dy < 0) or, if horizontal, rightwards."""
    Wf, Hf = (cam.width + ds - 1) // ds, (cam.height + ds - 1) // ds
    f32 = np.float32
    fx, fy, cx, cy = f32(cam.fx) / f32(ds), f32(cam.fy) / f32(ds), f32(cam.cx) / f32(ds), f32(cam.cy) / f32(ds)
    buf = np.full((Hf, Wf), (1 << 64) - 1, dtype=object)
    for t, tri in enumerate(tris):
        P = []
        for k in tri:
            x, y, z = (f32(v) for v in verts[k])
            V = cam.view
            cxp = f32(f32(f32(V[0, 0] * x) + f32(V[0, 1] * y)) + f32(V[0, 2] * z)) + V[0, 3]
            cyp = f32(f32(f32(V[1, 0] * x) + f32(V[1, 1] * y)) + f32(V[1, 2] * z)) + V[1, 3]
            czp = f32(f32(f32(V[2, 0] * x) + f32(V[2, 1] * y)) + f32(V[2, 2] * z)) + V[2, 3]
            assert czp > 0.2
            P.append((_snap(f32(fx * f32(cxp / czp)) + cx), _snap(f32(fy * f32(cyp / czp)) + cy), czp))
        for j in range(Hf):
            for i in range(Wf):
                px, py = i * 256 + 128, j * 256 + 128
                (X0, Y0, Z0), (X1, Y1, Z1), (X2, Y2, Z2) = P
                area = (X1 - X0) * (Y2 - Y0) - (Y1 - Y0) * (X2 - X0)
                if area == 0:
                    continue
                vs = P if area > 0 else [P[0], P[2], P[1]]
                area = abs(area)
                E = []
                ok = True
                for a, b in ((1, 2), (2, 0), (0, 1)):
                    dx, dy = vs[b][0] - vs[a][0], vs[b][1] - vs[a][1]
                    e = dx * (py - vs[a][1]) - dy * (px - vs[a][0])
                    own = dy < 0 or (dy == 0 and dx > 0)
                    if not (e > 0 or (e == 0 and own)):
                        ok = False
                    E.append(e)
                if not ok:
                    continue
                # 1/z is affine in screen space: z = E_sum / sum_k E_k / z_k
                ws = [f32(f32(1.0) / vs[k][2]) for k in range(3)]
                s = f32(f32(f32(E[0]) * ws[0]) + f32(f32(E[1]) * ws[1])) + f32(f32(E[2]) * ws[2])
                zp = f32(f32(area) / s)
                key = (struct.unpack("<I", struct.pack("<f", zp))[0] << 32) | (int(face_page[t]) + 1)
                buf[j, i] = min(buf[j, i], key)
    return buf.astype(np.uint64)


def test_raster_matches_bruteforce_every_pixel():
    rng = np.random.default_rng(8)
    cam = _cam(w=37, h=29, f=30.0)
    n = 40
    verts = np.stack([rng.uniform(-1.5, 1.5, 3 * n), rng.uniform(-1.2, 1.2, 3 * n), rng.uniform(0.5, 4.0, 3 * n)],
                     1).astype(np.float32)
    tris = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    pages = rng.integers(-1, 9, n).astype(np.int32)
    for ds in (1, 2):
        got = oracle.feedback_raster(verts, tris, pages, cam, ds)
        ref = _bruteforce_raster(verts, tris, pages, cam, ds)
        np.testing.assert_array_equal(got, ref)


def test_near_plane_clipping_keeps_visible_part():
    """A large floor triangle passing under and behind the camera: after
    clipping, the covered set equals the brute-force coverage of the part in
    front of z = 0.2 (computed here analytically for a plane y = 1)."""
    cam = _cam(w=64, h=48, f=40.0)
    verts = np.array([[-50, 1.0, -10.0], [50, 1.0, -10.0], [0, 1.0, 80.0]], np.float32)
    buf = oracle.feedback_raster(verts, np.array([[0, 1, 2]], np.int32), np.array([3], np.int32), cam, 1)
    covered = buf != np.iinfo(np.uint64).max
    # rows below the horizon (v > cy) see the floor; the triangle is wide enough to
    # fill them except far away where its apex narrows it
    assert covered[30:, 20:44].all()
    assert not covered[:23].any()
    # depth on a row: the floor y = 1 seen at v gives z = f / (v - cy)
    z = (buf[40, 32] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert abs(float(z) - 40.0 / (40.5 - 24.0)) < 1e-4


def test_reduce_and_compact_bruteforce():
    rng = np.random.default_rng(1)
    n_vp = 20
    Hf, Wf = 12, 16
    z = rng.uniform(0.5, 50.0, (Hf, Wf)).astype(np.float32)
    page1 = rng.integers(0, n_vp + 1, (Hf, Wf))
    buf = (z.view(np.uint32).astype(np.uint64) << np.uint64(32)) | page1.astype(np.uint64)
    buf[0, :3] = np.iinfo(np.uint64).max
    rows = {q: sorted(set(rng.integers(0, n_vp, 3).tolist()) - {q}) for q in range(n_vp)}
    ptr = np.zeros(n_vp + 1, np.int64)
    for q in range(n_vp):
        ptr[q + 1] = ptr[q] + len(rows[q])
    col = np.array([c for q in range(n_vp) for c in rows[q]], np.int32)
    for links in (True, False):
        req, direct = oracle.feedback_reduce(buf, n_vp, ptr, col, links)
        want, wd = {}, set()
        for j in range(Hf):
            for i in range(Wf):
                if int(buf[j, i]) == (1 << 64) - 1 or page1[j, i] == 0:
                    continue
                p = int(page1[j, i]) - 1
                enc = 0xFFFFFFFF - int(z[j, i].view(np.uint32))
                wd.add(p)
                for q in [p] + (rows[p] if links else []):
                    want[q] = max(want.get(q, 0), enc)
        assert {int(p): int(v) for p, v in enumerate(req) if v} == want
        assert set(np.nonzero(direct)[0].tolist()) == wd
        pg, en, di = oracle.compact(req, direct)
        assert pg.tolist() == sorted(want) and [int(e) for e in en] == [want[p] for p in sorted(want)]
        # nearer depth -> larger request word
    a, b = np.float32(1.0), np.float32(2.0)
    assert 0xFFFFFFFF - int(a.view(np.uint32)) > 0xFFFFFFFF - int(b.view(np.uint32)) > 0
