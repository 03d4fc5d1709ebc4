"""Batched multi-view rendering: the batch (one projection, one sort over all
views' pairs, one persistent blend with per-view tile shapes) gives every
view the same sorted pairs as rendering it alone and the same image; a
captured CUDA graph replayed with new poses equals the direct batch; the
autotuner returns valid shapes."""
import numpy as np
import pytest

import scenegen
from _common import import_scene
from oracle import build as ob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_19415_b300 as mod
    return mod


def _scene(v):
    raw = scenegen.blob_scene(n=60_000, n_blobs=30, lo=0.0, hi=30.0, sh_degree=2, seed=12)
    sc = ob.build_scene(raw, ob.BuildParams(page_size=512, paging="octree", lo=(-5, -5, -5), hi=(35, 35, 35),
                                            voxel=1.0, kappa=1.0, link_samples=2))
    return sc, import_scene(v, raw, sc, fp16=True)


def _views(n, tiles):
    cams = scenegen.batched_views(n_views=n, seed=77, centre=(15, 15, 15), radius=40.0)
    out = []
    for k, c in enumerate(cams):
        c.width, c.height = min(c.width, 640), min(c.height, 400)
        c.cx, c.cy = np.float32(c.width / 2), np.float32(c.height / 2)
        c.tile_w, c.tile_h = tiles[k % len(tiles)]
        out.append(c)
    return out


def test_batched_equals_single_views(v):
    import torch
    sc, scene = _scene(v)
    cams = _views(6, [(16, 16), (8, 8), (32, 8)])
    cfg = v.RenderConfig(max_width=640, max_height=400, lod=False, fp16_pool=True, max_views=8,
                         staging_bytes=1 << 40)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.request_all()
    r.update_residency()
    singles, keys = [], []
    for c in cams:
        singles.append(r.render([c])[0].cpu().numpy())
        keys.append(r.debug(v.DBG_KEYS, np.uint64))
    imgs = [im.cpu().numpy() for im in r.render_batched(cams)]
    bk = r.debug(v.DBG_KEYS, np.uint64)
    # split the batch's keys by view (global tile -> view, local tile)
    off = [0]
    for c in cams:
        off.append(off[-1] + ((c.width + c.tile_w - 1) // c.tile_w) * ((c.height + c.tile_h - 1) // c.tile_h))
    tile = (bk >> np.uint64(32)).astype(np.int64)
    for k, c in enumerate(cams):
        sel = (tile >= off[k]) & (tile < off[k + 1])
        local = ((tile[sel] - off[k]).astype(np.uint64) << np.uint64(32)) | (bk[sel] & np.uint64(0xFFFFFFFF))
        np.testing.assert_array_equal(local, keys[k])
        np.testing.assert_allclose(imgs[k], singles[k], atol=2e-6)
    assert r.stats()["status"] == 0


def test_graph_replay_matches_direct(v):
    import torch
    sc, scene = _scene(v)
    cams = _views(5, [(16, 16), (32, 8)])
    cfg = v.RenderConfig(max_width=640, max_height=400, lod=False, fp16_pool=True, max_views=8,
                         staging_bytes=1 << 40)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.request_all()
    r.update_residency()
    r.render_batched(cams)  # warm (first launches set kernel attributes)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gimgs = r.batch_graph_capture(cams, stream=s)
    moved = _views(5, [(16, 16), (32, 8)])
    for c in moved:
        c.view[:, 3] += np.float32(1.5)
    with torch.cuda.stream(s):
        r.batch_graph_launch(moved, stream=s)
    s.synchronize()
    got = [im.cpu().numpy() for im in gimgs]
    want = [im.cpu().numpy() for im in r.render_batched(moved)]
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_autotuner_picks_valid_shapes(v):
    sc, scene = _scene(v)
    cams = _views(6, [(16, 16)])
    cfg = v.RenderConfig(max_width=640, max_height=400, lod=False, fp16_pool=True, max_views=8,
                         staging_bytes=1 << 40)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.request_all()
    r.update_residency()
    tuned = r.autotune_tiles(cams, repeats=2)
    assert all((c.tile_w, c.tile_h) in ((16, 16), (8, 8), (32, 8)) for c in tuned)
    imgs = r.render_batched(tuned)
    assert r.stats()["status"] == 0 and all(np.isfinite(im.cpu().numpy()).all() for im in imgs)


def test_interleaved_streams_equal_one_stream(v):
    """Single-view renders on two streams (the two render contexts) and
    batched renders (context 0) interleaved with no host sync: every image
    equals the same sequence rendered on one stream."""
    import torch
    sc, scene = _scene(v)
    cams = _views(6, [(16, 16), (8, 8), (32, 8)])
    cfg = v.RenderConfig(max_width=640, max_height=400, lod=False, fp16_pool=True, max_views=8,
                         staging_bytes=1 << 40)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.request_all()
    r.update_residency()
    plan = [("one", 0), ("one", 1), ("batch", None), ("one", 2), ("one", 3), ("batch", None), ("one", 4)]

    def run(streams):
        out = []
        for k, (what, i) in enumerate(plan):
            s = streams[k % len(streams)]
            if what == "one":
                img = torch.empty((3, cams[i].height, cams[i].width), dtype=torch.float32, device="cuda")
                r.render([cams[i]], [img], s)
                out.append([img])
            else:
                imgs = [torch.empty((3, c.height, c.width), dtype=torch.float32, device="cuda") for c in cams]
                r.render_batched(cams, imgs, s)
                out.append(imgs)
        torch.cuda.synchronize()
        return [[im.cpu().numpy() for im in group] for group in out]

    ref = run([torch.cuda.current_stream()])
    got = run([torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()])
    for a, b in zip(ref, got):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert r.stats()["status"] == 0


def test_batched_views_against_oracle(v):
    """Every view of a batch (uneven sizes, 16x16 / 8x8 / 32x8 tiles, fp16
    pool, SH2) against the oracle run on the fp16-rounded attributes of the
    drawn Gaussians: the view's share of the batch's sorted keys (global tile
    mapped back to the view's tile) and values (record index mapped back to
    the view's splat) and its tile ranges bit-exact, its image within the
    FP32 tolerance."""
    import oracle
    from _common import compare_image, round16_scene
    sc, scene = _scene(v)
    cams = _views(6, [(16, 16), (8, 8), (32, 8)])
    cfg = v.RenderConfig(max_width=640, max_height=400, lod=False, fp16_pool=True, max_views=8,
                         staging_bytes=1 << 40)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.request_all()
    r.update_residency()
    imgs = [im.cpu().numpy() for im in r.render_batched(cams)]
    st = r.stats()
    assert st["status"] == 0
    bk = r.debug(v.DBG_KEYS, np.uint64)
    bv = r.debug(v.DBG_VALUES, np.uint32).astype(np.int64)
    brng = r.debug(v.DBG_RANGES, np.uint32).reshape(-1, 2).astype(np.int64)
    g, vid = oracle.full_scene(round16_scene(sc))
    N = len(vid)
    assert st["drawn_gaussians"] == N
    off = [0]
    for c in cams:
        off.append(off[-1] + ((c.width + c.tile_w - 1) // c.tile_w) * ((c.height + c.tile_h - 1) // c.tile_h))
    tile = (bk >> np.uint64(32)).astype(np.int64)
    for k, c in enumerate(cams):
        ref = oracle.render(g, vid, c)
        sel = (tile >= off[k]) & (tile < off[k + 1])
        local = ((tile[sel] - off[k]).astype(np.uint64) << np.uint64(32)) | (bk[sel] & np.uint64(0xFFFFFFFF))
        np.testing.assert_array_equal(local, ref["keys"])
        np.testing.assert_array_equal(bv[sel] - k * N, ref["idx"])
        first = np.flatnonzero(sel)[0] if sel.any() else 0
        rk = brng[off[k]:off[k + 1]]
        rk = np.where(rk[:, 1:] > rk[:, :1], rk - first, 0)
        np.testing.assert_array_equal(rk, ref["ranges"])
        compare_image(imgs[k], ref)


def test_multi_camera_feedback_against_oracle(v):
    """Page determination over several cameras in one call: the request words
    are the maximum over the cameras of each camera's oracle request words
    (links included), the direct flags their union, and the request list the
    pages with a non-zero word."""
    import oracle
    sc, scene = _scene(v)
    cams = _views(4, [(16, 16)])
    cfg = v.RenderConfig(max_width=640, max_height=400, lod=False, fp16_pool=True, max_views=8,
                         staging_bytes=1 << 40)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.render_feedback(cams)
    req = np.zeros(sc.n_pages, np.uint32)
    direct = np.zeros(sc.n_pages, np.uint8)
    for c in cams:
        buf = oracle.feedback_raster(sc.verts, sc.tris, sc.face_page, c, 4)
        q, d = oracle.feedback_reduce(buf, sc.n_pages, sc.link_ptr, sc.link_col, True)
        req = np.maximum(req, q)
        direct |= d
    assert (req != 0).sum() > 10
    np.testing.assert_array_equal(r.debug(v.DBG_REQ, np.uint32), req)
    np.testing.assert_array_equal(r.debug(v.DBG_DIRECT, np.uint8), direct)
    r.update_residency()
    reqs = r.debug(v.DBG_REQUESTS, np.int32).reshape(-1, 4)
    np.testing.assert_array_equal(reqs[:, 0], np.flatnonzero(req))
    np.testing.assert_array_equal(reqs[:, 1].view(np.uint32), req[req != 0])


def test_batched_vq_pool_equals_single_views(v):
    """The batched projection reads VQ records and the codebook as the
    single-view projection does."""
    sc, scene = _scene(v)
    scene.quantize_sh(64, 4)
    cams = _views(4, [(16, 16), (8, 8)])
    cfg = v.RenderConfig(max_width=640, max_height=400, lod=False, fp16_pool=v.POOL_VQ, max_views=8,
                         staging_bytes=1 << 40)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.request_all()
    r.update_residency()
    singles = [r.render([c])[0].cpu().numpy() for c in cams]
    imgs = [im.cpu().numpy() for im in r.render_batched(cams)]
    for a, b in zip(imgs, singles):
        np.testing.assert_allclose(a, b, atol=2e-6)
    assert r.stats()["status"] == 0


def test_batched_cross_fade_equals_single_views(v):
    """With an LOD cross-fade running, the batched projection applies the
    draw items' opacity weights as the single-view projection does."""
    from _common import city_scene
    raw, sc = city_scene()
    scene = import_scene(v, raw, sc)
    cfg = v.RenderConfig(max_width=200, max_height=120, lod=True, max_views=4, staging_bytes=12 * 512 * 236,
                         tau0=10.0, step0=1.5, lod_fade_frames=4)
    r = v.Renderer(scene, cfg, pool_slots=24)
    faded = 0
    for k in range(10):
        cams = [scenegen.look_at((80, -260 + 15 * k, 40 - 2 * k), (80, 80, 0), (0, 0, 1), 200, 120, 60.0, (16, 16)),
                scenegen.look_at((60, -250 + 15 * k, 30), (80, 80, 0), (0, 0, 1), 160, 96, 70.0, (8, 8))]
        r.render_feedback(cams)
        r.update_residency()
        st = r.stats()
        faded += st["fading"]
        singles = [r.render([c])[0].cpu().numpy() for c in cams]
        imgs = [im.cpu().numpy() for im in r.render_batched(cams)]
        for a, b in zip(imgs, singles):
            np.testing.assert_allclose(a, b, atol=2e-6)
    assert faded > 0 and r.stats()["status"] == 0
