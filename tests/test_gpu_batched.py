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
