"""GPU parity of the splatting path against the oracle, through the C ABI:
discrete per-Gaussian results, the sorted (tile, depth) pairs and tile
ranges bit-exact; continuous results and images within the FP32 tolerance."""
import numpy as np
import pytest

import oracle
import scenegen
from _common import compare_image, expected_tmask, import_scene, tiny_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_19415_b300 as mod
    return mod


def _full_render(v, raw, sc, cam, fp16=False, separate_values=False, sort_mode=0, vq_codes=0):
    scene = import_scene(v, raw, sc, fp16=fp16)
    if vq_codes:
        scene.quantize_sh(vq_codes, 8)
    cfg = v.RenderConfig(max_width=cam.width, max_height=cam.height, lod=False, staging_bytes=1 << 40,
                         fp16_pool=v.POOL_VQ if vq_codes else fp16, separate_values=separate_values,
                         sort_mode=sort_mode)
    r = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    r.request_all()
    r.update_residency()
    img = r.render([cam])[0].cpu().numpy()
    st = r.stats()
    assert st["status"] == 0 and st["missing"] == 0 and st["drawn_pages"] == sc.n_pages
    return r, img, st


# the last two sort (key, splat) pairs instead of keys with the splat packed in
CAMS = [
    ("tiny_16x16", dict(), False),
    ("tiny_8x8", dict(tile=(8, 8)), False),
    ("tiny_32x8", dict(tile=(32, 8)), False),
    ("ragged_250x131", dict(width=250, height=131), False),
    ("tiny_16x16_pairs", dict(), True),
    ("ragged_250x131_8x8_pairs", dict(width=250, height=131, tile=(8, 8)), True),
]


@pytest.mark.parametrize("name,kw,sep", CAMS)
def test_full_scene_render_parity(v, name, kw, sep):
    raw, sc = tiny_scene()
    cam = scenegen.tiny_camera(**kw)
    r, img, st = _full_render(v, raw, sc, cam, separate_values=sep)
    g, vid = oracle.full_scene(sc)
    ref = oracle.render(g, vid, cam)
    pr = ref["proj"]
    N = len(vid)
    assert st["drawn_gaussians"] == N
    rect = r.debug(v.DBG_SPLAT_RECT, np.int32).reshape(N, 4)
    depth = r.debug(v.DBG_SPLAT_DEPTH, np.float32)
    rad = r.debug(v.DBG_SPLAT_RADIUS, np.float32)
    vis = pr["vis"] != 0
    np.testing.assert_array_equal(rect[vis], pr["rect"][vis])
    np.testing.assert_array_equal(rect[~vis], 0)
    np.testing.assert_array_equal(depth.view(np.uint32), np.where(vis, pr["depth"], 0).view(np.uint32))
    np.testing.assert_array_equal(rad, np.where(vis, pr["radius"], 0))
    tmask = r.debug(v.DBG_SPLAT_TMASK, np.uint64)
    np.testing.assert_array_equal(tmask, expected_tmask(pr, cam))
    np.testing.assert_array_equal(r.debug(v.DBG_SPLAT_TOUCHED, np.uint32), np.where(vis, pr["touched"], 0))
    keys = r.debug(v.DBG_KEYS, np.uint64)
    vals = r.debug(v.DBG_VALUES, np.uint32)
    assert st["pairs"] == len(ref["keys"])
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(vals.astype(np.int64), ref["idx"])
    rng = r.debug(v.DBG_RANGES, np.uint32).reshape(-1, 2)
    np.testing.assert_array_equal(rng.astype(np.int64), ref["ranges"])
    xy = r.debug(v.DBG_SPLAT_XY, np.float32).reshape(N, 2)
    co = r.debug(v.DBG_SPLAT_CONIC, np.float32).reshape(N, 4)
    rgb = r.debug(v.DBG_SPLAT_RGB, np.float32).reshape(N, 3)
    np.testing.assert_allclose(xy[vis], pr["centre"][vis], rtol=1e-6, atol=1e-4)
    np.testing.assert_allclose(co[vis, :3], pr["conic"][vis], rtol=2e-5, atol=1e-6)
    np.testing.assert_allclose(rgb[vis], pr["rgb"][vis], rtol=1e-5, atol=1e-6)
    e0, nflag = compare_image(img, ref)
    assert nflag < 0.005 * cam.width * cam.height


def test_crowded_tiles(v):
    """The whole tiny scene seen from afar in a 40x40 view: a few tiles hold
    thousands of pairs each (one over 4096); keys, values, ranges and the
    image still equal the oracle's."""
    raw, sc = tiny_scene()
    cam = scenegen.look_at((0.0, 0.0, -70.0), (0, 0, 0), (0, -1, 0), 40, 40, 12.0, (16, 16))
    r, img, st = _full_render(v, raw, sc, cam)
    g, vid = oracle.full_scene(sc)
    ref = oracle.render(g, vid, cam)
    rng = ref["ranges"]
    assert (rng[:, 1] - rng[:, 0]).max() > 4096
    np.testing.assert_array_equal(r.debug(v.DBG_KEYS, np.uint64), ref["keys"])
    np.testing.assert_array_equal(r.debug(v.DBG_VALUES, np.uint32).astype(np.int64), ref["idx"])
    np.testing.assert_array_equal(r.debug(v.DBG_RANGES, np.uint32).reshape(-1, 2).astype(np.int64), rng)
    compare_image(img, ref)


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (32, 8)])
def test_large_splat_binning(v, tile):
    """Gaussians close to a ragged 250x131 view, half of them stretched along
    one axis: many rectangles hold more than 64 tiles, some with at most 32
    kept tiles (their rows walked by the whole warp in the first emission
    kernel) and some with more (cut into pieces of 256 pairs whose rows a
    warp walks).  Tile counts, keys, values and
    ranges equal the oracle's bit for bit; the image is within tolerance."""
    raw = scenegen.uniform_scene(n=6000, seed=41, lo=-1.6, hi=1.6, ls_mu=-3.2, ls_sd=0.6, sh_degree=1)
    raw.log_scale[::2, 0] += np.float32(2.0)
    raw.log_scale[::61] += np.float32(2.0)
    from oracle import build as ob
    bp = ob.BuildParams(page_size=256, paging="morton", lo=(-2, -2, -2), hi=(2, 2, 2), voxel=0.25, kappa=0.5,
                        link_samples=0)
    sc = ob.build_scene(raw, bp)
    cam = scenegen.look_at((0.3, -0.2, -2.6), (0, 0, 0), (0, -1, 0), 250, 131, 70.0, tile)
    r, img, st = _full_render(v, raw, sc, cam)
    g, vid = oracle.full_scene(sc)
    ref = oracle.render(g, vid, cam)
    pr = ref["proj"]
    vis = pr["vis"] != 0
    rc = pr["rect"]
    area = (rc[:, 2] - rc[:, 0]) * (rc[:, 3] - rc[:, 1])
    wide = vis & (area > 64)
    assert (wide & (pr["touched"] <= 32)).sum() > 20 and (wide & (pr["touched"] > 32)).sum() > 20
    assert (wide & (pr["touched"] > 100)).sum() >= 3
    np.testing.assert_array_equal(r.debug(v.DBG_SPLAT_TOUCHED, np.uint32), np.where(vis, pr["touched"], 0))
    np.testing.assert_array_equal(r.debug(v.DBG_KEYS, np.uint64), ref["keys"])
    np.testing.assert_array_equal(r.debug(v.DBG_VALUES, np.uint32).astype(np.int64), ref["idx"])
    np.testing.assert_array_equal(r.debug(v.DBG_RANGES, np.uint32).reshape(-1, 2).astype(np.int64), ref["ranges"])
    compare_image(img, ref)


@pytest.mark.parametrize("sep", [False, True])
@pytest.mark.parametrize("cam_kw", [dict(), dict(width=250, height=131, tile=(8, 8)), dict(width=24, height=16)])
def test_sort_modes_agree(v, sep, cam_kw):
    """The cooperative sort (all passes in one launch) and the onesweep sort
    (a launch per pass) give the same sorted pairs, tile ranges and image,
    bit for bit; the 24x16 view has fewer pairs than the cooperative grid has
    CTAs (most chunks empty)."""
    raw, sc = tiny_scene()
    cam = scenegen.tiny_camera(**cam_kw)
    out = []
    for mode in (0, 1):
        r, img, st = _full_render(v, raw, sc, cam, separate_values=sep, sort_mode=mode)
        out.append((img, r.debug(v.DBG_KEYS, np.uint64), r.debug(v.DBG_VALUES, np.uint32),
                    r.debug(v.DBG_RANGES, np.uint32), st["pairs"]))
    assert out[0][4] == out[1][4] > 0
    for a, b in zip(out[0][:4], out[1][:4]):
        assert np.array_equal(a, b)


def test_empty_and_degenerate_views(v):
    """A camera looking away from the scene draws nothing: zero pairs, background image."""
    raw, sc = tiny_scene()
    cam = scenegen.look_at((0, 0, -15), (0, 0, -30), (0, -1, 0), 64, 48, 60.0)
    r, img, st = _full_render(v, raw, sc, cam)
    assert st["pairs"] == 0
    assert np.all(img == 0)


def test_render_is_deterministic(v):
    raw, sc = tiny_scene()
    cam = scenegen.tiny_camera(width=200, height=120)
    _, a, _ = _full_render(v, raw, sc, cam)
    _, b, _ = _full_render(v, raw, sc, cam)
    assert np.array_equal(a, b)


def test_fp16_pool_parity_and_psnr(v):
    """fp16 pool: discrete results equal the oracle run on the fp16-rounded
    attributes; the image stays within 45 dB PSNR of the FP64 fp32-scene render."""
    raw = scenegen.blob_scene(n=20000, n_blobs=20, lo=-4.0, hi=4.0, blob_sigma=0.4, seed=31)
    from oracle import build as ob
    bp = ob.BuildParams(page_size=512, paging="octree", lo=(-8, -8, -8), hi=(8, 8, 8), voxel=0.5, kappa=1.0,
                        link_samples=0)
    sc = ob.build_scene(raw, bp)
    cam = scenegen.look_at((0, -14, 3), (0, 0, 0), (0, 0, 1), 256, 192, 60.0)
    r, img, st = _full_render(v, raw, sc, cam, fp16=True)
    g, vid = oracle.full_scene(sc)
    g16 = dict(g)
    for k in ("scale", "rot", "sh"):
        g16[k] = g[k].astype(np.float16).astype(np.float32)
    ref16 = oracle.render(g16, vid, cam)
    N = len(vid)
    rect = r.debug(v.DBG_SPLAT_RECT, np.int32).reshape(N, 4)
    vis = ref16["proj"]["vis"] != 0
    np.testing.assert_array_equal(rect[vis], ref16["proj"]["rect"][vis])
    np.testing.assert_array_equal(r.debug(v.DBG_KEYS, np.uint64), ref16["keys"])
    compare_image(img, ref16)
    ref32 = oracle.render(g, vid, cam)
    mse = np.mean((np.clip(img, 0, 1) - np.clip(ref32["image"], 0, 1)) ** 2)
    psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
    assert psnr >= 45.0, psnr


def test_vq_pool_parity(v):
    """Compressed pages (VQ records, a 128-code SH codebook) through the
    TMA-staged projection: discrete results equal the oracle run on the
    attributes the records decode to, the image within the FP32 tolerance;
    the PSNR against the FP64 render of the fp32 scene is reported."""
    import dataclasses
    from oracle import build as ob
    raw = scenegen.blob_scene(n=20000, n_blobs=20, lo=-4.0, hi=4.0, blob_sigma=0.4, seed=31)
    bp = ob.BuildParams(page_size=512, paging="octree", lo=(-8, -8, -8), hi=(8, 8, 8), voxel=0.5, kappa=1.0,
                        link_samples=0)
    sc = ob.build_scene(raw, bp)
    cam = scenegen.look_at((0, -14, 3), (0, 0, 0), (0, 0, 1), 256, 192, 60.0)
    r, img, st = _full_render(v, raw, sc, cam, vq_codes=128)
    assert st["staged_projection"] == 1
    cb, codes = ob.quantize_sh(sc.levels, 128, 8)
    gq, vid = oracle.full_scene(dataclasses.replace(sc, levels=ob.vq_levels(sc.levels, cb, codes)))
    refq = oracle.render(gq, vid, cam)
    N = len(vid)
    rect = r.debug(v.DBG_SPLAT_RECT, np.int32).reshape(N, 4)
    vis = refq["proj"]["vis"] != 0
    np.testing.assert_array_equal(rect[vis], refq["proj"]["rect"][vis])
    np.testing.assert_array_equal(r.debug(v.DBG_KEYS, np.uint64), refq["keys"])
    np.testing.assert_allclose(r.debug(v.DBG_SPLAT_RGB, np.float32).reshape(N, 3)[vis], refq["proj"]["rgb"][vis],
                               rtol=2e-5, atol=2e-6)
    compare_image(img, refq)
    g, _ = oracle.full_scene(sc)
    ref32 = oracle.render(g, vid, cam)
    mse = np.mean((np.clip(img, 0, 1) - np.clip(ref32["image"], 0, 1)) ** 2)
    print("VQ pool PSNR against the FP64 fp32-scene render: %.2f dB" % (10 * np.log10(1.0 / max(mse, 1e-30))))
