"""Full-size parity: the headline's frame layout against the oracle.

A 1M-Gaussian city (500 m x 500 m, 300 boxes, SH3) in octree pages of 4096
with 3 LOD levels (fanout 8) and a 2 GiB fp16 pool (4096 slots): at 1920x1080
with 16x16 tiles (8160 tiles) the packed sort key has the headline's layout,
13 tile + 27 depth + 24 index bits, sorted in 5 passes of its 40 tile and
depth bits.  Along three street-level frames, bit-exact against the oracle run
on the fp16-rounded attributes: the visibility buffer, the request list with
its levels, the page table, the copy and draw lists, the controller's tau, the
splat tile counts, the sorted keys and values and the tile ranges; each image
within the FP32 tolerance of the oracle's; and each image's PSNR against the
oracle's FP64 render of the fp32 attributes of the same pages at least 45 dB
(the quality gate of the fp16 pool)."""
import os

import numpy as np
import pytest

import oracle
from _common import city_cam, city_scene, compare_image, import_scene, round16_scene
from oracle import residency as rs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_19415_b300 as mod
    return mod


def test_fullsize_city_frames(v):
    raw, sc = city_scene(n=1_000_000, n_boxes=300, extent=500.0, levels=3, fanout=8, page_size=4096)
    scene = import_scene(v, raw, sc, fp16=True)
    P = 4096
    rec = scene.info.record_bytes16
    budget = 64 * 4096 * rec
    cams = [city_cam(500.0, k, width=1920, height=1080) for k in range(3)]
    cfg = v.RenderConfig(max_width=1920, max_height=1080, lod=True, staging_bytes=budget, tau0=1.0, fp16_pool=True)
    r = v.Renderer(scene, cfg, pool_slots=P)
    pt = rs.PageTable(rs.ResidencyParams(n_entries=P, page_size=4096, levels=3, fanout=8, record_bytes=rec,
                                         budget_bytes=budget, lod=True, tau0=1.0))
    sc16 = round16_scene(sc)
    oracle.set_threads(os.cpu_count() or 1)
    try:
        for f, cam in enumerate(cams):
            r.render_feedback([cam])
            r.update_residency()
            img = r.render([cam])[0].cpu().numpy()
            st = r.stats()
            assert st["status"] == 0
            assert (st["key_tile_bits"], st["key_depth_bits"], st["key_index_bits"], st["key_packed"]) == (13, 27, 24, 1)
            ref = oracle.frame(sc16, pt, cam, ds=4)
            np.testing.assert_array_equal(r.debug(v.DBG_FEEDBACK, np.uint64).reshape(ref["buf"].shape), ref["buf"])
            reqs = r.debug(v.DBG_REQUESTS, np.int32).reshape(-1, 4)
            np.testing.assert_array_equal(reqs[:, 0], ref["pages"])
            np.testing.assert_array_equal(reqs[:, 3], ref["levels"])
            up = ref["update"]
            np.testing.assert_array_equal(r.debug(v.DBG_PT_LOD, np.int32), pt.lod)
            np.testing.assert_array_equal(r.debug(v.DBG_PT_SLOT, np.int32).reshape(P, 64), pt.slot)
            np.testing.assert_array_equal(r.debug(v.DBG_COPIES, np.int32).reshape(-1, 4),
                                          np.array(up["copies"], np.int32).reshape(-1, 4))
            np.testing.assert_array_equal(r.debug(v.DBG_DRAW, np.int32).reshape(-1, 4),
                                          np.array(up["draw"], np.int32).reshape(-1, 4))
            assert st["tau"] == np.float32(pt.tau) and st["missing"] == len(up["missing"])
            ren = ref["render"]
            pr = ren["proj"]
            np.testing.assert_array_equal(r.debug(v.DBG_SPLAT_TOUCHED, np.uint32),
                                          np.where(pr["vis"] != 0, pr["touched"], 0))
            assert st["pairs"] == len(ren["keys"]) > 1_000_000
            np.testing.assert_array_equal(r.debug(v.DBG_KEYS, np.uint64), ren["keys"])
            np.testing.assert_array_equal(r.debug(v.DBG_VALUES, np.uint32).astype(np.int64), ren["idx"])
            np.testing.assert_array_equal(r.debug(v.DBG_RANGES, np.uint32).reshape(-1, 2).astype(np.int64),
                                          ren["ranges"])
            e0, nflag = compare_image(img, ren)
            # each 1080p pixel of the dense city evaluates dozens of splats, so
            # more pixels see an alpha within rounding of 1/255 than in the
            # small views (1.2% measured); they are held to the derived bound
            assert nflag < 0.03 * 1920 * 1080
            # the quality gate: the fp32 attributes of the same pages, FP64 render
            g32, vid = oracle.gather_draw(sc, up["draw"])
            ref32 = oracle.render(g32, vid, cam)
            mse = np.mean((np.clip(img, 0, 1) - np.clip(ref32["image"], 0, 1)) ** 2)
            psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
            assert psnr >= 45.0, (f, psnr)
            print("frame %d: %d pairs, %d pages drawn, max err %.2e, %d flagged, PSNR %.1f dB" %
                  (f, st["pairs"], len(up["draw"]), e0, nflag, psnr))
    finally:
        oracle.set_threads(1)
