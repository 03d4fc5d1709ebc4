"""GPU parity of the virtual-memory frame (page determination, page table,
streaming, LOD) against the oracle over camera trajectories, bit-exact:
visibility buffer, request words and list, page-table state, copy, draw and
missing lists, controller state; the pool holds exactly the host pages the
table says; images within the FP32 tolerance."""
import numpy as np
import pytest

import oracle
import scenegen
from _common import city_cam, city_scene, compare_image, import_scene, round16_scene, tiny_scene
from oracle import residency as rs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_19415_b300 as mod
    return mod


def _run_trajectory(v, raw, sc, cams, pool_slots, budget_pages, lod=True, links=True, tau0=1.0, check_images=(),
                    fp16=False, vq_codes=0, fade=0, step0=0.1):
    """vq_codes > 0: the pool holds VQ records (compressed pages) with an SH
    codebook of that many codes; images are compared with the oracle run on
    the attributes those records decode to.  fade > 0: LOD cross-fade of
    that many frames (draw weights compared too)."""
    scene = import_scene(v, raw, sc, fp16=fp16)
    W, H = cams[0].width, cams[0].height
    fmt = int(fp16)
    rec = scene.info.record_bytes16 if fp16 else scene.info.record_bytes
    if vq_codes:
        import dataclasses
        from oracle import build as ob
        scene.quantize_sh(vq_codes, 6)
        cb, codes = ob.quantize_sh(sc.levels, vq_codes, 6)
        np.testing.assert_array_equal(scene.codebook(), cb)
        fmt, rec = v.POOL_VQ, scene.info.record_bytes_vq
    budget = budget_pages * sc.params.page_size * rec
    cfg = v.RenderConfig(max_width=W, max_height=H, lod=lod, links=links, staging_bytes=budget, tau0=tau0,
                         fp16_pool=fmt, lod_fade_frames=fade, step0=step0)
    r = v.Renderer(scene, cfg, pool_slots=pool_slots)
    rp = rs.ResidencyParams(n_entries=pool_slots, page_size=sc.params.page_size, levels=len(sc.levels),
                            fanout=sc.params.lod_fanout, record_bytes=rec, budget_bytes=budget, lod=lod, tau0=tau0,
                            fade_frames=fade, step0=step0)
    pt = rs.PageTable(rp)
    smax = sc.params.lod_fanout ** (len(sc.levels) - 1)
    host_pages = [scene.pages(l, fp16=fp16) for l in range(len(sc.levels))]
    # images of an fp16 or VQ pool are compared with the oracle on the attributes it stores
    osc = round16_scene(sc) if fp16 else sc
    faded = []
    if vq_codes:
        host_pages = [scene.export(v.SCENE_PAGES_VQ, l).reshape(sc.n_pages, -1) for l in range(len(sc.levels))]
        osc = dataclasses.replace(sc, levels=ob.vq_levels(sc.levels, cb, codes))
    for f, cam in enumerate(cams):
        r.render_feedback([cam])
        r.update_residency()
        img = r.render([cam])[0].cpu().numpy()
        ref = oracle.frame(osc, pt, cam, ds=4, links=links, render_image=f in check_images)
        st = r.stats()
        assert st["status"] == 0
        # page determination
        np.testing.assert_array_equal(r.debug(v.DBG_FEEDBACK, np.uint64).reshape(ref["buf"].shape), ref["buf"])
        np.testing.assert_array_equal(r.debug(v.DBG_REQ, np.uint32), ref["req"])
        np.testing.assert_array_equal(r.debug(v.DBG_DIRECT, np.uint8), ref["direct"])
        reqs = r.debug(v.DBG_REQUESTS, np.int32).reshape(-1, 4)
        np.testing.assert_array_equal(reqs[:, 0], ref["pages"])
        np.testing.assert_array_equal(reqs[:, 1].view(np.uint32), ref["enc"])
        np.testing.assert_array_equal(reqs[:, 2], ref["direct"][ref["pages"]])
        np.testing.assert_array_equal(reqs[:, 3], ref["levels"])
        # page table
        up = ref["update"]
        np.testing.assert_array_equal(r.debug(v.DBG_PT_LOD, np.int32), pt.lod)
        np.testing.assert_array_equal(r.debug(v.DBG_PT_LAST, np.int32), pt.last_used)
        np.testing.assert_array_equal(r.debug(v.DBG_PT_SLOT, np.int32).reshape(pool_slots, smax), pt.slot)
        np.testing.assert_array_equal(r.debug(v.DBG_COPIES, np.int32).reshape(-1, 4),
                                      np.array(up["copies"], np.int32).reshape(-1, 4))
        draw = r.debug(v.DBG_DRAW, np.int32).reshape(-1, 4)
        np.testing.assert_array_equal(draw, np.array(up["draw"], np.int32).reshape(-1, 4))
        np.testing.assert_array_equal(r.debug(v.DBG_DRAW_W, np.float32), np.array(up["draw_w"], np.float32))
        assert st["fading"] == up["fading"]
        faded.append(up["fading"])
        np.testing.assert_array_equal(r.debug(v.DBG_MISSING, np.int32), np.array(up["missing"], np.int32))
        assert st["usage"] == np.float32(up["usage"])
        assert st["tau"] == np.float32(pt.tau)
        assert st["streamed_bytes"] == up["streamed_bytes"]
        # the pool holds the host bytes of every drawn page
        pool = r.debug(v.DBG_POOL, np.uint8).reshape(pool_slots, -1)
        for (p, l, e, s) in draw:
            blk = host_pages[l][p]
            np.testing.assert_array_equal(pool[e, s * len(blk):(s + 1) * len(blk)], blk)
        if f in check_images:
            compare_image(img, ref["render"])
    r.faded = faded
    return r


def test_tiny_scene_feedback_frames(v):
    raw, sc = tiny_scene()
    cams = [scenegen.look_at((12 * np.cos(a), 3.0, 12 * np.sin(a)), (0, 0, 0), (0, -1, 0), 128, 96, 60.0)
            for a in np.linspace(0, 1.5, 8)]
    _run_trajectory(v, raw, sc, cams, pool_slots=20, budget_pages=6, lod=False, check_images=(0, 7))


@pytest.mark.parametrize("links", [True, False])
def test_city_lod_trajectory(v, links):
    raw, sc = city_scene()
    cams = [city_cam(160.0, k) for k in range(14)]
    _run_trajectory(v, raw, sc, cams, pool_slots=8, budget_pages=5, lod=True, links=links, tau0=2.0,
                    check_images=(0, 13))


def test_city_lod_trajectory_fp16(v):
    raw, sc = city_scene(levels=3, fanout=8, page_size=512)
    cams = [city_cam(160.0, k, width=200, height=120) for k in range(6)]
    _run_trajectory(v, raw, sc, cams, pool_slots=5, budget_pages=3, lod=True, tau0=1.0, fp16=True)


@pytest.mark.parametrize("fp16", [False, True])
def test_city_lod_trajectory_staged_projection(v, fp16):
    """Level blocks of 1024, 256 and 64 Gaussians: the projection stages the
    records with tensor-map tile loads of 64 Gaussians (fp32 and fp16 pools);
    scenes with a block of 8 gather them with plain loads."""
    raw, sc = city_scene(levels=3, fanout=4, page_size=1024)
    cams = [city_cam(160.0, k, width=200, height=120) for k in range(6)]
    r = _run_trajectory(v, raw, sc, cams, pool_slots=6, budget_pages=3, lod=True, tau0=1.0, fp16=fp16,
                        check_images=(0, 3, 5))
    assert r.stats()["staged_projection"] == 1


def test_halving_lod_four_levels(v):
    """The paper's own LOD shape: four levels, each halving the page (blocks
    of 256, 128, 64 and 32 Gaussians: staged in tile loads of 32)."""
    raw, sc = city_scene(levels=4, fanout=2, page_size=256, n=30000)
    cams = [city_cam(160.0, k, width=160, height=96) for k in range(8)]
    r = _run_trajectory(v, raw, sc, cams, pool_slots=10, budget_pages=4, lod=True, tau0=4.0, check_images=(0, 7))
    assert r.stats()["staged_projection"] == 1


def test_gather_projection_for_blocks_of_eight(v):
    """Level blocks of 512, 64 and 8 Gaussians: no tile width divides them
    all, so the projection gathers with plain loads."""
    raw, sc = city_scene(levels=3, fanout=8, page_size=512)
    cams = [city_cam(160.0, k, width=160, height=96) for k in range(4)]
    r = _run_trajectory(v, raw, sc, cams, pool_slots=8, budget_pages=4, lod=True, tau0=2.0, check_images=(3,))
    assert r.stats()["staged_projection"] == 0


@pytest.mark.parametrize("fp16", [False, True])
def test_kmeans_lod_trajectory(v, fp16):
    """The paper's k-means LOD (four levels, halving per level): LOD choice,
    residency, streaming and images along a trajectory equal the oracle's
    on the k-means levels."""
    raw, sc = city_scene(levels=4, fanout=2, page_size=256, n=30000, lod_method="kmeans")
    cams = [city_cam(160.0, k, width=160, height=96) for k in range(8)]
    _run_trajectory(v, raw, sc, cams, pool_slots=10, budget_pages=4, lod=True, tau0=4.0, fp16=fp16,
                    check_images=(0, 7))


def test_fully_resident_vm_render_equals_full_scene(v):
    """Pool holding the whole scene, LOD off: after feedback-driven streaming
    frames (pages land in arbitrary slots), requesting every page renders the
    same bits as a renderer that loaded the scene in page order."""
    raw, sc = tiny_scene()
    scene = import_scene(v, raw, sc)
    cam = scenegen.tiny_camera(width=192, height=160)
    cfg = v.RenderConfig(max_width=192, max_height=160, lod=False, staging_bytes=1 << 40)
    a = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    walk = [scenegen.look_at((12 * np.cos(t), -4.0, 12 * np.sin(t)), (0, 0, 0), (0, -1, 0), 192, 160, 60.0)
            for t in np.linspace(0.3, 5.0, 10)]
    for c in walk:
        a.render_feedback([c])
        a.update_residency()
        a.render([c])
    a.request_all()
    a.update_residency()
    img_a = a.render([cam])[0].cpu().numpy()
    b = v.Renderer(scene, cfg, pool_slots=sc.n_pages)
    b.request_all()
    b.update_residency()
    img_b = b.render([cam])[0].cpu().numpy()
    assert a.stats()["missing"] == 0
    assert np.array_equal(img_a, img_b)
    g, vid = oracle.full_scene(sc)
    compare_image(img_a, oracle.render(g, vid, cam))


def test_zero_budget_streams_nothing(v):
    raw, sc = tiny_scene()
    scene = import_scene(v, raw, sc)
    cfg = v.RenderConfig(max_width=128, max_height=96, lod=False, staging_bytes=0)
    r = v.Renderer(scene, cfg, pool_slots=4)
    cam = scenegen.tiny_camera(width=128, height=96)
    r.render_feedback([cam])
    r.update_residency()
    img = r.render([cam])[0].cpu().numpy()
    st = r.stats()
    assert st["streamed_pages"] == 0 and st["drawn_pages"] == 0 and st["missing"] == st["requested"] > 0
    assert np.all(img == 0)


@pytest.mark.parametrize("fp16,mode", [(False, "feedback"), (True, "feedback"), (False, "front"), (True, "front"),
                                       (False, "two_renders"), (True, "two_renders"), (False, "split"),
                                       (True, "split")])
def test_feedback_on_own_stream_matches_one_stream(v, fp16, mode):
    """Page determination of frame t+1 on its own stream (front: with its
    page-table update; two_renders: and consecutive renders on two streams,
    i.e. the two render contexts in flight; split: as two_renders with page
    determination and update on separate streams, so that page determination
    runs a frame ahead on the double-buffered request words), copies on
    another stream, no host sync between frames: every image, the final page
    table, the last render's sorted pairs and the running sums equal the
    single-stream run bit for bit."""
    import torch
    raw, sc = city_scene(levels=3, fanout=4, page_size=1024)
    scene = import_scene(v, raw, sc, fp16=fp16)
    cams = [city_cam(160.0, k, width=200, height=120) for k in range(10)]
    rec = scene.info.record_bytes16 if fp16 else scene.info.record_bytes
    cfg = v.RenderConfig(max_width=200, max_height=120, lod=True, staging_bytes=3 * sc.params.page_size * rec,
                         tau0=1.0, fp16_pool=fp16)
    a = v.Renderer(scene, cfg, pool_slots=6)
    ref = []
    for c in cams:
        a.render_feedback([c])
        a.update_residency()
        ref.append(a.render([c])[0].cpu().numpy())
    b = v.Renderer(scene, cfg, pool_slots=6)
    st, fst, cst, st2, ust = (torch.cuda.Stream() for _ in range(5))
    imgs = [torch.empty((3, 120, 200), dtype=torch.float32, device="cuda") for _ in cams]
    for f, (c, im) in enumerate(zip(cams, imgs)):
        b.render_feedback([c], fst)
        b.update_residency({"feedback": st, "split": ust}.get(mode, fst), cst)
        b.render([c], [im], st2 if mode in ("two_renders", "split") and f % 2 else st)
    torch.cuda.synchronize()
    for f, im in enumerate(imgs):
        assert np.array_equal(im.cpu().numpy(), ref[f]), f"frame {f}"
    for what, dt in ((v.DBG_PT_LOD, np.int32), (v.DBG_PT_LAST, np.int32), (v.DBG_PT_SLOT, np.int32),
                     (v.DBG_REQ, np.uint32), (v.DBG_FEEDBACK, np.uint64), (v.DBG_KEYS, np.uint64),
                     (v.DBG_VALUES, np.uint32), (v.DBG_RANGES, np.uint32), (v.DBG_SPLAT_DEPTH, np.uint32)):
        assert np.array_equal(a.debug(what, dt), b.debug(what, dt, st))
    sa, sb = a.stats(), b.stats(st)
    for k in ("acc_frames", "acc_views", "acc_pairs", "acc_drawn_gaussians", "acc_streamed_bytes", "acc_missing",
              "acc_requested", "pairs", "drawn_gaussians"):
        assert sa[k] == sb[k], k
    assert sb["status"] == 0


def test_city_lod_trajectory_vq(v):
    """Compressed pages: VQ records (40 bytes) in the pool with a 64-code SH
    codebook, three LOD levels of pages of 512 with fanout 8 (level blocks of
    8: the gathering projection), page table and images against the oracle."""
    raw, sc = city_scene()
    cams = [city_cam(160.0, k) for k in range(10)]
    _run_trajectory(v, raw, sc, cams, pool_slots=8, budget_pages=5, lod=True, tau0=2.0, check_images=(0, 5, 9),
                    vq_codes=64)


@pytest.mark.parametrize("fp16", [False, True])
def test_city_lod_trajectory_fade(v, fp16):
    """LOD cross-fade of 4 frames along a walk whose pages change level: page
    table, the draw list with both levels of fading pages and its weights,
    and images (opacities scaled by the weights) against the oracle; fp16
    pools go through the TMA-staged projection (pages of 512, fanout 4)."""
    if fp16:
        raw, sc = city_scene(levels=3, fanout=4, page_size=512)
    else:
        raw, sc = city_scene()
    # a dolly towards the city while the controller lowers tau (a large
    # initial tau and step): many pages move to finer levels
    cams = [scenegen.look_at((80, -260 + 15 * k, 40 - 2 * k), (80, 80, 0), (0, 0, 1), 200, 120, 60.0, (16, 16))
            for k in range(16)]
    r = _run_trajectory(v, raw, sc, cams, pool_slots=24, budget_pages=12, lod=True, tau0=10.0, step0=1.5,
                        check_images=(2, 5, 9, 14), fp16=fp16, fade=4)
    assert sum(r.faded) > 20
