"""A scene opened from a file (Sec. 3.5 memory-mapped Gaussians; pages pass
through a page-locked staging buffer the host fills, Sec. 4.1 "Transfer")
renders exactly what the same scene held in memory renders: page tables,
copy lists, pool bytes, counters and images bit for bit along a trajectory
that streams pages every frame."""
import numpy as np
import pytest

import scenegen
from _common import city_cam

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2506_19415_b300 as v
    return v


@pytest.mark.parametrize("fp16", [False, True])
def test_mapped_scene_frames_equal_in_memory(v, tmp_path, fp16):
    import torch
    raw = scenegen.city_scene(n=60000, n_boxes=20, extent=160.0)
    sc = v.vm3dgs_build_pages(raw, v.BuildConfig(page_size=512, paging="octree", lod_levels=3, lod_fanout=8,
                                                   lo=(-4, -4, -4), hi=(164, 164, 84), voxel=4.0, kappa=0.5,
                                                   link_samples=4, fp16=True))
    path = tmp_path / "city.vm3dgs"
    sc.save(path)
    op = v.vm3dgs_scene_open(path)
    rec = sc.info.record_bytes16 if fp16 else sc.info.record_bytes
    cams = [city_cam(160.0, k, width=200, height=120) for k in range(12)]
    cfg = v.RenderConfig(max_width=200, max_height=120, lod=True, links=True, staging_bytes=3 * 512 * rec, tau0=1.0,
                         fp16_pool=fp16)
    ra, rb = v.Renderer(sc, cfg, pool_slots=8), v.Renderer(op, cfg, pool_slots=8)
    copy_stream = torch.cuda.Stream()
    host = [sc.pages(l, fp16=fp16) for l in range(3)]
    streamed = 0
    for cam in cams:
        ra.render_feedback([cam])
        ra.update_residency()
        rb.render_feedback([cam])
        rb.update_residency(None, copy_stream)   # a file-backed renderer streams on the update's stream
        ia, ib = ra.render([cam])[0], rb.render([cam])[0]
        torch.cuda.synchronize()
        assert torch.equal(ia, ib)
        sa, sb = ra.stats(), rb.stats()
        assert sa["status"] == 0 and sa == sb
        streamed += sb["streamed_pages"]
        for what, dt in ((v.DBG_COPIES, np.int32), (v.DBG_DRAW, np.int32), (v.DBG_PT_SLOT, np.int32),
                         (v.DBG_PT_LOD, np.int32)):
            np.testing.assert_array_equal(ra.debug(what, dt), rb.debug(what, dt))
        # every drawn sub-slot holds the scene's bytes in both pools (the rest
        # of a pool is whatever its memory held before)
        pa = ra.debug(v.DBG_POOL, np.uint8).reshape(8, -1)
        pb = rb.debug(v.DBG_POOL, np.uint8).reshape(8, -1)
        for (p, l, e, s_) in ra.debug(v.DBG_DRAW, np.int32).reshape(-1, 4):
            blk = host[l][p]
            np.testing.assert_array_equal(pa[e, s_ * len(blk):(s_ + 1) * len(blk)], blk)
            np.testing.assert_array_equal(pb[e, s_ * len(blk):(s_ + 1) * len(blk)], blk)
    assert streamed > 8   # pages were replaced, not only loaded once


def test_prefetch_refused_on_a_file_backed_renderer(v, tmp_path):
    """The prefetcher pulls pages from page-locked scene memory, which a
    scene opened from a file does not have: the call returns E_STATE."""
    raw = scenegen.city_scene(n=20000, n_boxes=8, extent=100.0)
    sc = v.vm3dgs_build_pages(raw, v.BuildConfig(page_size=512, paging="octree", lod_levels=1, lo=(-4, -4, -4),
                                                   hi=(104, 104, 84), voxel=4.0, kappa=0.5, link_samples=2))
    path = tmp_path / "city.vm3dgs"
    sc.save(path)
    op = v.vm3dgs_scene_open(path)
    cam = city_cam(100.0, 0, width=160, height=96)
    r = v.Renderer(op, v.RenderConfig(max_width=160, max_height=96, staging_bytes=4 * 512 * sc.info.record_bytes),
                   pool_slots=8)
    r.render_feedback([cam])
    r.update_residency()
    O = 256
    p = v.Prefetcher(v.MlpShape(n_in=12 + O // 16, n_hidden=64, n_out=O, max_batch=8, seed=1, lr=0.0))
    with pytest.raises(v.Vm3dgsError) as e:
        v.vm3dgs_prefetch(r, p, cam, cam, 0.0)
    assert e.value.code == v.E_STATE
