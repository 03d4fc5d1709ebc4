"""The library's SH codebook (vm3dgs_scene_quantize_sh, host C++) against the
oracle's (oracle.build.quantize_sh) on the same pages: codebook and the code
of every Gaussian of every level bit for bit; the VQ records carry the fp32
position and opacity and the fp16 scale, rotation and SH band 0; argument and
state errors.  Host code only: no GPU."""
import numpy as np
import pytest

import scenegen
from _common import import_scene
from oracle import build as ob


@pytest.fixture(scope="module")
def v():
    import paper_2506_19415_b300 as mod
    return mod


def _scene(sh_degree=3, levels=3):
    raw = scenegen.city_scene(n=9000, n_boxes=4, extent=40.0)
    if sh_degree != 3:
        raw = scenegen.blob_scene(n=6000, n_blobs=5, lo=0.0, hi=10.0, blob_sigma=0.7, ls_mu=-2.0,
                                  sh_degree=sh_degree, seed=9)
        bp = ob.BuildParams(page_size=256, paging="octree", lod_levels=levels, lod_fanout=4, lo=(-2, -2, -2),
                            hi=(12, 12, 12), voxel=1.0, link_samples=2)
    else:
        bp = ob.BuildParams(page_size=256, paging="octree", lod_levels=levels, lod_fanout=4, lo=(-4, -4, -4),
                            hi=(44, 44, 84), voxel=3.0, link_samples=2)
    return raw, ob.build_scene(raw, bp)


@pytest.mark.parametrize("sh_degree,n_codes,iters,n_train", [(3, 64, 6, 100000), (3, 48, 20, 1500), (1, 16, 4, 3000),
                                                             (2, 33, 0, 500)])
def test_codebook_and_codes_equal_oracle(v, sh_degree, n_codes, iters, n_train):
    raw, sc = _scene(sh_degree)
    scene = import_scene(v, raw, sc)
    scene.quantize_sh(n_codes, iters, n_train)
    cb, codes = ob.quantize_sh(sc.levels, n_codes, iters, n_train)
    assert scene.info.n_codes == n_codes and scene.info.record_bytes_vq == 40
    np.testing.assert_array_equal(scene.codebook(), cb)
    for l, c in enumerate(codes):
        np.testing.assert_array_equal(scene.vq_codes(l), c, err_msg="level %d" % l)


def test_vq_record_fields(v):
    raw, sc = _scene()
    scene = import_scene(v, raw, sc)
    scene.quantize_sh(32, 4)
    for l, L in enumerate(sc.levels):
        m = sc.m(l)
        b = scene.export(v.SCENE_PAGES_VQ, l).reshape(sc.n_pages, -1)
        assert b.shape[1] == 40 * m
        f = b[:, :16 * m].copy().view(np.float32).reshape(sc.n_pages, 4, m)
        h = b[:, 16 * m:].copy().view(np.float16).reshape(sc.n_pages, 12, m)
        np.testing.assert_array_equal(f[:, 0:3].transpose(0, 2, 1), L["pos"])
        np.testing.assert_array_equal(f[:, 3], L["opacity"])
        np.testing.assert_array_equal(h[:, 0:3].transpose(0, 2, 1), L["scale"].astype(np.float16))
        np.testing.assert_array_equal(h[:, 3:7].transpose(0, 2, 1), L["rot"].astype(np.float16))
        np.testing.assert_array_equal(h[:, 7:10].transpose(0, 2, 1), L["sh"][:, :, 0, :].astype(np.float16))
        assert np.all(h[:, 11].view(np.uint16) == 0)


def test_errors(v):
    raw, sc = _scene()
    scene = import_scene(v, raw, sc)
    for bad in ((0, 4, 100), (70000, 4, 100), (8, -1, 100), (8, 4, 0), (10 ** 6 // 2, 4, 10 ** 6)):
        with pytest.raises(v.Vm3dgsError) as e:
            scene.quantize_sh(*bad)
        assert e.value.code == v.E_INVAL
    scene.quantize_sh(8, 2)
    with pytest.raises(v.Vm3dgsError) as e:
        scene.quantize_sh(8, 2)
    assert e.value.code == v.E_STATE
    # degree 0 has nothing to quantise; a pool of VQ records needs them
    raw0 = scenegen.uniform_scene(n=2048, seed=2)
    sc0 = ob.build_scene(raw0, ob.BuildParams(page_size=256, voxel=10 / 32, link_samples=2))
    s0 = import_scene(v, raw0, sc0)
    with pytest.raises(v.Vm3dgsError) as e:
        s0.quantize_sh(4)
    assert e.value.code == v.E_INVAL
    with pytest.raises(v.Vm3dgsError) as e:
        v.vm3dgs_pool_slot_bytes(s0, v.POOL_VQ)
    assert e.value.code == v.E_STATE
    assert v.vm3dgs_pool_slot_bytes(scene, v.POOL_VQ) == 40 * 256
