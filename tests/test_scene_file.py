"""Scene files (Sec. 3.5, "Scene Storage": Gaussians in a memory-mapped file
read by the OS on demand): a saved and reopened scene exports the same bytes
as the scene it was saved from; broken files are rejected.  CPU only."""
import numpy as np
import pytest

import paper_2506_19415_b300 as v
import scenegen


def _scene(fp16=True):
    raw = scenegen.city_scene(n=20000, n_boxes=8, extent=100.0)
    return v.vm3dgs_build_pages(raw, v.BuildConfig(page_size=512, paging="octree", lod_levels=3, lod_fanout=8,
                                                   lo=(-4, -4, -4), hi=(104, 104, 84), voxel=4.0, kappa=0.5,
                                                   link_samples=2, fp16=fp16))


@pytest.mark.parametrize("fp16", [True, False])
def test_save_open_roundtrip(tmp_path, fp16):
    sc = _scene(fp16)
    path = tmp_path / "city.vm3dgs"
    sc.save(path)
    op = v.vm3dgs_scene_open(path)
    for f, _ in v.SceneInfo._fields_:
        assert getattr(op.info, f) == getattr(sc.info, f), f
    for what in (v.SCENE_PAGE_COUNT, v.SCENE_PAGE_SRC, v.SCENE_ERR, v.SCENE_VERTS, v.SCENE_TRIS, v.SCENE_FACE_PAGE,
                 v.SCENE_LINK_PTR, v.SCENE_LINK_COL):
        np.testing.assert_array_equal(op.export(what), sc.export(what))
    for l in range(sc.info.lod_levels):
        np.testing.assert_array_equal(op.pages(l), sc.pages(l))
        if fp16:
            np.testing.assert_array_equal(op.pages(l, fp16=True), sc.pages(l, fp16=True))
    # page data sits at 4096-byte aligned offsets of the file
    assert path.stat().st_size >= sc.info.host_bytes


def test_bad_scene_files_rejected(tmp_path):
    with pytest.raises(v.Vm3dgsError):
        v.vm3dgs_scene_open(tmp_path / "missing.vm3dgs")
    sc = _scene()
    path = tmp_path / "city.vm3dgs"
    sc.save(path)
    data = path.read_bytes()
    cut = tmp_path / "cut.vm3dgs"
    cut.write_bytes(data[:len(data) // 2])
    with pytest.raises(v.Vm3dgsError):
        v.vm3dgs_scene_open(cut)
    bad = tmp_path / "magic.vm3dgs"
    bad.write_bytes(b"NOTSCENE" + data[8:])
    with pytest.raises(v.Vm3dgsError):
        v.vm3dgs_scene_open(bad)
    wrong = bytearray(data)
    wrong[8:12] = (0).to_bytes(4, "little")   # n_pages = 0
    (tmp_path / "fields.vm3dgs").write_bytes(bytes(wrong))
    with pytest.raises(v.Vm3dgsError):
        v.vm3dgs_scene_open(tmp_path / "fields.vm3dgs")


def test_quantize_after_open(tmp_path):
    """Compressed pages are not written to scene files: quantising an opened
    scene gives the codebook and VQ records of quantising the original."""
    sc = _scene()
    path = tmp_path / "city.vm3dgs"
    sc.save(path)
    op = v.vm3dgs_scene_open(path)
    sc.quantize_sh(24, 4, 4000)
    op.quantize_sh(24, 4, 4000)
    np.testing.assert_array_equal(op.codebook(), sc.codebook())
    for l in range(sc.info.lod_levels):
        np.testing.assert_array_equal(op.export(v.SCENE_PAGES_VQ, l), sc.export(v.SCENE_PAGES_VQ, l))
