"""The paper's mesh proxy on the GPU (paging "mesh": ellipsoid occupancy of
the scene slices, closing and the cube-by-cube surface in kernels; QEM and
page assignment on the host) against the oracle's build, bit for bit: page
assignment, level-0 records, the subdivided mesh, triangle pages and links;
LOD levels within the FP64 rounding of the other pagings; then frames of
page determination and residency over the mesh equal the oracle's."""
import numpy as np
import pytest

import scenegen
from _common import city_cam, compare_image, import_scene
from oracle import build as ob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_19415_b300 as mod
    return mod


CASES = {
    "blobs": (lambda: scenegen.blob_scene(n=8000, n_blobs=8, lo=0.0, hi=10.0, blob_sigma=0.7, ls_mu=-2.0,
                                          sh_degree=1, seed=13),
              dict(page_size=256, paging="mesh", lo=(-2, -2, -2), hi=(12, 12, 12), voxel=0.5, link_samples=2,
                   mesh_kappa=2.0, mesh_op_min=0.1, mesh_closing=1, mesh_qem_ratio=0.3)),
    "city_lod": (lambda: scenegen.city_scene(n=12000, n_boxes=5, extent=50.0),
                 dict(page_size=256, paging="mesh", lod_levels=3, lod_fanout=4, lo=(-4, -4, -4), hi=(54, 54, 84),
                      voxel=3.0, link_samples=2, mesh_kappa=2.0, mesh_op_min=0.1, mesh_closing=1,
                      mesh_qem_ratio=0.25)),
}


_ORACLE = {}


def _oracle(name):
    """The raw input and the oracle's scene of a case (built once per run)."""
    if name not in _ORACLE:
        gen, kw = CASES[name]
        raw = gen()
        _ORACLE[name] = (raw, ob.build_scene(raw, ob.BuildParams(**kw, seed=123)))
    return _ORACLE[name]


def _both(v, name):
    raw, osc = _oracle(name)
    psc = v.vm3dgs_build_pages(raw, v.BuildConfig(**CASES[name][1], seed=123, fp16=True))
    return raw, osc, psc


@pytest.mark.parametrize("name", list(CASES))
def test_mesh_build_matches_oracle(v, name):
    raw, osc, psc = _both(v, name)
    mp = osc.proxy["mesh"]
    assert mp["occ"].sum() > 100 and len(mp["surf_tris"]) > 100 and len(osc.tris) > 50
    assert psc.info.n_pages == osc.n_pages
    np.testing.assert_array_equal(psc.export(v.SCENE_PAGE_COUNT, dtype=np.int64), osc.count)
    src = psc.export(v.SCENE_PAGE_SRC, dtype=np.int64).reshape(osc.n_pages, -1)
    np.testing.assert_array_equal(src, np.where(osc.src >= 0, osc.dec_src[np.maximum(osc.src, 0)], -1))
    L0 = psc.unpack(0)
    for k in ("pos", "scale", "rot", "opacity", "sh"):
        np.testing.assert_array_equal(L0[k], osc.levels[0][k], err_msg=k)
    for l in range(1, len(osc.levels)):
        np.testing.assert_allclose(psc.unpack(l)["pos"], osc.levels[l]["pos"], rtol=1e-6, atol=1e-5)
    np.testing.assert_array_equal(psc.export(v.SCENE_VERTS, dtype=np.float32).reshape(-1, 3), osc.verts)
    np.testing.assert_array_equal(psc.export(v.SCENE_TRIS, dtype=np.int32).reshape(-1, 3), osc.tris)
    np.testing.assert_array_equal(psc.export(v.SCENE_FACE_PAGE, dtype=np.int32), osc.face_page)
    np.testing.assert_array_equal(psc.export(v.SCENE_LINK_PTR, dtype=np.int64), osc.link_ptr)
    np.testing.assert_array_equal(psc.export(v.SCENE_LINK_COL, dtype=np.int32), osc.link_col)


def test_mesh_proxy_frames_match_oracle(v):
    """A walk over the city built with the mesh proxy: visibility buffer,
    request words, page table, draw list and images equal the oracle's."""
    from test_gpu_vm import _run_trajectory
    raw, sc = _oracle("city_lod")
    cams = [city_cam(50.0, k, width=200, height=120) for k in range(6)]
    _run_trajectory(v, raw, sc, cams, pool_slots=10, budget_pages=4, lod=True, tau0=2.0, check_images=(0, 5))
