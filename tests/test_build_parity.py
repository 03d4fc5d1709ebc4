"""Host page builder (vm3dgs_build_pages) against the oracle's preparation:
page assignment, level-0 records, proxy mesh and links bit-exact; LOD levels
within FP64-rounding tolerance; fp16 records equal to IEEE round-to-nearest
half conversion.  Runs on the CPU (the builder needs no GPU)."""
import numpy as np
import pytest

import paper_2506_19415_b300 as v
import scenegen
from oracle import build as ob

CASES = {
    "tiny_morton": (lambda: scenegen.uniform_scene(),
                    dict(page_size=256, paging="morton", lo=(-5, -5, -5), hi=(5, 5, 5), voxel=10 / 32, kappa=0.5,
                         link_samples=8)),
    "blobs_octree_sh3": (lambda: scenegen.blob_scene(n=30000, n_blobs=12, seed=5),
                         dict(page_size=1024, paging="octree", lo=(-5, -5, -5), hi=(55, 55, 55), voxel=60 / 64,
                              kappa=2.0, link_samples=4)),
    "city_lod": (lambda: scenegen.city_scene(n=40000, n_boxes=12, extent=120.0),
                 dict(page_size=512, paging="octree", lod_levels=3, lod_fanout=8, lo=(-4, -4, -4),
                      hi=(124, 124, 84), voxel=4.0, kappa=0.5, link_samples=4)),
    "halving_lod": (lambda: scenegen.uniform_scene(n=5000, seed=8, sh_degree=1),
                    dict(page_size=256, paging="octree", lod_levels=4, lod_fanout=2, lo=(-5, -5, -5), hi=(5, 5, 5),
                         voxel=0.5, kappa=0.3, link_samples=2)),
    # the paper's own LOD: k-means per page, halving per level (Sec. 3.4)
    "kmeans_halving": (lambda: scenegen.uniform_scene(n=5000, seed=9, sh_degree=1),
                       dict(page_size=256, paging="octree", lod_levels=4, lod_fanout=2, lo=(-5, -5, -5),
                            hi=(5, 5, 5), voxel=0.5, kappa=0.3, link_samples=2, lod_method="kmeans", kmeans_iters=8)),
    "kmeans_city": (lambda: scenegen.city_scene(n=20000, n_boxes=8, extent=100.0),
                    dict(page_size=512, paging="octree", lod_levels=3, lod_fanout=2, lo=(-4, -4, -4),
                         hi=(104, 104, 84), voxel=4.0, kappa=0.5, link_samples=2, lod_method="kmeans",
                         kmeans_iters=10, kmeans_attr_weight=0.2)),
}


def _both(name):
    gen, kw = CASES[name]
    raw = gen()
    bp = ob.BuildParams(**kw, seed=123)
    osc = ob.build_scene(raw, bp)
    cfg = v.BuildConfig(**kw, seed=123, fp16=True)
    psc = v.vm3dgs_build_pages(raw, cfg)
    return raw, osc, psc


@pytest.mark.parametrize("name", list(CASES))
def test_builder_matches_oracle(name):
    raw, osc, psc = _both(name)
    assert psc.info.n_pages == osc.n_pages
    np.testing.assert_array_equal(psc.export(v.SCENE_PAGE_COUNT, dtype=np.int64), osc.count)
    src = psc.export(v.SCENE_PAGE_SRC, dtype=np.int64).reshape(osc.n_pages, -1)
    want = np.where(osc.src >= 0, osc.dec_src[np.maximum(osc.src, 0)], -1)
    np.testing.assert_array_equal(src, want)
    # level 0: decoded records bit-exact
    L0 = psc.unpack(0)
    for k in ("pos", "scale", "rot", "opacity", "sh"):
        np.testing.assert_array_equal(L0[k], osc.levels[0][k], err_msg=k)
    # LOD levels: moment matching in FP64, rounded to fp32 (eigen solvers differ in the last bits)
    for l in range(1, len(osc.levels)):
        Pl = psc.unpack(l)
        O = osc.levels[l]
        np.testing.assert_array_equal(Pl["opacity"] > 0, O["opacity"] > 0)
        np.testing.assert_allclose(Pl["pos"], O["pos"], rtol=1e-6, atol=1e-5)
        np.testing.assert_allclose(Pl["opacity"], O["opacity"], rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(Pl["sh"], O["sh"], rtol=1e-5, atol=1e-6)
        # compare covariances, not eigenvectors (equal eigenvalues leave them free)
        def cov(d):
            R = ob.quat_to_rot(d["rot"].astype(np.float64))
            s = d["scale"].astype(np.float64)
            return np.einsum("...ik,...k,...jk->...ij", R, s * s, R)
        cp, co = cov(Pl), cov(O)
        scale = np.abs(co).max(axis=(-1, -2), keepdims=True) + 1e-30
        assert np.max(np.abs(cp - co) / scale) < 1e-5
    np.testing.assert_allclose(psc.export(v.SCENE_ERR, dtype=np.float32).reshape(osc.n_pages, -1), osc.err, rtol=1e-6)
    # proxy and links: exact
    np.testing.assert_array_equal(psc.export(v.SCENE_VERTS, dtype=np.float32).reshape(-1, 3), osc.verts)
    np.testing.assert_array_equal(psc.export(v.SCENE_TRIS, dtype=np.int32).reshape(-1, 3), osc.tris)
    np.testing.assert_array_equal(psc.export(v.SCENE_FACE_PAGE, dtype=np.int32), osc.face_page)
    np.testing.assert_array_equal(psc.export(v.SCENE_LINK_PTR, dtype=np.int64), osc.link_ptr)
    np.testing.assert_array_equal(psc.export(v.SCENE_LINK_COL, dtype=np.int32), osc.link_col)


def test_fp16_records_round_to_nearest_even():
    raw, osc, psc = _both("blobs_octree_sh3")
    K = (raw.sh_degree + 1) ** 2
    m = psc.info.page_size
    rec16 = psc.info.record_bytes16
    assert rec16 == 16 + 2 * ((7 + 3 * K + 1) & ~1) == 128
    b = psc.pages(0, fp16=True)
    f = b[:, :16 * m].view(np.float32).reshape(osc.n_pages, 4, m)
    h = b[:, 16 * m:].view(np.float16).reshape(osc.n_pages, -1, m)
    O = osc.levels[0]
    np.testing.assert_array_equal(f[:, 0:3].transpose(0, 2, 1), O["pos"])
    np.testing.assert_array_equal(f[:, 3], O["opacity"])
    np.testing.assert_array_equal(h[:, 0:3].transpose(0, 2, 1), O["scale"].astype(np.float16))
    np.testing.assert_array_equal(h[:, 3:7].transpose(0, 2, 1), O["rot"].astype(np.float16))
    sh = h[:, 7:7 + 3 * K].transpose(0, 2, 1).reshape(osc.n_pages, m, K, 3)
    np.testing.assert_array_equal(sh, O["sh"].astype(np.float16))


def test_import_roundtrip():
    raw, osc, psc = _both("city_lod")
    imp = v.vm3dgs_scene_import(osc.levels, osc.err, osc.count, osc.verts, osc.tris, osc.face_page, osc.link_ptr,
                                osc.link_col, osc.params.page_size, osc.params.lod_fanout, raw.sh_degree, fp16=True)
    for l in range(len(osc.levels)):
        U = imp.unpack(l)
        for k in U:
            np.testing.assert_array_equal(U[k], osc.levels[l][k])
    np.testing.assert_array_equal(imp.pages(0, fp16=True), psc.pages(0, fp16=True))


def _ulps(a, b):
    """Distance in units in the last place between fp32 arrays."""
    ia = a.astype(np.float32).view(np.int32).astype(np.int64)
    ib = b.astype(np.float32).view(np.int32).astype(np.int64)
    ia = np.where(ia < 0, -(ia & 0x7FFFFFFF), ia)
    ib = np.where(ib < 0, -(ib & 0x7FFFFFFF), ib)
    return np.abs(ia - ib)


@pytest.mark.parametrize("name", ["kmeans_halving", "kmeans_city"])
def test_kmeans_levels_match_oracle(name):
    """k-means LOD: the same clusters (hence the same parents in the same
    slots) and every merged attribute within one fp32 ulp of the oracle's;
    both sides run the same sequence of FP64 operations except the
    quaternion norms and the error's distance, which may round differently."""
    raw, osc, psc = _both(name)
    for l in range(1, len(osc.levels)):
        Pl, O = psc.unpack(l), osc.levels[l]
        np.testing.assert_array_equal(Pl["opacity"] > 0, O["opacity"] > 0)
        for k in ("pos", "scale", "rot", "opacity", "sh"):
            assert int(_ulps(Pl[k], O[k]).max()) <= 1, (l, k)
    e = psc.export(v.SCENE_ERR, dtype=np.float32).reshape(osc.n_pages, -1)
    assert int(_ulps(e, osc.err).max()) <= 1
    # the paper's halving: real parents per page at most ceil(children / fanout)
    F = osc.params.lod_fanout
    for l in range(1, len(osc.levels)):
        a = (osc.levels[l - 1]["opacity"] > 0).sum(1)
        b = (osc.levels[l]["opacity"] > 0).sum(1)
        assert np.all(b <= -(-a // F)) and np.all(b >= 1)


def test_kmeans_parameters_rejected():
    raw = scenegen.uniform_scene(n=500, seed=2)
    for bad in (dict(kmeans_iters=0), dict(kmeans_scale=-1.0), dict(kmeans_attr_weight=-0.5)):
        with pytest.raises(v.Vm3dgsError):
            v.vm3dgs_build_pages(raw, v.BuildConfig(page_size=64, lod_levels=2, lod_fanout=2, lod_method="kmeans",
                                                    **bad))
    with pytest.raises(ValueError):
        v.BuildConfig(lod_method="median").struct()
