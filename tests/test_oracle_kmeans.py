"""Pins of the oracle's k-means LOD (Sec. 3.4, "Level of Detail") against
what does not depend on it: SciPy's Lloyd iterations, closed forms on
separated pairs, the fixed-point property of a converged clustering, and the
halving of the Gaussian count per level."""
import warnings

import numpy as np
import pytest

import oracle.build as ob


def _page(rng, n, K=4):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return dict(pos=rng.uniform(-3, 3, (n, 3)).astype(np.float32),
                scale=rng.uniform(0.01, 0.2, (n, 3)).astype(np.float32),
                rot=q.astype(np.float32), opacity=rng.uniform(0.05, 1, n).astype(np.float32),
                sh=rng.normal(0, 0.5, (n, K, 3)).astype(np.float32))


@pytest.mark.parametrize("iters", [1, 3, 50])
def test_lloyd_equals_scipy_kmeans2(iters):
    """SciPy's kmeans2 with a given initial code book runs the same Lloyd
    rounds (nearest centroid, mean update, empty clusters kept) and returns
    the last assignment; the early stop must not change the result."""
    from scipy.cluster.vq import kmeans2
    rng = np.random.default_rng(3)
    g = _page(rng, 300)
    X = ob.kmeans_features(g["pos"], g["rot"], g["opacity"], g["sh"], 0.25)
    k = 150
    C0 = X[[i * 300 // k for i in range(k)]]
    lab, C = ob.kmeans_lloyd(X, C0, iters)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        Cs, ls = kmeans2(X, C0.copy(), iter=iters, minit="matrix")
    assert np.array_equal(lab, ls)
    np.testing.assert_allclose(C, Cs, rtol=0, atol=1e-12)


def test_features_definition():
    """Position centred and divided by the RMS radius (unit RMS after);
    quaternion sign folded to w >= 0; attributes weighted."""
    rng = np.random.default_rng(4)
    g = _page(rng, 64)
    X = ob.kmeans_features(g["pos"], g["rot"], g["opacity"], g["sh"], 0.5)
    assert abs(np.sqrt((X[:, :3] ** 2).sum(1).mean()) - 1) < 1e-12
    assert np.all(np.abs(X[:, :3].mean(0)) < 1e-12)
    assert np.all(X[:, 3] >= 0)
    np.testing.assert_allclose(np.abs(X[:, 3:7]), 0.5 * np.abs(g["rot"].astype(np.float64)), rtol=0, atol=0)
    np.testing.assert_array_equal(X[:, 10], 0.5 * g["opacity"].astype(np.float64))
    # q and -q are the same rotation and the same feature
    g2 = dict(g, rot=-g["rot"])
    X2 = ob.kmeans_features(g2["pos"], g2["rot"], g2["opacity"], g2["sh"], 0.5)
    np.testing.assert_array_equal(X[np.abs(g["rot"][:, 0]) > 0], X2[np.abs(g["rot"][:, 0]) > 0])


def test_merge_cluster_closed_forms():
    rng = np.random.default_rng(5)
    g = _page(rng, 3)
    one = ob.merge_cluster(g["pos"][:1], g["scale"][:1], g["rot"][:1], g["opacity"][:1], g["sh"][:1], 1.26)
    np.testing.assert_array_equal(one["pos"], g["pos"][0].astype(np.float64))
    np.testing.assert_array_equal(one["scale"], g["scale"][0].astype(np.float64))   # no factor for one member
    q0 = g["rot"][0].astype(np.float64)
    np.testing.assert_allclose(one["rot"], q0 / np.linalg.norm(q0) * np.sign(q0[0]), atol=1e-7)
    # two members, the second stored as the opposite quaternion of the first
    rot = np.stack([g["rot"][0], -g["rot"][0]])
    two = ob.merge_cluster(g["pos"][:2], g["scale"][:2], rot, g["opacity"][:2], g["sh"][:2], 2 ** (1 / 3))
    np.testing.assert_allclose(two["rot"], one["rot"], atol=1e-7)
    np.testing.assert_allclose(two["pos"], g["pos"][:2].astype(np.float64).mean(0), atol=1e-12)
    np.testing.assert_allclose(two["scale"], g["scale"][:2].astype(np.float64).mean(0) * 2 ** (1 / 3), atol=1e-12)
    np.testing.assert_allclose(two["opacity"], g["opacity"][:2].astype(np.float64).mean(), atol=1e-12)
    np.testing.assert_allclose(two["sh"], g["sh"][:2].astype(np.float64).mean(0), atol=1e-12)


@pytest.mark.parametrize("shared_attrs,weight", [(True, 0.1), (True, 1.0), (False, 0.0)])
def test_separated_pairs_merge_pairwise(shared_attrs, weight):
    """32 tight pairs on a line, 10 apart, one page of 64 (pair members
    adjacent in slot order): halving merges exactly each pair -- whatever the
    attribute weight when the members of a pair share their other
    attributes, and on position alone (weight 0) when they do not.  Parents
    are the pair means with the mean scale times 2^(1/3); e_1 is half the
    pair spread plus the largest member scale."""
    rng = np.random.default_rng(6)
    n = 64
    g = _page(rng, n)
    if shared_attrs:
        for k in ("rot", "opacity", "sh"):
            g[k][1::2] = g[k][0::2]
    base = np.repeat(np.arange(32) * 10.0, 2)
    g["pos"] = np.stack([base + np.tile([0.0, 0.02], 32), np.zeros(n), np.zeros(n)], 1).astype(np.float32)
    pages = {k: v[None] for k, v in g.items()}
    levels, err, labels = ob.lod_build_kmeans(pages, 2, 2, iters=10, attr_weight=weight)
    assert np.array_equal(labels[1][0], np.repeat(np.arange(32), 2))
    L1 = levels[1]
    for j in range(32):
        np.testing.assert_allclose(L1["pos"][0, j], g["pos"][2 * j:2 * j + 2].astype(np.float64).mean(0), atol=1e-5)
        np.testing.assert_allclose(L1["scale"][0, j],
                                   g["scale"][2 * j:2 * j + 2].astype(np.float64).mean(0) * 2 ** (1 / 3), rtol=1e-6)
    want = max(0.01 + float(g["scale"][i].max()) for i in range(n))
    assert abs(float(err[0, 1]) - want) < 1e-5


def test_converged_clustering_is_a_fixed_point():
    """Run to convergence: every real child's own centroid (the mean of its
    cluster's features) is its nearest one, and the number of parents is the
    number of non-empty clusters, at most ceil(n / fanout)."""
    rng = np.random.default_rng(7)
    n, F = 120, 2
    g = _page(rng, n)
    X = ob.kmeans_features(g["pos"], g["rot"], g["opacity"], g["sh"], 0.25)
    k = -(-n // F)
    lab, C = ob.kmeans_lloyd(X, X[[i * n // k for i in range(k)]], 1000)
    used = np.unique(lab)
    for c in used:
        np.testing.assert_allclose(C[c], X[lab == c].mean(0), atol=1e-12)
    D = ((X[:, None, :] - C[None, used, :]) ** 2).sum(-1)
    assert np.array_equal(used[D.argmin(1)], lab)
    pages = {kk: np.concatenate([v, np.zeros((8,) + v.shape[1:], v.dtype)])[None] for kk, v in g.items()}
    levels, err, labels = ob.lod_build_kmeans(pages, 2, F, iters=1000)
    n_par = int((levels[1]["opacity"][0] > 0).sum())
    assert n_par == len(used) <= k
    assert np.all(levels[1]["opacity"][0, n_par:] == 0)      # padding after the parents


def test_kmeans_scene_halves_per_level():
    """A full oracle build with the paper's halving (fanout 2, 4 levels):
    block sizes m_l = page_size / 2^l, real parents per page at most
    ceil(real children / 2), errors non-negative and 0 at level 0."""
    import scenegen
    raw = scenegen.city_scene(n=6000, n_boxes=6, extent=60.0)
    bp = ob.BuildParams(page_size=128, paging="octree", lod_levels=4, lod_fanout=2, lo=(-4, -4, -4),
                        hi=(64, 64, 88), voxel=2.0, kappa=0.5, link_samples=0, lod_method="kmeans", kmeans_iters=6)
    sc = ob.build_scene(raw, bp)
    for l in range(4):
        assert sc.m(l) == 128 >> l
    for l in range(1, 4):
        prev = (sc.levels[l - 1]["opacity"] > 0).sum(1)
        cur = (sc.levels[l]["opacity"] > 0).sum(1)
        assert np.all(cur <= -(-prev // 2)) and np.all(cur >= 1) and np.all(cur >= prev // 4)
    assert np.all(sc.err[:, 0] == 0) and np.all(sc.err[:, 1:] > 0)
