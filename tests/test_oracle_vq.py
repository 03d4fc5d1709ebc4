"""Pins of the oracle's SH codebook (compressed pages: oracle.build.quantize_sh,
nearest_code, vq_levels) against closed forms and independent recomputation:
- exact recovery: SH vectors drawn from n_codes prototypes, laid out so that
  the initial codewords are the prototypes, come back exactly;
- every code is a nearest codeword (brute force with numpy's norm), the
  lowest index on a tie;
- after convergence every codeword is the mean of its training vectors, and
  the codebook equals SciPy's kmeans2 from the same initial codewords;
- the decoded record keeps position and opacity, rounds scale, rotation and
  SH band 0 to fp16 and takes bands 1..3 from the codebook."""
import numpy as np
import pytest

import scenegen
from oracle import build as ob


def _levels(n_pages=6, m=64, K=16, seed=3, padding=8):
    rng = np.random.default_rng(seed)
    L = dict(pos=rng.normal(size=(n_pages, m, 3)).astype(np.float32),
             scale=np.exp(rng.normal(-3, 0.3, size=(n_pages, m, 3))).astype(np.float32),
             rot=rng.normal(size=(n_pages, m, 4)).astype(np.float32),
             opacity=rng.uniform(0.1, 1.0, size=(n_pages, m)).astype(np.float32),
             sh=rng.normal(0, 0.1, size=(n_pages, m, K, 3)).astype(np.float32))
    L["opacity"][:, m - padding:] = 0.0       # padding slots
    L["sh"][:, m - padding:] = 0.0
    return [L]


def test_exact_recovery_of_prototypes():
    n_codes, K = 16, 16
    levels = _levels(n_pages=4, m=64, K=K, padding=0)
    L = levels[0]
    rng = np.random.default_rng(11)
    proto = rng.normal(0, 0.2, size=(n_codes, K - 1, 3)).astype(np.float32)
    T = L["opacity"].size                       # all real: 256 = 16 per prototype
    r = T // n_codes
    which = (np.arange(T) // r).reshape(L["opacity"].shape)
    L["sh"][:, :, 1:, :] = proto[which]
    cb, codes = ob.quantize_sh(levels, n_codes, iters=5)
    np.testing.assert_array_equal(cb, proto.reshape(n_codes, -1))
    np.testing.assert_array_equal(codes[0], which)
    dec = ob.vq_levels(levels, cb, codes)[0]
    np.testing.assert_array_equal(dec["sh"][:, :, 1:, :], L["sh"][:, :, 1:, :])


def test_codes_are_nearest_codewords():
    levels = _levels()
    cb, codes = ob.quantize_sh(levels, 32, iters=4, n_train=200)
    X = ob.sh_rest(levels[0]["sh"]).reshape(-1, cb.shape[1]).astype(np.float64)
    D = np.linalg.norm(X[:, None, :] - cb.astype(np.float64)[None], axis=2) ** 2
    c = codes[0].reshape(-1)
    best = D.min(1)
    got = D[np.arange(len(X)), c]
    assert np.all(got <= best * (1 + 1e-12) + 1e-300)
    # no lower index is clearly nearer (ties go to the lowest index)
    for i in range(len(X)):
        lower = D[i, :c[i]]
        assert not np.any(lower < got[i] * (1 - 1e-12))
    # padding (zero SH) also gets a code: the codeword nearest the origin
    pad = levels[0]["opacity"].reshape(-1) == 0
    assert np.all(c[pad] == np.argmin((cb.astype(np.float64) ** 2).sum(1)))


def test_converged_codebook_is_the_mean_of_its_vectors_and_equals_scipy():
    from scipy.cluster.vq import kmeans2
    levels = _levels(n_pages=8, m=64)
    n_codes = 12
    cb, _ = ob.quantize_sh(levels, n_codes, iters=200)
    X = ob.sh_rest(levels[0]["sh"]).reshape(-1, cb.shape[1]).astype(np.float64)
    train = X[levels[0]["opacity"].reshape(-1) > 0]
    lab = ob.nearest_code(train, cb)
    for j in range(n_codes):
        mem = train[lab == j]
        assert len(mem) > 0
        np.testing.assert_allclose(cb[j], mem.mean(0), rtol=0, atol=1e-6)
    T = len(train)
    C0 = train[[j * T // n_codes for j in range(n_codes)]]
    with np.errstate(all="ignore"):
        Cs, _ = kmeans2(train, C0.copy(), iter=200, minit="matrix")
    np.testing.assert_allclose(cb, Cs.astype(np.float32), rtol=0, atol=1e-6)


def test_training_sample_positions():
    """With n_train below the real Gaussians the training set is the real
    Gaussians at floor(j T / n_train): a codebook of n_train codes is that set."""
    levels = _levels(n_pages=2, m=64, padding=4)
    cb, _ = ob.quantize_sh(levels, 10, iters=0, n_train=10)
    X = ob.sh_rest(levels[0]["sh"]).reshape(-1, cb.shape[1])
    real = X[levels[0]["opacity"].reshape(-1) > 0]
    T = len(real)
    np.testing.assert_array_equal(cb, real[[j * T // 10 for j in range(10)]])


def test_decoded_record_fields():
    levels = _levels()
    cb, codes = ob.quantize_sh(levels, 8, iters=3)
    L, D = levels[0], ob.vq_levels(levels, cb, codes)[0]
    np.testing.assert_array_equal(D["pos"], L["pos"])
    np.testing.assert_array_equal(D["opacity"], L["opacity"])
    for k in ("scale", "rot"):
        np.testing.assert_array_equal(D[k], L[k].astype(np.float16).astype(np.float32))
    np.testing.assert_array_equal(D["sh"][:, :, 0], L["sh"][:, :, 0].astype(np.float16).astype(np.float32))
    np.testing.assert_array_equal(D["sh"][:, :, 1:].reshape(-1, cb.shape[1]), cb[codes[0].reshape(-1)])


def test_degree_zero_is_refused():
    levels = _levels(K=1)
    with pytest.raises(ValueError):
        ob.quantize_sh(levels, 4)


def test_all_levels_of_a_built_scene_get_codes():
    raw = scenegen.blob_scene(n=3000, n_blobs=4, lo=0.0, hi=10.0, blob_sigma=0.7, ls_mu=-2.0, sh_degree=2, seed=5)
    sc = ob.build_scene(raw, ob.BuildParams(page_size=256, paging="octree", lod_levels=2, lod_fanout=4,
                                            lo=(-2, -2, -2), hi=(12, 12, 12), voxel=1.0, link_samples=2))
    cb, codes = ob.quantize_sh(sc.levels, 16, iters=4)
    assert cb.shape == (16, 24) and len(codes) == 2
    for L, c in zip(sc.levels, codes):
        assert c.shape == L["opacity"].shape and c.min() >= 0 and c.max() < 16
        X = ob.sh_rest(L["sh"]).reshape(-1, 24).astype(np.float64)
        np.testing.assert_array_equal(c.reshape(-1), ob.nearest_code(X, cb))
