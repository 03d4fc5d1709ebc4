"""The host steps of the mesh proxy (quadric simplification, page
assignment by nearest triangle with subdivision and merging) in the library
against the oracle, bit for bit, on surfaces the oracle extracts (no GPU
needed)."""
import numpy as np
import pytest

from oracle import mesh as om


@pytest.fixture(scope="module")
def v():
    import paper_2506_19415_b300 as mod
    return mod


def _ball_surface(n=12, r2=16.0, seed=0):
    rng = np.random.default_rng(seed)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    c = np.array([(n - 1) / 2] * 3) + rng.normal(0, 0.3, 3)
    occ = ((x - c[0]) ** 2 + 1.3 * (y - c[1]) ** 2 + (z - c[2]) ** 2) <= r2
    D, T = om.surface(occ)
    return 0.25 + D.astype(np.float64) * 0.125, T


@pytest.mark.parametrize("seed,ratio", [(0, 0.25), (1, 0.5), (2, 0.1)])
def test_simplify_matches_oracle(v, seed, ratio):
    V, T = _ball_surface(seed=seed)
    target = max(4, int(len(T) * ratio))
    ov, ot = om.qem_simplify(V, T, target)
    gv, gt = v.vm3dgs_mesh_simplify(V, T, target)
    np.testing.assert_array_equal(gt.astype(np.int64), ot)
    np.testing.assert_array_equal(gv, ov)


@pytest.mark.parametrize("page_size", [32, 100])
def test_assign_pages_matches_oracle(v, page_size):
    V, T = _ball_surface(n=10, r2=12.0, seed=3)
    V, T = om.qem_simplify(V, T, len(T) // 3)
    rng = np.random.default_rng(4)
    d = rng.normal(size=(2500, 3))
    mu = (0.25 + 0.125 * 4.5 + d / np.linalg.norm(d, axis=1, keepdims=True) *
          rng.uniform(0.3, 0.62, (2500, 1))).astype(np.float32)
    want = om.assign_pages(mu, V, T, page_size)
    got = v.vm3dgs_mesh_assign_pages(mu, page_size, V, T)
    np.testing.assert_array_equal(got["verts"], want["verts"])
    np.testing.assert_array_equal(got["tris"].astype(np.int64), want["tris"])
    np.testing.assert_array_equal(got["face_page"].astype(np.int64), want["face_page"])
    np.testing.assert_array_equal(got["order"], want["order"])
    np.testing.assert_array_equal(got["counts"], want["counts"])
    np.testing.assert_array_equal(got["parent"], want["parent"])
