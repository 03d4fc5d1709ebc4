"""The sort entry point that allocates nothing (vm3dgs_sort_pairs_noalloc).

It serves callers that cannot allocate device memory: a host that owns all of
it and hands libraries only its own buffers, or a frame loop that cannot pay
the device-wide synchronisation of cudaMalloc and cudaFree.  Checked here:
- against the sort inside vm3dgs_render: the renderer's own pairs, put back
  in emission order (splat by splat, tiles ascending), sorted by the new call
  give exactly the keys and values vm3dgs_render sorted, on two calls in a
  row (the second on another view, so leftovers of the first are exercised);
- against a host stable sort on the masked key (numpy, kind="stable") for
  n in {0, 1, 2, 2^19} and key_bits in {1, 13, 40, 45, 64}, on the default
  stream and on another one;
- that a call leaves the device's free memory unchanged once the library
  is loaded;
- that the binding refuses tensors the C ABI cannot check.
Collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

import scenegen
from _common import import_scene, tiny_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_19415_b300 as mod
    return mod


def _render_pairs(v, r, cam):
    """Sorted pairs of vm3dgs_render, and the same pairs in emission order
    (by splat, then by tile: a splat's tiles ascend in row-major order)."""
    r.request_all()
    r.update_residency()
    r.render([cam])
    keys = r.debug(v.DBG_KEYS, np.uint64)
    vals = r.debug(v.DBG_VALUES, np.uint32)
    order = np.lexsort((keys >> np.uint64(32), vals))
    ntiles = ((cam.width + cam.tile_w - 1) // cam.tile_w) * ((cam.height + cam.tile_h - 1) // cam.tile_h)
    bits = 32 + max(int(ntiles - 1).bit_length(), 0)
    return keys, vals, keys[order].copy(), vals[order].copy(), bits


def _sort(v, k, val, bits, stream=None):
    import torch
    kd = torch.from_numpy(k.view(np.int64).copy()).cuda()
    vd = torch.from_numpy(val.view(np.int32).copy()).cuda()
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    v.vm3dgs_sort_pairs_noalloc(kd, vd, len(k), bits, status, stream=stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return kd.cpu().numpy().view(np.uint64), vd.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_render_sort(v):
    raw, sc = tiny_scene()
    scene = import_scene(v, raw, sc)
    cams = [scenegen.tiny_camera(width=256, height=256),
            scenegen.look_at((9.0, -6.0, -11.0), (0, 0, 0), (0, -1, 0), 200, 144, 60.0, (8, 8))]
    for cam in cams:
        r = v.Renderer(scene, v.RenderConfig(max_width=cam.width, max_height=cam.height, lod=False,
                                             staging_bytes=1 << 40), pool_slots=sc.n_pages)
        want_k, want_v, k, val, bits = _render_pairs(v, r, cam)
        assert 0 < len(k) <= v.NOALLOC_MAX_PAIRS
        gk, gv = _sort(v, k, val, bits)
        np.testing.assert_array_equal(gk, want_k)
        np.testing.assert_array_equal(gv, want_v)


@pytest.mark.parametrize("n", [0, 1, 2, 1 << 19])
@pytest.mark.parametrize("key_bits", [1, 13, 40, 45, 64])
def test_noalloc_sort_matches_host_stable_sort(v, n, key_bits):
    """Random 64-bit keys (bits above key_bits set too, so they must not
    order), values = input position; a second call on a non-default stream
    with the reversed input."""
    import torch
    rng = np.random.default_rng(1000 * key_bits + n % 997)
    k = rng.integers(0, 2 ** 63, size=n, dtype=np.int64).view(np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=n, dtype=np.int64).view(np.uint64)
    if key_bits < 64 and n > 4:
        k[: n // 4] &= ~np.uint64((1 << key_bits) - 1)  # equal masked keys: stability matters
    val = np.arange(n, dtype=np.uint32)
    mask = np.uint64(0xFFFFFFFFFFFFFFFF) if key_bits == 64 else np.uint64((1 << key_bits) - 1)
    for kk, vv, stream in ((k, val, None), (k[::-1].copy(), val[::-1].copy(), torch.cuda.Stream())):
        order = np.argsort(kk & mask, kind="stable")
        gk, gv = _sort(v, kk, vv, key_bits, stream)
        np.testing.assert_array_equal(gk, kk[order])
        np.testing.assert_array_equal(gv, vv[order])


def test_noalloc_sort_allocates_nothing(v):
    """After a first call (which loads the library's module on the device),
    further calls leave the device's free memory unchanged."""
    import torch
    n = 1 << 19
    rng = np.random.default_rng(7)
    kd = torch.from_numpy(rng.integers(0, 2 ** 40, size=n, dtype=np.int64)).cuda()
    vd = torch.arange(n, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    v.vm3dgs_sort_pairs_noalloc(kd, vd, n, 40, status)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for bits in (40, 64, 13):
        v.vm3dgs_sort_pairs_noalloc(kd, vd, n, bits, status)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(status.item()) == 0


def test_noalloc_sort_rejects_bad_arguments(v):
    import torch
    kd = torch.zeros(4, dtype=torch.int64, device="cuda")
    vd = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(v.Vm3dgsError) as e:
        v.vm3dgs_sort_pairs_noalloc(kd, vd, v.NOALLOC_MAX_PAIRS + 1, 40)
    assert e.value.code == v.E_CAPACITY
    for bad_k, bad_v, n, bits in ((kd, vd, 5, 40),                      # n beyond the tensors
                                  (kd.cpu(), vd, 4, 40),                # host tensor
                                  (kd[::2], vd[:2], 2, 40),             # not contiguous
                                  (kd.to(torch.float64), vd, 4, 40),    # wrong dtype
                                  (kd, vd, 4, 0), (kd, vd, 4, 65)):     # key_bits out of range
        with pytest.raises(v.Vm3dgsError) as e:
            v.vm3dgs_sort_pairs_noalloc(bad_k, bad_v, n, bits)
        assert e.value.code == v.E_INVAL
