"""The sort entry point that allocates nothing (vm3dgs_sort_pairs_noalloc),
for callers that cannot allocate device memory (their host owns all of it,
or their frame loop cannot afford cudaMalloc's synchronisation), against the
sort inside vm3dgs_render: the renderer's own pairs, rebuilt in emission
order from its splat rectangles and depths, sorted by the new call give
exactly the keys and values vm3dgs_render sorted, on two calls in a row
(the second on another view, so leftovers of the first are exercised).
Pairs of a splat are the tiles of its rectangle met by its 3-sigma ellipse
(read back as its tile mask), row-major.  Collected last so that a failure
here leaves every other test already run."""
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
    """Sorted pairs of vm3dgs_render, and the same pairs in emission order."""
    r.request_all()
    r.update_residency()
    r.render([cam])
    keys = r.debug(v.DBG_KEYS, np.uint64)
    vals = r.debug(v.DBG_VALUES, np.uint32)
    n = r.stats()["drawn_gaussians"]
    rect = r.debug(v.DBG_SPLAT_RECT, np.int32).reshape(n, 4)
    depth = r.debug(v.DBG_SPLAT_DEPTH, np.float32).view(np.uint32)
    tmask = r.debug(v.DBG_SPLAT_TMASK, np.uint64)
    gx = (cam.width + cam.tile_w - 1) // cam.tile_w
    ek, ev = [], []
    for i in range(n):
        x0, y0, x1, y1 = (int(c) for c in rect[i])
        bit = 0
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                if (x1 - x0) * (y1 - y0) > 64 or (int(tmask[i]) >> bit) & 1:
                    ek.append((int(ty * gx + tx) << 32) | int(depth[i]))
                    ev.append(i)
                bit += 1
    ntiles = gx * ((cam.height + cam.tile_h - 1) // cam.tile_h)
    bits = 32 + max(int(ntiles - 1).bit_length(), 0)
    return keys, vals, np.array(ek, np.uint64), np.array(ev, np.uint32), bits


def test_noalloc_sort_matches_render_sort(v):
    import torch
    raw, sc = tiny_scene()
    scene = import_scene(v, raw, sc)
    cams = [scenegen.tiny_camera(width=256, height=256),
            scenegen.look_at((9.0, -6.0, -11.0), (0, 0, 0), (0, -1, 0), 200, 144, 60.0, (8, 8))]
    for cam in cams:
        r = v.Renderer(scene, v.RenderConfig(max_width=cam.width, max_height=cam.height, lod=False,
                                             staging_bytes=1 << 40), pool_slots=sc.n_pages)
        want_k, want_v, k, val, bits = _render_pairs(v, r, cam)
        assert 0 < len(k) <= v.NOALLOC_MAX_PAIRS
        kd = torch.from_numpy(k.view(np.int64)).cuda()
        vd = torch.from_numpy(val.view(np.int32)).cuda()
        status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
        v.vm3dgs_sort_pairs_noalloc(kd, vd, len(k), bits, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        np.testing.assert_array_equal(kd.cpu().numpy().view(np.uint64), want_k)
        np.testing.assert_array_equal(vd.cpu().numpy().view(np.uint32), want_v)


def test_noalloc_sort_rejects_oversize(v):
    import torch
    kd = torch.zeros(4, dtype=torch.int64, device="cuda")
    vd = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(v.Vm3dgsError) as e:
        v.vm3dgs_sort_pairs_noalloc(kd, vd, v.NOALLOC_MAX_PAIRS + 1, 40)
    assert e.value.code == v.E_CAPACITY
