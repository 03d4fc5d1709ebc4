"""Pins of the oracle's LOD cross-fade (oracle.residency.update with
fade_frames > 0; oracle.gather_draw weights) against scripted closed-form
sequences, brute-force invariants and the compositing formula:
- without a level change a fading table equals a non-fading one;
- a page that moves from level 0 to 1 is drawn at both for F frames with
  weights (a+1)/(F+1) and 1 - that, then at its new level alone;
- the old copy is never evicted or copied during the fade and the new one
  is placed as without fading;
- a return to the old level ends the fade; a page seen for the first time,
  or whose old level is not resident, does not fade;
- two equal co-located Gaussians with weights w and 1 - w composite as
  front-to-back blending of alphas w a and (1 - w) a."""
import numpy as np

import oracle
import scenegen
from oracle import build as ob
from oracle import residency as rs

F32 = np.float32


def _table(F, entries=6, levels=2, fanout=2, page_size=8, budget_pages=10):
    rp = rs.ResidencyParams(n_entries=entries, page_size=page_size, levels=levels, fanout=fanout, record_bytes=4,
                            budget_bytes=budget_pages * page_size * 4, lod=True, fade_frames=F)
    return rs.PageTable(rp)


def _frame(pt, req):
    """req: {page: level}; all direct, nearer pages first by page id."""
    pages = np.array(sorted(req), np.int64)
    enc = np.array([1000 - p for p in pages], np.uint32)
    direct = np.ones(len(pages), np.uint8)
    lv = np.array([req[p] for p in pages], np.int64)
    up = rs.update(pt, pages, enc, direct, lv)
    pt.frame += 1
    return up


def test_no_level_change_equals_no_fade():
    rng = np.random.default_rng(5)
    a, b = _table(0), _table(4)
    for f in range(30):
        req = {int(p): 0 for p in rng.choice(12, size=5, replace=False)}
        ua, ub = _frame(a, req), _frame(b, req)
        for k in ("copies", "draw", "missing"):
            assert ua[k] == ub[k], (f, k)
        assert all(w == F32(1) for w in ub["draw_w"])
        np.testing.assert_array_equal(a.slot, b.slot)


def test_scripted_fade_weights_and_end():
    F = 4
    pt = _table(F)
    _frame(pt, {3: 0})
    _frame(pt, {3: 0})
    seen = []
    for f in range(F + 2):
        up = _frame(pt, {3: 1})
        seen.append([(t[1], float(w)) for t, w in zip(up["draw"], up["draw_w"])])
        if f == 0:
            assert len(up["copies"]) == 1 and up["copies"][0][:2] == (3, 1)   # only the new level is copied
        else:
            assert up["copies"] == []
    for a in range(F):
        wn = F32(a + 1) / F32(F + 1)
        assert seen[a] == [(1, float(wn)), (0, float(F32(1) - wn))], (a, seen[a])
        assert abs(float(wn) + float(F32(1) - wn) - 1.0) <= 2 ** -23
    assert seen[F] == [(1, 1.0)] and seen[F + 1] == [(1, 1.0)]


def test_old_copy_is_kept_under_pressure():
    """Two entries only: the page's level-0 entry stays required (last used
    = this frame) through the fade, so other requests cannot evict it."""
    F = 3
    pt = _table(F, entries=3)
    _frame(pt, {0: 0})                      # entry for (0, L0)
    e_old = int(np.nonzero(pt.lod == 0)[0][0])
    for f in range(F):
        up = _frame(pt, {0: 1, 5: 0, 6: 0, 7: 0})   # pressure: more pages than entries
        assert pt.lod[e_old] == 0 and pt.slot[e_old, 0] == 0
        assert pt.last_used[e_old] == pt.frame - 1
        assert (0, 0, e_old, 0) in up["draw"]
        assert all(c[0] != 0 or c[1] == 1 for c in up["copies"])
        # no (page, level) twice in the table
        held = [(int(pt.slot[e, s]), int(pt.lod[e])) for e in range(3) for s in range(2 ** max(pt.lod[e], 0))
                if pt.lod[e] >= 0 and pt.slot[e, s] >= 0]
        assert len(held) == len(set(held))


def test_return_to_old_level_and_no_fade_cases():
    F = 5
    pt = _table(F)
    up = _frame(pt, {2: 1})                 # first appearance at level 1: no fade
    assert up["fading"] == 0
    _frame(pt, {2: 1})
    up = _frame(pt, {2: 0})                 # 1 -> 0: level 0 not resident yet, old (level 1) resident
    assert up["fading"] == 1 and [t[1] for t in up["draw"]] == [0, 1]
    up = _frame(pt, {2: 1})                 # back to the fade's old level: the fade ends
    # a new fade starts from level 0 (drawn last frame) to 1
    assert up["fading"] == 1 and [t[1] for t in up["draw"]] == [1, 0]
    assert float(up["draw_w"][0]) == float(F32(1) / F32(F + 1))
    up = _frame(pt, {9: 0})                 # page 2 not requested: its state is forgotten
    assert 2 not in pt.fade
    up = _frame(pt, {2: 0})
    assert up["fading"] == 0


def test_weighted_pair_composites_front_to_back():
    """One Gaussian drawn twice (as a page at two levels with equal
    attributes) with weights w, 1 - w at the same depth: a pixel gets
    c (w a + (1 - w a) (1 - w) a) with a the unweighted alpha, not c a."""
    raw = scenegen.uniform_scene(n=1, seed=1, lo=-0.01, hi=0.01, ls_mu=-1.0, ls_sd=0.0, sh_degree=0)
    raw.pos[:] = 0.0
    raw.op_logit[:] = 0.5
    sc = ob.build_scene(raw, ob.BuildParams(page_size=4, lod_levels=1, lo=(-1, -1, -1), hi=(1, 1, 1), voxel=0.5,
                                            link_samples=0))
    sc.levels.append({k: v.copy() for k, v in sc.levels[0].items()})
    cam = scenegen.look_at((0, 0, -5), (0, 0, 0), (0, -1, 0), 32, 32, 40.0, (16, 16))
    w = F32(0.3)
    g1, v1 = oracle.gather_draw(sc, [(0, 0, 0, 0)])
    one = oracle.render(g1, v1, cam)
    g2, v2 = oracle.gather_draw(sc, [(0, 1, 0, 0), (0, 0, 1, 0)], [w, F32(1) - w])
    two = oracle.render(g2, v2, cam)
    o = float(sc.levels[0]["opacity"][0, 0])
    a = one["image"] / np.maximum(one["proj"]["rgb"][0][:, None, None], 1e-30)   # unweighted alpha per pixel
    a = np.minimum(a, 0.99)
    wa, wb = float(w) * a, float(F32(1) - w) * a
    expect = one["proj"]["rgb"][0][:, None, None] * (wa + (1 - wa) * wb)
    keep = a * min(float(w), float(F32(1) - w)) >= 1.0 / 255.0      # both items above the skip threshold
    assert keep.sum() > 20 and o > 0.5
    # (the weighted opacities are rounded to float32: relative 6e-8 each)
    np.testing.assert_allclose(two["image"][keep], expect[keep], rtol=1e-6, atol=1e-12)
    # and not the plain sum of the two weights' alphas (the unweighted image)
    assert np.abs(one["image"][keep] - expect[keep]).max() > 1e-3
