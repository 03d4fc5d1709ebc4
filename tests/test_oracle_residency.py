"""Pins of the page-table / LOD oracle by brute-force simulation invariants
over random request streams, the screen-space-error rule in FP64 and the
controller's band-keeping behaviour."""
import numpy as np
import pytest

from oracle import residency as rs


def _random_stream(rng, n_vp, frames, levels):
    for _ in range(frames):
        k = rng.integers(0, n_vp + 1)
        pages = np.sort(rng.choice(n_vp, size=k, replace=False)).astype(np.int64)
        enc = rng.integers(0x80800000, 0xC0000000, size=k).astype(np.uint32)
        direct = (rng.random(k) < 0.6).astype(np.uint8)
        lv = rng.integers(0, levels, size=k)
        yield pages, enc, direct, lv


@pytest.mark.parametrize("levels,fanout,P,budget_pages", [(1, 8, 10, 4), (3, 8, 6, 3), (4, 2, 12, 6), (2, 4, 3, 100)])
def test_page_table_invariants(levels, fanout, P, budget_pages):
    rng = np.random.default_rng(levels * 100 + P)
    rp = rs.ResidencyParams(n_entries=P, page_size=64, levels=levels, fanout=fanout, record_bytes=56,
                            budget_bytes=budget_pages * 64 * 56)
    pt = rs.PageTable(rp)
    n_vp = 40
    for pages, enc, direct, lv in _random_stream(rng, n_vp, 60, levels):
        before_lru = pt.last_used.copy()
        before_slot = pt.slot.copy()
        before_lod = pt.lod.copy()
        up = rs.update(pt, pages, enc, direct, lv)
        want = {int(p): int(l) for p, l in zip(pages, lv)}
        # every request is drawn at its level or missing, never both
        drawn = {t[0]: t[1] for t in up["draw"]}
        assert set(drawn) | set(up["missing"]) == set(want) and not (set(drawn) & set(up["missing"]))
        assert all(drawn[p] == want[p] for p in drawn)
        assert [t[0] for t in up["draw"]] == sorted(drawn)
        # the table holds what the draw list says
        for (p, l, e, s) in up["draw"]:
            assert pt.slot[e, s] == p and pt.lod[e] == l and s < fanout ** l
        # no virtual page twice at one level anywhere in the table
        seen = set()
        for e in range(P):
            if pt.lod[e] < 0:
                continue
            for s in range(fanout ** pt.lod[e]):
                if pt.slot[e, s] >= 0:
                    key = (int(pt.slot[e, s]), int(pt.lod[e]))
                    assert key not in seen
                    seen.add(key)
        # copies within budget, and only for pages not resident at their level before
        assert up["streamed_bytes"] <= rp.budget_bytes
        for (p, l, e, s) in up["copies"]:
            was = any(before_lod[e2] == l and p in before_slot[e2, :fanout ** l] for e2 in range(P) if before_lod[e2] >= 0)
            assert not was
        # a fresh entry (its LOD changed or it was cleared) was LRU-minimal among the free entries
        req_before = set()
        for (p, l, e, s) in up["draw"]:
            if (p, l, e, s) not in up["copies"]:
                req_before.add(e)
        free = [e for e in range(P) if e not in req_before]
        fresh = {e for (p, l, e, s) in up["copies"] if e not in req_before}
        order = sorted(free, key=lambda e: (before_lru[e], e))
        assert fresh == set(order[:len(fresh)])
        rs.control(pt, up["usage"], up["draw"])


def test_all_requests_fit_means_no_misses_and_second_frame_no_copies():
    rp = rs.ResidencyParams(n_entries=16, page_size=64, levels=1, fanout=8, record_bytes=4, budget_bytes=1 << 30)
    pt = rs.PageTable(rp)
    pages = np.arange(0, 30, 2)
    enc = np.full(len(pages), 0x90000000, np.uint32)
    up = rs.update(pt, pages, enc, np.ones(len(pages), np.uint8), np.zeros(len(pages), int))
    assert up["missing"] == [] and len(up["copies"]) == len(pages)
    rs.control(pt, up["usage"], up["draw"])
    up2 = rs.update(pt, pages, enc, np.ones(len(pages), np.uint8), np.zeros(len(pages), int))
    assert up2["copies"] == [] and up2["resident"] == len(pages)


def test_priority_order_direct_then_nearest():
    """With budget for two pages, direct pages beat linked ones, nearer beat farther."""
    rp = rs.ResidencyParams(n_entries=8, page_size=64, levels=1, fanout=8, record_bytes=4, budget_bytes=2 * 64 * 4)
    pt = rs.PageTable(rp)
    pages = np.array([1, 2, 3, 4])
    enc = np.array([0x90000000, 0xA0000000, 0xB0000000, 0xA0000000], np.uint32)
    direct = np.array([1, 0, 1, 1], np.uint8)
    up = rs.update(pt, pages, enc, direct, np.zeros(4, int))
    assert [c[0] for c in up["copies"]] == [3, 4]
    assert up["missing"] == [1, 2]


def test_lod_select_matches_fp64_screen_space_error():
    rng = np.random.default_rng(2)
    n = 500
    err = np.zeros((n, 3), np.float32)
    err[:, 1] = rng.uniform(0.01, 0.5, n)
    err[:, 2] = err[:, 1] * rng.uniform(1.5, 4, n)
    d = rng.uniform(1, 500, n).astype(np.float32)
    enc = (np.uint32(0xFFFFFFFF) - d.view(np.uint32)).astype(np.uint32)
    f, tau = 960.0, 2.0
    lv = rs.lod_select(np.arange(n), enc, err, f, tau, True)
    for i in range(n):
        sse = [f * float(err[i, l]) / float(d[i]) for l in range(3)]
        ok = [l for l in (1, 2) if sse[l] <= tau]
        want = max(ok) if ok else 0
        near = any(abs(sse[l] - tau) < 1e-5 for l in (1, 2))
        assert lv[i] == want or near
    assert np.all(rs.lod_select(np.arange(n), enc, err, f, tau, False) == 0)


def test_controller_keeps_usage_in_band():
    """A synthetic scene whose usage falls with tau (u = 1.2 / (1 + tau)) is
    driven into the 50-80% band and stays there."""
    rp = rs.ResidencyParams(n_entries=4, page_size=8, levels=2, fanout=2, record_bytes=4, budget_bytes=0)
    pt = rs.PageTable(rp)
    pt.tau = np.float32(0.0)
    hist = []
    for _ in range(400):
        u = np.float32(1.2 / (1.0 + float(pt.tau)))
        rs.control(pt, u, [(0, 1, 0, 0)])
        hist.append(float(u))
    assert all(0.5 - 0.05 <= u <= 0.8 + 0.05 for u in hist[-50:])
    # the step grows on repeated same-direction moves
    pt2 = rs.PageTable(rp)
    for _ in range(5):
        rs.control(pt2, np.float32(0.95), [(0, 1, 0, 0)])
    assert abs(float(pt2.step) - 0.1 * 1.01 ** 4) < 1e-6
    # and shrinks on a quick reversal
    rs.control(pt2, np.float32(0.1), [(0, 1, 0, 0)])
    assert abs(float(pt2.step) - 0.1 * 1.01 ** 4 * 0.99) < 1e-6


# --------------------------------------------------------------------------- prefetch placement
def _resident_pairs(pt):
    out = []
    for e in range(pt.rp.n_entries):
        if pt.lod[e] < 0:
            continue
        for s in range(pt.rp.fanout ** int(pt.lod[e])):
            if pt.slot[e, s] >= 0:
                out.append((int(pt.slot[e, s]), int(pt.lod[e])))
    return out


def _sse_level_fp64(f_px, err_p, centre, campos, tau, levels):
    """The screen-space-error level recomputed in FP64 (d = the distance from
    the camera to the page sphere, at least 0.2); None near a threshold."""
    d = max(float(np.linalg.norm(np.asarray(centre[:3], np.float64) - np.asarray(campos, np.float64)))
            - float(centre[3]), 0.2)
    for l in range(levels - 1, 0, -1):
        sse = f_px * float(err_p[l]) / d
        if abs(sse - float(tau)) < 1e-4 * max(1.0, float(tau)):
            return None
        if sse <= float(tau):
            return l
    return 0


@pytest.mark.parametrize("levels,fanout,P,budget_pages,lod", [(1, 8, 12, 5, False), (3, 8, 10, 4, True),
                                                              (4, 2, 14, 7, True), (2, 4, 6, 50, True)])
def test_prefetch_placement_invariants(levels, fanout, P, budget_pages, lod):
    """Random tables, logits, requests and cameras; every placement checked
    against what the sequential definition promises, each property computed
    here independently: the candidates are the window pages with logit above
    the threshold, not requested, not resident at their (FP64-recomputed)
    level; the copies are the longest prefix of (logit desc, level asc, page
    asc) that fits the budget; fresh entries are the least recently used of
    those not used this frame; entries used this frame are untouched; every
    copied page sits at its level in a slot of its entry; no (page, level) is
    resident twice."""
    rng = np.random.default_rng(1000 * levels + P)
    ps = 64
    rp = rs.ResidencyParams(n_entries=P, page_size=ps, levels=levels, fanout=fanout, record_bytes=56,
                            budget_bytes=budget_pages * ps * 56, lod=lod, tau0=1.5)
    n_vp = 48
    err = np.zeros((n_vp, levels), np.float32)
    for l in range(1, levels):
        err[:, l] = (err[:, l - 1] if l > 1 else 0) + rng.uniform(0.02, 0.3, n_vp).astype(np.float32)
    centroid = np.concatenate([rng.uniform(-20, 20, (n_vp, 3)), rng.uniform(0.5, 3, (n_vp, 1))], 1).astype(np.float32)
    checked = admitted_total = 0
    for it in range(40):
        pt = rs.PageTable(rp)
        # a random earlier history: entries at random levels and ages
        for e in range(P):
            if rng.random() < 0.7:
                l = int(rng.integers(0, levels))
                pt.lod[e] = l
                pt.last_used[e] = int(rng.integers(0, 10))
                for s in range(fanout ** l):
                    if rng.random() < 0.8:
                        pt.slot[e, s] = int(rng.integers(0, n_vp))
        # de-duplicate (page, level) as a real table never holds twice
        seen = set()
        for e in range(P):
            for s in range(fanout ** max(int(pt.lod[e]), 0)):
                k = (int(pt.slot[e, s]), int(pt.lod[e]))
                if pt.slot[e, s] >= 0 and k in seen:
                    pt.slot[e, s] = -1
                seen.add(k)
        frame_now = 10
        pt.tau = np.float32(rng.uniform(0.5, 4.0))
        req = (rng.random(n_vp) < 0.3).astype(np.uint32) * np.uint32(0x90000000)
        base = int(rng.integers(0, 8))
        logits = (rng.integers(-2, 5, size=32) * 0.5).astype(np.float32)  # ties: the tie order matters
        campos = rng.uniform(-25, 25, 3).astype(np.float32)
        f_px = 500.0
        budget_left = int(rng.integers(0, budget_pages + 1)) * ps * 56
        before_lod, before_slot, before_last = pt.lod.copy(), pt.slot.copy(), pt.last_used.copy()
        resident_before = set(_resident_pairs(pt))
        copies = rs.prefetch(pt, logits, base, 0.0, req, err, centroid, campos, f_px, budget_left, frame_now)
        # candidates, recomputed
        cands, ambiguous = [], False
        for j in range(len(logits)):
            p = base + j
            if p >= n_vp or not logits[j] > 0.0 or req[p] != 0:
                continue
            lev = _sse_level_fp64(f_px, err[p], centroid[p], campos, pt.tau, levels) if lod and levels > 1 else 0
            if lev is None:
                ambiguous = True
                continue
            if (p, lev) not in resident_before:
                cands.append((-float(logits[j]), lev, p))
        if ambiguous:
            continue
        checked += 1
        cands.sort()
        adm, cum = [], 0
        for c in cands:
            cost = ps // fanout ** c[1] * 56
            if cum + cost > budget_left:
                break
            cum += cost
            adm.append(c)
        free = sorted([e for e in range(P) if before_last[e] < frame_now], key=lambda e: (before_last[e], e))
        need = sum((sum(1 for c in adm if c[1] == l) + fanout ** l - 1) // fanout ** l for l in range(levels))
        # copies: the admitted prefix in order, as far as fresh entries last
        got = [(p, l) for (p, l, e, s) in copies]
        want = [(c[2], c[1]) for c in adm]
        if need <= len(free):
            assert got == want
        else:
            assert got == [w for w in want if w in set(got)] and len(got) < len(want)
        admitted_total += len(got)
        assert sum(ps // fanout ** l * 56 for (p, l) in got) <= budget_left
        used = {e for (p, l, e, s) in copies}
        assert used <= set(free[:need])
        assert used == set(free[:len(used)]) or need > len(free)
        for e in range(P):
            if before_last[e] >= frame_now:
                assert pt.lod[e] == before_lod[e] and np.array_equal(pt.slot[e], before_slot[e])
        for (p, l, e, s) in copies:
            assert pt.lod[e] == l and pt.slot[e, s] == p and s < fanout ** l and pt.last_used[e] == frame_now
        pairs = _resident_pairs(pt)
        assert len(pairs) == len(set(pairs))
    assert checked >= 30 and admitted_total > 20


def test_page_centroids_closed_form_and_containment():
    """Closed form: a page of eight Gaussians at the corners of a cube of
    half-side h around c with scale s has centroid c and radius
    h sqrt(3) + 3 s.  On a built scene: every Gaussian's 3-sigma ball (its
    mean, 3 x its largest scale) lies inside its page's sphere and touches it
    for at least one Gaussian; the centre is the mean (zero sum of offsets)."""
    import dataclasses
    from _common import tiny_scene
    raw, sc = tiny_scene(links=False)
    h, s, c = 1.25, 0.03, np.array([2.0, -1.0, 0.5])
    corners = np.array([[x, y, z] for x in (-h, h) for y in (-h, h) for z in (-h, h)]) + c
    L0 = dict(sc.levels[0])
    L0["pos"] = L0["pos"].copy()
    L0["scale"] = L0["scale"].copy()
    L0["pos"][0, :8] = corners
    L0["scale"][0, :8] = s
    count = sc.count.copy()
    count[0] = 8
    sc2 = dataclasses.replace(sc, levels=[L0] + list(sc.levels[1:]), count=count)
    cen = rs.page_centroids(sc2)
    np.testing.assert_allclose(cen[0, :3], c, atol=1e-6)
    np.testing.assert_allclose(cen[0, 3], h * np.sqrt(3) + 3 * s, rtol=1e-6)
    cen = rs.page_centroids(sc)
    for p in range(sc.n_pages):
        n = int(sc.count[p])
        pos = sc.levels[0]["pos"][p, :n].astype(np.float64)
        reach = np.linalg.norm(pos - cen[p, :3], axis=1) + 3 * sc.levels[0]["scale"][p, :n].max(1)
        assert reach.max() <= cen[p, 3] * (1 + 1e-6) + 1e-6
        assert reach.max() >= cen[p, 3] * (1 - 1e-6) - 1e-6
        np.testing.assert_allclose((pos - cen[p, :3]).sum(0) / n, 0, atol=1e-5)
