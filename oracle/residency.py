"""ORACLE (test infrastructure only): LOD choice, page table and LOD controller.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; it shares no code with the CUDA library.

Follows Sec. 4.1 ("Level of Detail", "Page Table Management") and the
evaluation's "Page determination details":
  * one flat array of physical-page entries, each with its LOD, the frame it
    was last required, and one (virtual page, required) pair per contained
    virtual page (fanout^lod of them);
  * stage one marks required entries and drops requests already resident at
    the requested LOD; entries with nothing required are free and remember
    when they were last used;
  * stage two places the remaining requests, least-recently-used free
    entries first, within the copy budget of the staging buffer;
  * LOD thresholds move to keep usage between 50% and 80%; the step grows by
    1% after successive moves in the same direction and shrinks by 1% after
    a quick reversal.

Readings where the paper is silent, written out as a sequential definition
(all float arithmetic float32, correctly rounded):
  LOD     d = float(0xFFFFFFFF - enc); level = the largest l >= 1 with
          (f_px * e_l(p)) / d <= tau, else 0 (screen-space error in pixels).
  order   unmatched requests by (direct desc, enc desc, page asc).
  budget  the longest prefix of that order whose level-page bytes fit the
          budget; everything after it is missing.
  place   per level, admitted requests first fill non-required sub-slots of
          entries already required this frame at that level (entry asc,
          sub-slot asc); the rest go to fresh entries taken from the free
          list ordered by (last used asc, index asc), levels served in
          ascending order, packed fanout^l per entry; no free entry left ->
          missing.  A fresh entry forgets everything it held.
  draw    stage-one matches plus placements, ascending virtual page.
  usage   drawn Gaussian capacity / (entries * page size).
  fade    (LOD cross-fade, fade_frames F > 0; the blending between levels
          that Sec. 4.1 and 4.3 leave to a renderer with 3DGS alpha blending,
          with both levels resident during the transition): per requested
          page, state (cur = level drawn last frame, from, age); a running
          fade ages by one and ends at age F or when the page returns to
          `from`; a page drawn last frame at cur != its requested level
          starts a fade from cur (age 0).  A fading page also requests
          `from`: stage one keeps that copy required if it is resident (it
          is never copied); it is drawn after the page's own item with
          opacity weight 1 - w and the new level with w = (age+1)/(F+1), in
          float32 (one item alone: weight 1).  Pages not requested forget
          their state.
  control usage > hi: tau += step; usage < lo and a level > 0 drawn:
          tau = max(0, tau - step); before moving, step *= 1.01 when the last
          move (within 10 frames) had the same direction, *= 0.99 when it
          had the opposite one.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

F32 = np.float32


@dataclass
class ResidencyParams:
    n_entries: int
    page_size: int
    levels: int
    fanout: int
    record_bytes: int
    budget_bytes: int
    lod: bool = True
    usage_lo: float = 0.5
    usage_hi: float = 0.8
    tau0: float = 1.0
    step0: float = 0.1
    fade_frames: int = 0

    def m(self, l):
        return self.page_size // (self.fanout ** l)

    def page_bytes(self, l):
        return self.m(l) * self.record_bytes


class PageTable:
    def __init__(self, rp: ResidencyParams):
        self.rp = rp
        smax = rp.fanout ** (rp.levels - 1)
        self.lod = np.full(rp.n_entries, -1, np.int64)
        self.last_used = np.full(rp.n_entries, -1, np.int64)
        self.slot = np.full((rp.n_entries, smax), -1, np.int64)
        self.tau = F32(rp.tau0)
        self.step = F32(rp.step0)
        self.last_dir = 0
        self.last_move = -1000
        self.frame = 0
        self.fade = {}          # page -> [cur, from, age] (cross-fade state)


def float_from_bits(u):
    return np.asarray(u, np.uint32).view(np.float32)


def lod_select(pages, enc, err, f_px, tau, lod_on):
    """Level per request by screen-space error (fp32)."""
    lv = np.zeros(len(pages), np.int64)
    if not lod_on or err.shape[1] <= 1:
        return lv
    d = float_from_bits(np.uint32(0xFFFFFFFF) - np.asarray(enc, np.uint32))
    f = F32(f_px)
    for i, p in enumerate(pages):
        for l in range(err.shape[1] - 1, 0, -1):
            sse = F32(f * err[p, l]) / d[i]
            if sse <= F32(tau):
                lv[i] = l
                break
    return lv


def update(pt: PageTable, pages, enc, direct, levels):
    """One page-table update.  Returns dict with copies [(p,l,e,s)] in
    priority order, draw [(p,l,e,s)] ascending p, missing [p], usage and counts."""
    rp = pt.rp
    P = rp.n_entries
    frame = pt.frame
    req_level = {int(p): int(l) for p, l in zip(pages, levels)}
    # ---- cross-fade state
    F = rp.fade_frames
    fade_level = {}
    if F > 0:
        state = {}
        for p in sorted(req_level):
            l = req_level[p]
            cur, frm, age = pt.fade.get(p, (-1, -1, 0))
            if frm >= 0:
                age += 1
                if age >= F or frm == l:
                    frm = -1
            if cur >= 0 and l != cur:
                frm, age = cur, 0
            state[p] = [cur, frm, age]
            if frm >= 0:
                fade_level[p] = frm
        pt.fade = state
    # ---- stage 1
    required = np.zeros_like(pt.slot, dtype=bool)
    matched = set()
    fade_slot = {}
    for e in range(P):
        l = pt.lod[e]
        if l < 0:
            continue
        for s in range(rp.fanout ** l):
            p = int(pt.slot[e, s])
            if p >= 0 and req_level.get(p, -1) == l:
                required[e, s] = True
                matched.add(p)
            elif p >= 0 and fade_level.get(p, -1) == l:
                required[e, s] = True
                fade_slot[p] = (e, s)
    any_req = required.any(1)
    pt.last_used[any_req] = frame
    # ---- stage 2
    U = [(int(p), int(en), int(d), int(l)) for p, en, d, l in zip(pages, enc, direct, levels) if int(p) not in matched]
    U.sort(key=lambda r: (-r[2], -r[1], r[0]))
    admitted, cum = [], 0
    for r in U:
        c = rp.page_bytes(r[3])
        if cum + c > rp.budget_bytes:
            break
        cum += c
        admitted.append(r)
    missing = [r[0] for r in U[len(admitted):]]
    rank = {r[0]: i for i, r in enumerate(admitted)}
    placed = []
    rest = {}
    for l in range(rp.levels):
        R = [r for r in admitted if r[3] == l]
        O = [(e, s) for e in range(P) if pt.lod[e] == l and any_req[e] for s in range(rp.fanout ** l)
             if not required[e, s]]
        k = min(len(R), len(O))
        for i in range(k):
            e, s = O[i]
            pt.slot[e, s] = R[i][0]
            placed.append((R[i][0], l, e, s))
        rest[l] = R[k:]
    free = sorted([e for e in range(P) if not any_req[e]], key=lambda e: (pt.last_used[e], e))
    fi = 0
    for l in range(rp.levels):
        R = rest[l]
        S = rp.fanout ** l
        for f in range((len(R) + S - 1) // S):
            chunk = R[f * S:(f + 1) * S]
            if fi >= len(free):
                missing.extend(r[0] for r in chunk)
                continue
            e = free[fi]
            fi += 1
            pt.slot[e, :] = -1
            pt.lod[e] = l
            pt.last_used[e] = frame
            for s, r in enumerate(chunk):
                pt.slot[e, s] = r[0]
                placed.append((r[0], l, e, s))
    placed.sort(key=lambda t: rank[t[0]])
    own = [(int(pt.slot[e, s]), int(pt.lod[e]), e, s) for e in range(P) for s in range(rp.fanout ** max(pt.lod[e], 0))
           if pt.lod[e] >= 0 and required[e, s] and req_level.get(int(pt.slot[e, s]), -1) == pt.lod[e]]
    own += placed
    items = [(t, 0) for t in own] + [((p, fade_level[p], e, s), 1) for p, (e, s) in fade_slot.items()]
    items.sort(key=lambda it: (it[0][0], it[1]))
    draw = [t for t, _ in items]
    n_items = {}
    for t in draw:
        n_items[t[0]] = n_items.get(t[0], 0) + 1
    draw_w = []
    for t, k in items:
        w = F32(1)
        if n_items[t[0]] == 2:
            wn = F32(pt.fade[t[0]][2] + 1) / F32(F + 1)
            w = wn if k == 0 else F32(F32(1) - wn)
        draw_w.append(w)
    if F > 0:
        drawn_level = {t[0]: t[1] for t, k in items if k == 0}
        for p in pt.fade:
            pt.fade[p][0] = drawn_level.get(p, -1)
    used = sum(rp.m(t[1]) for t in draw)
    usage = F32(used) / F32(P * rp.page_size) if P > 0 else F32(0)
    streamed_bytes = sum(rp.page_bytes(t[1]) for t in placed)
    return dict(copies=placed, draw=draw, draw_w=draw_w, missing=sorted(missing), usage=usage, resident=len(matched),
                streamed_pages=len(placed), streamed_bytes=streamed_bytes, required=len(pages),
                direct=int(np.sum(np.asarray(direct) != 0)), fading=sum(1 for v in n_items.values() if v == 2))


def control(pt: PageTable, usage, draw):
    """LOD threshold controller, applied after the frame's update; advances the frame."""
    rp = pt.rp
    if rp.lod and rp.levels > 1:
        d = 0
        if usage > F32(rp.usage_hi):
            d = 1
        elif usage < F32(rp.usage_lo) and any(t[1] > 0 for t in draw):
            d = -1
        if d != 0:
            recent = pt.frame - pt.last_move <= 10
            if recent and pt.last_dir == d:
                pt.step = F32(pt.step * F32(1.01))
            elif recent and pt.last_dir == -d:
                pt.step = F32(pt.step * F32(0.99))
            pt.tau = F32(pt.tau + pt.step) if d > 0 else max(F32(0), F32(pt.tau - pt.step))
            pt.last_dir = d
            pt.last_move = pt.frame
    pt.frame += 1


# --------------------------------------------------------------------------- prefetch
def page_centroids(scene):
    """Per page: mean of the level-0 means (FP64, stored fp32) and a radius =
    max over its Gaussians of distance to the mean + 3 x largest scale."""
    L0 = scene.levels[0]
    out = np.zeros((scene.n_pages, 4), np.float32)
    for p in range(scene.n_pages):
        n = int(scene.count[p])
        pos = L0["pos"][p, :n].astype(np.float64)
        c = pos.mean(0) if n else np.zeros(3)
        r = 0.0
        if n:
            d = np.sqrt(((pos - c) ** 2).sum(1)) + 3.0 * L0["scale"][p, :n].astype(np.float64).max(1)
            r = d.max()
        out[p, :3] = c
        out[p, 3] = r
    return out


def prefetch(pt: PageTable, logits, base, threshold, req, err, centroid, campos, f_px, budget_left, frame_now):
    """Placement of predicted pages for the next frame (sequential definition).

    Candidates: window pages p = base + j (j < len(logits), p < n_pages) with
    logit > threshold, not requested this frame, not resident at their level
    (SSE rule with d = max(|campos - centroid| - radius, 0.2) when LOD is on).
    Order (logit desc, level asc, page asc); the longest prefix fitting
    budget_left is admitted; per level in ascending order they take fresh
    entries from those not used this frame (last used < frame_now), least
    recently used first, packed fanout^l per entry.  Returns the copy list
    [(p, l, e, s)] in admitted order."""
    rp = pt.rp
    P = rp.n_entries
    n_vp = len(req)
    resident = set()
    for e in range(P):
        if pt.lod[e] < 0:
            continue
        for s in range(rp.fanout ** pt.lod[e]):
            if pt.slot[e, s] >= 0:
                resident.add((int(pt.slot[e, s]), int(pt.lod[e])))
    F = np.float32
    cands = []
    for j in range(len(logits)):
        p = base + j
        if p >= n_vp:
            continue
        lev = 0
        if rp.lod and rp.levels > 1:
            c = centroid[p]
            dx, dy, dz = F(c[0] - F(campos[0])), F(c[1] - F(campos[1])), F(c[2] - F(campos[2]))
            d = max(F(np.sqrt(F(F(F(dx * dx) + F(dy * dy)) + F(dz * dz))) - c[3]), F(0.2))
            for l in range(rp.levels - 1, 0, -1):
                if F(F(F(f_px) * err[p, l]) / d) <= pt.tau:
                    lev = l
                    break
        if F(logits[j]) > F(threshold) and req[p] == 0 and (p, lev) not in resident:
            cands.append((-float(logits[j]), lev, p))
    cands.sort()
    adm, cum = [], 0
    for c in cands:
        cost = rp.page_bytes(c[1])
        if cum + cost > budget_left:
            break
        cum += cost
        adm.append(c)
    free = sorted([e for e in range(P) if pt.last_used[e] < frame_now], key=lambda e: (pt.last_used[e], e))
    n_l = [sum(1 for c in adm if c[1] == l) for l in range(rp.levels)]
    fresh_start, acc = [], 0
    for l in range(rp.levels):
        fresh_start.append(acc)
        acc += (n_l[l] + rp.fanout ** l - 1) // rp.fanout ** l
    for k in range(min(acc, len(free))):
        e = free[k]
        l = max(i for i in range(rp.levels) if fresh_start[i] <= k and (i + 1 == rp.levels or fresh_start[i + 1] > k))
        pt.slot[e, :] = -1
        pt.lod[e] = l
        pt.last_used[e] = frame_now
    copies, rank = [], [0] * rp.levels
    for (_, l, p) in adm:
        S = rp.fanout ** l
        k = fresh_start[l] + rank[l] // S
        s = rank[l] % S
        rank[l] += 1
        if k < len(free):
            e = free[k]
            pt.slot[e, s] = p
            copies.append((p, l, e, s))
    return copies
