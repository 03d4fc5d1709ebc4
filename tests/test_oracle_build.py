"""Pins of the offline-preparation oracle: the paper's format arithmetic,
brute-force recomputations on tiny inputs and the closed-form moments of a
Gaussian mixture."""
import math
import os
from collections import Counter

import numpy as np

import scenegen
from oracle import build as ob

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_format.txt")


def _golden():
    kv, scenes = {}, []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if len(parts) == 2:
            kv[parts[0]] = float(parts[1])
        else:
            scenes.append((parts[0], int(parts[1]), float(parts[2]), int(parts[3]), int(parts[4]), int(parts[5])))
    return kv, scenes


def test_decoded_record_is_59_floats_and_file_sizes_match_paper():
    kv, scenes = _golden()
    raw = scenegen.uniform_scene(n=10, sh_degree=3)
    d = ob.decode(raw, (-9, -9, -9), (9, 9, 9))
    floats = d["pos"].shape[1] + d["scale"].shape[1] + d["rot"].shape[1] + 1 + d["sh"].shape[1] * d["sh"].shape[2]
    assert floats == kv["record_floats_render"] == kv["record_floats_kerbl"] - 3
    rec = 4 * floats
    assert 4 * kv["record_floats_kerbl"] == kv["record_bytes_kerbl"]
    staging = kv["staging_pages"] * kv["staging_page_size"] * rec / 2 ** 20
    assert abs(staging - kv["staging_mib"]) < 0.05
    for name, pages, mib, ps, levels, fanout in scenes:
        # page sizes of the levels as the LOD builder makes them: ps / fanout^l
        m = [ps // fanout ** l for l in range(levels)]
        size = pages * sum(m) * rec / 2 ** 20
        assert abs(size - mib) < 0.05, (name, size, mib)


def test_decode_properties():
    raw = scenegen.uniform_scene(n=5000, sh_degree=2, seed=3)
    raw.rot *= 3.0   # unnormalised input
    d = ob.decode(raw, (-4, -4, -4), (4, 4, 4))
    inside = np.all((raw.pos >= -4) & (raw.pos <= 4), 1)
    np.testing.assert_array_equal(d["src"], np.nonzero(inside)[0])
    np.testing.assert_allclose(np.linalg.norm(d["rot"].astype(np.float64), axis=1), 1.0, atol=2e-7)
    # opacity is the logistic function: logit(opacity) recovers the input
    o = d["opacity"].astype(np.float64)
    np.testing.assert_allclose(np.log(o / (1 - o)), raw.op_logit[inside], atol=2e-5)
    np.testing.assert_allclose(np.log(d["scale"].astype(np.float64)), raw.log_scale[inside], atol=1e-6)
    # SH reorder: coefficient k of channel c = DC for k=0, else rest[c][k-1]
    i = 7
    src = d["src"][i]
    assert d["sh"][i, 0, 2] == raw.f_dc[src, 2]
    assert d["sh"][i, 5, 1] == raw.f_rest[src, 1, 4]


def _interleave_bruteforce(x, y, z):
    c = 0
    for b in range(21):
        c |= ((x >> b) & 1) << (3 * b)
        c |= ((y >> b) & 1) << (3 * b + 1)
        c |= ((z >> b) & 1) << (3 * b + 2)
    return c


def test_morton_codes_bruteforce():
    rng = np.random.default_rng(0)
    pos = rng.uniform(-5, 5, (200, 3)).astype(np.float32)
    codes = ob.morton_codes(pos, (-5, -5, -5), (5, 5, 5))
    for i in range(200):
        q = [min(max(int(math.floor((float(pos[i, a]) + 5) / 10 * 2 ** 21)), 0), 2 ** 21 - 1) for a in range(3)]
        assert int(codes[i]) == _interleave_bruteforce(*q)


def test_octree_pages_partition_and_greedy_rule():
    raw = scenegen.blob_scene(n=20000, n_blobs=7, sh_degree=0, seed=9)
    d = ob.decode(raw, (-5, -5, -5), (55, 55, 55))
    codes = ob.morton_codes(d["pos"], (-5, -5, -5), (55, 55, 55))
    ps = 512
    order, starts, counts = ob.octree_pages(codes, ps)
    assert counts.max() <= ps and counts.min() > 0
    assert starts[0] == 0 and np.all(starts[1:] == starts[:-1] + counts[:-1]) and starts[-1] + counts[-1] == len(codes)
    assert sorted(order.tolist()) == list(range(len(codes)))
    assert len(starts) >= math.ceil(len(codes) / ps)
    # brute-force leaves: recursive split over explicit prefix tests
    sc = codes[order].astype(object)

    def leaves(idx, depth):
        if len(idx) <= ps:
            return [idx] if len(idx) else []
        shift = 3 * (21 - depth - 1)
        out = []
        for c in range(8):
            out += leaves([i for i in idx if (int(sc[i]) >> shift) & 7 == c], depth + 1)
        return out
    lv = leaves(list(range(len(sc))), 0)
    # greedy: a page never has room for the first leaf of the next page
    sizes = [len(x) for x in lv]
    pages, cur = [], 0
    for s in sizes:
        if cur and cur + s <= ps:
            cur += s
        else:
            if cur:
                pages.append(cur)
            cur = s
    pages.append(cur)
    np.testing.assert_array_equal(counts, pages)


def test_lod_merge_matches_mixture_moments():
    """Mean and covariance of the parent equal the first and second moments of
    the weighted mixture, computed here from raw second moments E[x x^T]."""
    rng = np.random.default_rng(4)
    G, c = 50, 8
    pos = rng.normal(size=(G, c, 3)).astype(np.float32)
    scale = np.exp(rng.normal(-2, 0.5, (G, c, 3))).astype(np.float32)
    q = rng.normal(size=(G, c, 4))
    rot = (q / np.linalg.norm(q, axis=-1, keepdims=True)).astype(np.float32)
    op = rng.uniform(0.05, 1, (G, c)).astype(np.float32)
    op[0, 3:] = 0       # padding children
    op[1] = 0           # all padding -> padding parent
    sh = rng.normal(size=(G, c, 4, 3)).astype(np.float32)
    par, smax = ob.merge_moments(pos, scale, rot, op, sh)
    for g in range(G):
        w = op[g].astype(np.float64) * np.prod(scale[g].astype(np.float64), 1)
        if w.sum() == 0:
            assert np.all(par["opacity"][g] == 0) and np.all(par["scale"][g] == 0)
            continue
        w = w / w.sum()
        m1 = (w[:, None] * pos[g]).sum(0)
        m2 = np.zeros((3, 3))
        for i in range(c):
            qq = rot[g, i].astype(np.float64)
            # rotation from the Hamilton product, independent of quat_to_rot
            def hm(a, b):
                return np.array([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                                 a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                                 a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                                 a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])
            qn = qq / np.linalg.norm(qq)
            R = np.stack([hm(hm(qn, np.r_[0, e]), qn * [1, -1, -1, -1])[1:] for e in np.eye(3)], 1)
            Si = R @ np.diag(scale[g, i].astype(np.float64) ** 2) @ R.T
            m2 += w[i] * (Si + np.outer(pos[g, i], pos[g, i]))
        cov = m2 - np.outer(m1, m1)
        np.testing.assert_allclose(par["pos"][g], m1, rtol=1e-6, atol=1e-6)
        pq = par["rot"][g].astype(np.float64)
        assert abs(np.linalg.norm(pq) - 1) < 1e-6 and pq[0] >= 0
        R = ob.quat_to_rot(pq)
        rec = R @ np.diag(par["scale"][g].astype(np.float64) ** 2) @ R.T
        np.testing.assert_allclose(rec, cov, rtol=2e-5, atol=1e-7 * np.abs(cov).max())
        assert abs(smax[g] - math.sqrt(np.linalg.eigvalsh(cov).max())) < 1e-7 * smax[g]
        real = op[g] > 0
        assert abs(par["opacity"][g] - op[g][real].mean()) < 1e-6


def test_lod_levels_shapes_and_errors():
    raw = scenegen.uniform_scene(n=3000, seed=2, sh_degree=1)
    bp = ob.BuildParams(page_size=256, lod_levels=3, lod_fanout=8, link_samples=0)
    sc = ob.build_scene(raw, bp)
    assert [sc.m(l) for l in range(3)] == [256, 32, 4]
    assert np.all(sc.err[:, 0] == 0) and np.all(sc.err[:, 1:] > 0)
    # a padding page tail gives padding parents (last page is partial)
    last = sc.count[-1]
    assert np.all(sc.levels[1]["opacity"][-1, (last + 7) // 8:] == 0)


def test_splitmix64_published_vector():
    """SplitMix64 seeded with 0: first outputs 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4."""
    out = ob.splitmix64(np.array([0, 0x9E3779B97F4A7C15], np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def _sm_py(x):
    M = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def _tiny_scene(links=True):
    raw = scenegen.uniform_scene(n=600, seed=21, lo=-1.0, hi=1.0, ls_mu=-2.5, sh_degree=0)
    bp = ob.BuildParams(page_size=64, lo=(-1.2, -1.2, -1.2), hi=(1.2, 1.2, 1.2), voxel=0.3, kappa=0.5,
                        link_samples=4, seed=99, links=links)
    return raw, bp, ob.build_scene(raw, bp)


def test_voxel_proxy_bruteforce():
    raw, bp, sc = _tiny_scene()
    px = sc.proxy
    grid = px["grid"]
    nx, ny, nz = grid.dims
    # occupancy recount
    occ = np.zeros((nz, ny, nx))
    pages = sc.levels[0]
    for p in range(sc.n_pages):
        for s in range(sc.count[p]):
            c = [int(math.floor((float(pages["pos"][p, s, a]) - grid.lo[a]) / grid.h)) for a in range(3)]
            if all(0 <= c[a] < grid.dims[a] for a in range(3)):
                occ[c[2], c[1], c[0]] += float(pages["opacity"][p, s])
    np.testing.assert_array_equal(px["occ"], occ >= bp.kappa)
    # closing by explicit loops
    def at(m, z, y, x, fill):
        if 0 <= z < nz and 0 <= y < ny and 0 <= x < nx:
            return m[z, y, x]
        return fill
    dil = np.zeros_like(px["occ"])
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                dil[z, y, x] = any(at(px["occ"], z + a, y + b, x + c, False) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    clo = np.zeros_like(dil)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                clo[z, y, x] = all(at(dil, z + a, y + b, x + c, True) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    np.testing.assert_array_equal(px["closed"], clo)
    assert np.all(px["closed"] | ~px["occ"])      # closing is extensive
    # rasterise the quads back to faces: every exposed face exactly once, with its voxel's page
    faces = Counter()
    for t in range(0, len(sc.tris), 2):
        v = sc.verts[sc.tris[t]].astype(np.float64)
        v4 = sc.verts[sc.tris[t + 1][2]].astype(np.float64)
        quad = np.vstack([v, v4[None]])
        lo_, hi_ = quad.min(0), quad.max(0)
        a = int(np.argmin(hi_ - lo_))
        k = int(round((lo_[a] - grid.lo[a]) / grid.h))
        rng_ = [range(int(round((lo_[b] - grid.lo[b]) / grid.h)), int(round((hi_[b] - grid.lo[b]) / grid.h)))
                for b in range(3)]
        rng_[a] = [k]
        for zz in rng_[2]:
            for yy in rng_[1]:
                for xx in rng_[0]:
                    faces[(a, zz, yy, xx, int(sc.face_page[t]))] += 1
    expect = Counter()
    vp = px["vpage"].reshape(nz, ny, nx)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not clo[z, y, x]:
                    continue
                for a, s in ob.FACE_DIRS:
                    d = [0, 0, 0]
                    d[a] = s
                    if not at(clo, z + d[2], y + d[1], x + d[0], False):
                        c = [x, y, z]
                        c[a] += 1 if s > 0 else 0
                        expect[(a, c[2], c[1], c[0], int(vp[z, y, x]))] += 1
    assert faces == expect


def test_links_bruteforce():
    """Recompute every link with scalar Python: SplitMix64 on Python ints,
    spherical-coordinate samples, 2-sigma ellipsoid, nearest face voxel."""
    raw, bp, sc = _tiny_scene()
    px = sc.proxy
    grid = px["grid"]
    nx, ny, nz = grid.dims
    vp = px["vpage"].copy()
    closed = px["closed"]

    def isface(c):
        x, y, z = c
        if not (0 <= x < nx and 0 <= y < ny and 0 <= z < nz) or not closed[z, y, x]:
            return False
        for a, s in ob.FACE_DIRS:
            d = [0, 0, 0]
            d[a] = s
            xx, yy, zz = x + d[0], y + d[1], z + d[2]
            if not (0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz) or not closed[zz, yy, xx]:
                return True
        return False

    def lin(c):
        return (c[2] * ny + c[1]) * nx + c[0]

    L0 = sc.levels[0]
    links = set()
    for p in range(sc.n_pages):
        for s in range(sc.count[p]):
            vid = p * bp.page_size + s
            mu = L0["pos"][p, s].astype(np.float64)
            R = ob.quat_to_rot(L0["rot"][p, s])
            sc_ = L0["scale"][p, s].astype(np.float64)
            for j in range(bp.link_samples):
                u = [(_sm_py(bp.seed ^ ((vid * bp.link_samples + j) * 4 + a)) >> 11) / 2.0 ** 53 for a in range(3)]
                r, th, ph = u[0], 2 * math.pi * u[1], math.pi * u[2]
                e = np.array([r * math.sin(ph) * math.cos(th), r * math.sin(ph) * math.sin(th), r * math.cos(ph)])
                x = mu + R @ (bp.link_sigma * sc_ * e)
                c = [int(math.floor((x[a] - grid.lo[a]) / grid.h)) for a in range(3)]
                if not all(0 <= c[a] < grid.dims[a] for a in range(3)):
                    continue
                cand = None
                if isface(c):
                    cand = lin(c)
                else:
                    best = None
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                if dx == dy == dz == 0:
                                    continue
                                cc = [c[0] + dx, c[1] + dy, c[2] + dz]
                                if isface(cc):
                                    ctr = grid.lo + (np.array(cc) + 0.5) * grid.h
                                    key = (float(((ctr - x) ** 2).sum()), lin(cc))
                                    if best is None or key < best:
                                        best = key
                    cand = best[1] if best else None
                if cand is not None and vp[cand] >= 0 and vp[cand] != p:
                    links.add((int(vp[cand]), p))
            cvox = [int(math.floor((float(mu[a]) - grid.lo[a]) / grid.h)) for a in range(3)]
            if all(0 <= cvox[a] < grid.dims[a] for a in range(3)) and isface(cvox):
                q = vp[lin(cvox)]
                if q >= 0 and q != p:
                    links.add((int(q), p))
    got = set()
    for q in range(sc.n_pages):
        for k in range(sc.link_ptr[q], sc.link_ptr[q + 1]):
            got.add((q, int(sc.link_col[k])))
    assert got == links and len(got) > 0
    # CSR rows sorted, no duplicates
    for q in range(sc.n_pages):
        row = sc.link_col[sc.link_ptr[q]:sc.link_ptr[q + 1]]
        assert np.all(np.diff(row) > 0)
    # links off: empty CSR, same proxy
    _, _, sc0 = _tiny_scene(links=False)
    assert len(sc0.link_col) == 0 and np.array_equal(sc0.face_page, sc.face_page)
