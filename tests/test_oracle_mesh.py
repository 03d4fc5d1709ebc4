"""Pins of the mesh-proxy oracle (Sec. 3.1 Mesh Extraction, Sec. 3.2 Page
Assignment) against closed forms, Hartmann's slice construction, the
algebra of morphology, the topology of closed surfaces and brute force."""
import math

import numpy as np
import pytest

from oracle import mesh as om


def _rand_rot(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def test_occupancy_of_spheres_closed_form():
    """Isotropic Gaussians: a sample point is occupied exactly when it lies
    within kappa * s of a mean (FP64 distance, away from the boundary)."""
    rng = np.random.default_rng(1)
    n, h, kappa = 30, 0.25, 2.0
    pos = rng.uniform(0.5, 3.5, (n, 3)).astype(np.float32)
    s = rng.uniform(0.08, 0.3, n).astype(np.float32)
    scale = np.repeat(s[:, None], 3, 1)
    rot = np.tile(np.array([[1, 0, 0, 0]], np.float32), (n, 1))
    dims = (16, 16, 16)
    occ = om.occupancy(pos, scale, rot, np.ones(n), (0, 0, 0), h, dims, kappa, 0.1)
    z, y, x = np.mgrid[0:16, 0:16, 0:16]
    P = (np.stack([x, y, z], -1) + 0.5) * h
    d = np.sqrt(((P[..., None, :] - pos.astype(np.float64)) ** 2).sum(-1))   # [16,16,16,n]
    r = kappa * s.astype(np.float64)
    inside = (d <= r).any(-1)
    border = (np.abs(d - r) < 1e-4 * r).any(-1)
    assert inside.sum() > 300
    assert np.array_equal(occ[~border], inside[~border])


def test_occupancy_equals_hartmann_slices():
    """Rotated anisotropic Gaussians: in every slice z = z0 of the grid the
    occupied sample points of each Gaussian are those inside the ellipse that
    Hartmann's construction (Eqs. 1-4) gives for that plane (away from the
    ellipse's boundary); the construction's ellipse also lies on the
    ellipsoid's surface (closed form of the quadric)."""
    rng = np.random.default_rng(2)
    h, kappa = 0.1, 2.0
    dims = (40, 40, 40)
    checked = 0
    for g in range(12):
        mu = rng.uniform(1.3, 2.7, 3).astype(np.float32)
        s = rng.uniform(0.1, 0.4, 3).astype(np.float32)
        q = _rand_rot(rng, 1)
        R32 = om.quat_rot32(q)[0]
        occ = om.occupancy(mu[None], s[None], q, np.ones(1), (0, 0, 0), h, dims, kappa, 0.1)
        R = R32.astype(np.float64)
        Sig_inv = R @ np.diag(1.0 / (kappa * s.astype(np.float64)) ** 2) @ R.T
        for k in range(dims[2]):
            z0 = (k + 0.5) * h
            ell = om.hartmann_slice_ellipse(mu.astype(np.float64), R, s, kappa, z0)
            if ell is None:
                assert not occ[k].any()
                continue
            c, e1, e2 = ell
            assert abs(e1[2]) < 1e-12 and abs(e2[2]) < 1e-12 and abs(c[2] - z0) < 1e-9
            for t in np.linspace(0, 2 * np.pi, 7):
                pt = c + e1 * math.cos(t) + e2 * math.sin(t)
                dd = pt - mu.astype(np.float64)
                assert abs(dd @ Sig_inv @ dd - 1.0) < 1e-6  # (R in FP32: orthonormal to about 1e-7)
            M = np.stack([e1[:2], e2[:2]], 1)
            y, x = np.mgrid[0:dims[1], 0:dims[0]]
            P = (np.stack([x, y], -1) + 0.5) * h - c[:2]
            ab = np.linalg.solve(M, P.reshape(-1, 2).T).T
            rr = (ab ** 2).sum(1).reshape(dims[1], dims[0])
            away = np.abs(rr - 1.0) > 1e-4
            assert np.array_equal(occ[k][away], (rr <= 1.0)[away])
            checked += int(away.sum())
    assert checked > 10000


def test_closing_is_extensive_idempotent_and_fills_holes():
    rng = np.random.default_rng(3)
    a = rng.random((12, 14, 16)) < 0.2
    for r in (1, 2):
        c = om.closing(a, r)
        assert np.all(c >= a)
        assert np.array_equal(om.closing(c, r), c)
    block = np.zeros((9, 9, 9), bool)
    block[2:7, 2:7, 2:7] = True
    holed = block.copy()
    holed[4, 4, 4] = False
    assert np.array_equal(om.closing(holed, 1), block)
    assert np.array_equal(om.closing(block, 1), block)


def _edges(tris):
    e = {}
    for t in tris:
        for k in range(3):
            a, b = int(t[k]), int(t[(k + 1) % 3])
            e[(a, b)] = e.get((a, b), 0) + 1
    return e


def _signed_volume(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


@pytest.mark.parametrize("seed", [4, 5])
def test_surface_is_closed_oriented_and_of_genus_zero(seed):
    """The surface of a ball-like set: every directed edge appears once and
    its reverse once (closed and consistently oriented), V - E + F = 2, the
    enclosed volume is positive and lies between the volumes of the inner and
    outer voxel sets; every vertex is the midpoint of an inside and an
    outside sample point."""
    rng = np.random.default_rng(seed)
    n = 14
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    c = np.array([6.5, 6.7, 6.3]) + rng.normal(0, 0.3, 3)
    occ = ((x - c[0]) ** 2 / 25 + (y - c[1]) ** 2 / 16 + (z - c[2]) ** 2 / 20) <= 1.0
    D, T = om.surface(occ)
    e = _edges(T)
    assert all(v == 1 for v in e.values())
    assert all((b, a) in e for (a, b) in e)
    V = D.astype(np.float64) * 0.5   # in voxel units, sample i at i + 1/2
    assert len(D) - len(e) // 2 + len(T) == 2
    vol = _signed_volume(V, T)
    assert 0 < vol and abs(vol - occ.sum()) < 0.5 * (occ.sum() ** (2 / 3)) * 6
    # vertices: D odd on exactly the axes where the two samples agree
    pad = np.pad(occ, 1)
    for d in D[:200]:
        odd = d % 2 == 1
        lo = np.where(odd, (d - 1) // 2, (d - 2) // 2)
        hi = np.where(odd, (d - 1) // 2, d // 2)
        va = pad[lo[2] + 1, lo[1] + 1, lo[0] + 1]
        vb = pad[hi[2] + 1, hi[1] + 1, hi[0] + 1]
        assert va != vb


def test_surface_of_one_voxel_and_case_table():
    """One occupied sample: a closed surface around it (genus 0, positive
    volume below one voxel); the generated case table has no triangles for
    the empty and full cube and is symmetric under complement (same number of
    triangles)."""
    occ = np.zeros((3, 3, 3), bool)
    occ[1, 1, 1] = True
    D, T = om.surface(occ)
    e = _edges(T)
    assert all(v == 1 and (b, a) in e for (a, b), v in e.items())
    assert len(D) - len(e) // 2 + len(T) == 2
    vol = _signed_volume(D.astype(np.float64) * 0.5, T)
    assert 0 < vol < 1
    tab = om.case_table()
    assert tab[0] == [] and tab[255] == []
    assert all(len(tab[c]) == len(tab[255 - c]) for c in range(256))


def test_qem_plane_quadric_is_squared_distance():
    """The quadric of one triangle evaluates to the squared distance of a point
    from the triangle's plane (closed form)."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        p = rng.normal(size=(3, 3))
        q = om._plane_quadric(*[tuple(v) for v in p])
        n = np.cross(p[1] - p[0], p[2] - p[0])
        n /= np.linalg.norm(n)
        x = rng.normal(size=3) * 3
        assert abs(om._qeval(q, tuple(x)) - float(n @ (x - p[0])) ** 2) < 1e-9


def test_qem_keeps_a_plane_planar_and_reaches_the_target():
    """A planar grid of 2 x 12 x 12 triangles simplifies to the target count
    with every vertex still in the plane (all collapse costs are zero) and
    inside the grid's square."""
    k = 12
    xs, ys = np.meshgrid(np.arange(k + 1, dtype=float), np.arange(k + 1, dtype=float), indexing="ij")
    V = np.stack([xs.ravel(), ys.ravel(), np.zeros(xs.size)], 1)
    idx = lambda i, j: i * (k + 1) + j
    T = []
    for i in range(k):
        for j in range(k):
            T.append([idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)])
            T.append([idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)])
    v2, t2 = om.qem_simplify(V, np.array(T), 40)
    assert len(t2) <= 40
    assert np.all(v2[:, 2] == 0.0)
    assert np.all((v2[:, :2] >= 0) & (v2[:, :2] <= k))


def test_qem_on_a_closed_surface_stays_near_it():
    """The surface of a voxel ball simplified to a quarter of its triangles:
    every new vertex stays within a voxel of the original surface."""
    n = 12
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    occ = ((x - 5.5) ** 2 + (y - 5.5) ** 2 + (z - 5.5) ** 2) <= 16
    D, T = om.surface(occ)
    V = D.astype(np.float64) * 0.5
    v2, t2 = om.qem_simplify(V, T, len(T) // 4)
    assert len(t2) <= len(T) // 4
    d = np.sqrt(((v2[:, None, :] - V[None]) ** 2).sum(-1)).min(1)
    assert d.max() < 1.0


def test_point_triangle_distance_against_dense_sampling():
    rng = np.random.default_rng(7)
    s = np.linspace(0, 1, 301)
    uu, vv = np.meshgrid(s, s)
    keep = uu + vv <= 1
    uu, vv = uu[keep], vv[keep]
    for _ in range(10):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=(40, 3)) * 2
        tri = a + np.outer(uu, b - a) + np.outer(vv, c - a)
        brute = ((p[:, None, :] - tri[None]) ** 2).sum(-1).min(1)
        got = om.point_triangle_dist2(p, a, b, c)
        assert np.all(got <= brute + 1e-12)
        assert np.all(brute - got <= 2e-4 * (1 + brute))


def test_page_assignment_partitions_and_respects_page_size():
    """Means around the surface of a voxel ball: every mean in exactly one
    page, its triangle lying inside the triangle nearest to it before the
    subdivision (checked against the distances to every original triangle),
    no triangle and no page above page_size, subdivision keeps the surface's
    area, triangles without means carry no page, and merging makes far fewer
    pages than triangles with means."""
    rng = np.random.default_rng(8)
    n = 10
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    occ = ((x - 4.5) ** 2 + (y - 4.5) ** 2 + (z - 4.5) ** 2) <= 12
    D, T = om.surface(occ)
    V = D.astype(np.float64) * 0.5
    V, T = om.qem_simplify(V, T, len(T) // 3)
    d = rng.normal(size=(3000, 3))
    mu = 5.0 + d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(3.0, 4.6, (3000, 1))
    page_size = 64
    asg = om.assign_pages(mu, V, T, page_size)
    V2, T2, fp = asg["verts"], asg["tris"], asg["face_page"]

    def area(Vv, Tt):
        return 0.5 * np.linalg.norm(np.cross(Vv[Tt[:, 1]] - Vv[Tt[:, 0]], Vv[Tt[:, 2]] - Vv[Tt[:, 0]]), axis=1).sum()
    assert abs(area(V2, T2) - area(V, T)) < 1e-9 * area(V, T)
    face_of = asg["face_of"]
    d2 = np.stack([om.point_triangle_dist2(mu, V[t[0]], V[t[1]], V[t[2]]) for t in T], 1)
    parent = asg["orig"]   # the input triangle a final one lies in
    # (the nearest; equally near triangles sharing an edge may differ in the last bits)
    assert np.all(d2[np.arange(len(mu)), parent[face_of]] <= d2.min(1) * (1 + 1e-12) + 1e-15)
    # every final triangle lies in its input triangle (its vertices do)
    for f in range(len(T2)):
        t = T[parent[f]]
        assert np.all(om.point_triangle_dist2(V2[T2[f]], V[t[0]], V[t[1]], V[t[2]]) < 1e-18)
    per_face = np.bincount(face_of, minlength=len(T2))
    assert per_face.max() <= page_size
    assert np.all((fp >= 0) == (per_face > 0))
    assert np.all(asg["parent"] == -1)
    counts = asg["counts"]
    assert counts.sum() == len(mu) and counts.max() <= page_size
    assert np.array_equal(np.sort(asg["order"]), np.arange(len(mu)))
    assert np.all(np.diff(asg["page_of"][asg["order"]]) >= 0)
    assert asg["n_pages"] <= 2 * math.ceil(len(mu) / page_size) + 4
    assert asg["n_pages"] < (per_face > 0).sum() / 2


def test_build_scene_with_the_mesh_proxy():
    """paging="mesh" end to end on a small blob scene: every Gaussian in one
    page, pages within page_size, triangle pages in range, links valid (CSR,
    sorted, no self-links), LOD levels built, and a feedback frame over the
    mesh requests pages that contain Gaussians in view."""
    import oracle
    import scenegen
    from oracle import build as ob
    from oracle import residency as rs
    raw = scenegen.blob_scene(n=6000, n_blobs=6, lo=0.0, hi=8.0, blob_sigma=0.6, sh_degree=0, seed=9)
    bp = ob.BuildParams(page_size=256, paging="mesh", lod_levels=2, lod_fanout=4, lo=(-2, -2, -2), hi=(10, 10, 10),
                        voxel=0.4, link_samples=2, mesh_kappa=2.0, mesh_op_min=0.1, mesh_closing=1,
                        mesh_qem_ratio=0.3)
    sc = ob.build_scene(raw, bp)
    n = int(sc.count.sum())
    assert n == len(sc.dec_src) and sc.count.max() <= 256
    assert np.array_equal(np.sort(sc.src[sc.src >= 0]), np.arange(n))
    assert sc.face_page.min() >= -1 and sc.face_page.max() < sc.n_pages
    assert len(sc.tris) > 50 and sc.n_pages >= math.ceil(n / 256)
    lp, lc = sc.link_ptr, sc.link_col
    assert lp[0] == 0 and lp[-1] == len(lc) and np.all(np.diff(lp) >= 0)
    for q in range(sc.n_pages):
        row = lc[lp[q]:lp[q + 1]]
        assert np.all(np.diff(row) > 0) and not np.any(row == q)
    cam = scenegen.look_at((4.0, -9.0, 4.0), (4.0, 4.0, 4.0), (0, 0, 1), 160, 120, 60.0)
    pt = rs.PageTable(rs.ResidencyParams(n_entries=sc.n_pages, page_size=256, levels=2, fanout=4, record_bytes=56,
                                         budget_bytes=1 << 40, lod=False))
    out = oracle.frame(sc, pt, cam, ds=4, render_image=False)
    assert len(out["pages"]) > 0 and out["direct"].sum() > 0


def test_over_full_triangle_spills_into_linked_pages():
    """Means far off a small mesh on one side of it: splitting cannot
    separate them (the futile-split limit ends it), so the triangle keeps
    more than page_size means, which fill its page and extra pages whose
    parent is that page; every page stays within page_size."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.float64)
    T = np.array([[0, 1, 2], [1, 3, 2]])
    rng = np.random.default_rng(11)
    mu = np.array([5.0, 5.0, 3.0]) + rng.normal(0, 0.05, (300, 3))
    asg = om.assign_pages(mu, V, T, 64)
    assert asg["counts"].max() <= 64 and asg["counts"].sum() == 300
    par = asg["parent"]
    assert np.any(par >= 0)
    assert all(asg["face_page"][asg["face_page"] >= 0].tolist().count(q) >= 1 for q in set(par[par >= 0]))
    assert np.array_equal(np.sort(asg["order"]), np.arange(300))
