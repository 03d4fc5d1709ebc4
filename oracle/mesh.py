"""ORACLE (test infrastructure only): the paper's mesh proxy (Sec. 3.1 "Mesh
Extraction") and page assignment by nearest face (Sec. 3.2 "Page
Assignment"), written as plain sequential definitions.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; it shares no code with the CUDA library.

Steps, with the readings taken where the paper leaves a choice open:
  occupancy  The scene is sampled on a uniform grid (sample points at voxel
             centres, lo + (i + 1/2) h); a z-slice of the grid is a "scene
             slice" and a sample point is inside when it lies inside the
             kappa-sigma ellipsoid of a Gaussian of opacity >= op_min:
             u = S^-1 R^T (x - mu), |u|^2 <= kappa^2.  The test is an FP32
             formula in a fixed order (occupied() below).  Intersecting the
             ellipsoid with each slice plane (Hartmann's construction,
             Eqs. 1-4) draws exactly these points; the tests pin the two
             against each other.
  closing    Morphological closing (dilation then erosion) with the cube of
             radius r (Chebyshev distance <= r), of the occupancy as a set in
             unbounded empty space (so it only adds sample points).
  surface    The boundary of the closed occupancy, extracted cube by cube
             like Marching Cubes: each cube of 8 neighbouring sample points
             (the grid padded by one empty layer) is cut into the 6
             tetrahedra around its main diagonal (Kuhn), and each
             tetrahedron with inside and outside corners contributes one or
             two triangles whose vertices are the midpoints of its
             inside-outside edges (the level 1/2 of the binary field).
             Vertices live on the half-voxel lattice: integer doubled
             coordinates D (a sample point i has D = 2 i + 1), world position
             lo + D h / 2; triangles face from inside to outside.  The case
             table this implies is generated in code.
  simplify   Quadric error metric (Garland-Heckbert): per-vertex quadrics
             summed from the planes of the incident triangles; the edge of
             least cost is collapsed, the vertex moved to the quadric's
             minimiser (the edge midpoint when the 3x3 system is singular),
             until at most `target` triangles remain.  FP64; ties by edge
             (smaller vertex id, larger vertex id); the kept vertex is the
             smaller id.  Triangles that degenerate are dropped.
  pages      Each Gaussian mean goes to its nearest triangle (FP64 point-
             triangle distance, ties to the lower triangle id).  A triangle
             holding more than page_size means is split at the midpoint of
             its first edge (v0, v1) into (v2, v0, m) and (v1, v2, m) (the
             vertex order rotates, so the next split of a child takes
             another edge), its means going to the child with the nearer
             centroid (ties: the first; means whose nearest point on the
             surface is a vertex could never be separated by nearest
             distance); repeated until none holds more, except that a
             triangle whose splits moved all its means to one child 16 times
             in a row is not split again (means far off the surface on one
             side of it would split it forever).  Triangles with means
             then merge into pages: in ascending triangle order, a page grows
             breadth-first over triangles sharing a vertex (neighbours in
             ascending id) while its count stays within page_size; a triangle
             that would overflow it becomes the base of the next page; when
             no neighbour is left the unassigned triangle nearest (centroid
             distance, ties to the lower id) to the page's base continues it.
             An over-full triangle starts a page of its own and its means fill
             it and the pages after it, in order; those extra pages are linked
             from the triangle's page.  A triangle's page is -1 when it holds
             no mean.
"""
from __future__ import annotations

import heapq
import math

import numpy as np

F32 = np.float32


# --------------------------------------------------------------------------- occupancy
def quat_rot32(q):
    """Rotation matrices [n,3,3] of unit quaternions (w,x,y,z) in FP32, the
    3DGS formula in the projection's operation order."""
    q = np.asarray(q, F32)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    xx, yy, zz = x * x, y * y, z * z
    xy, xz, yz = x * y, x * z, y * z
    wx, wy, wz = w * x, w * y, w * z
    one, two = F32(1), F32(2)
    R = np.empty((len(q), 3, 3), F32)
    R[:, 0, 0] = one - two * (yy + zz); R[:, 0, 1] = two * (xy - wz); R[:, 0, 2] = two * (xz + wy)
    R[:, 1, 0] = two * (xy + wz); R[:, 1, 1] = one - two * (xx + zz); R[:, 1, 2] = two * (yz - wx)
    R[:, 2, 0] = two * (xz - wy); R[:, 2, 1] = two * (yz + wx); R[:, 2, 2] = one - two * (xx + yy)
    return R


def occupied(R, s, mu, x, kappa):
    """FP32: is point x inside the kappa-sigma ellipsoid (R, s, mu)?  d = x - mu;
    w_j = (R_0j d_0 + R_1j d_1) + R_2j d_2; u_j = w_j / s_j;
    (u_0^2 + u_1^2) + u_2^2 <= kappa^2.  Broadcasts over leading axes of x."""
    d = (np.asarray(x, F32) - mu).astype(F32)
    u = []
    for j in range(3):
        wj = (R[0, j] * d[..., 0] + R[1, j] * d[..., 1]) + R[2, j] * d[..., 2]
        u.append(wj / s[j])
    q = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]
    return q <= F32(kappa) * F32(kappa)


def occupancy(pos, scale, rot, opacity, lo, h, dims, kappa, op_min):
    """bool [nz, ny, nx]: sample points inside any Gaussian's ellipsoid."""
    nx, ny, nz = dims
    lo = np.asarray(lo, np.float64)
    occ = np.zeros((nz, ny, nx), bool)
    R = quat_rot32(rot)
    s = np.asarray(scale, F32)
    mu = np.asarray(pos, F32)
    h32 = F32(h)
    lo32 = lo.astype(F32)
    for g in range(len(mu)):
        if not F32(opacity[g]) >= F32(op_min):
            continue
        # a box that holds every sample point the FP32 test can accept
        Sig = (R[g].astype(np.float64) * s[g].astype(np.float64) ** 2) @ R[g].astype(np.float64).T
        ext = float(kappa) * np.sqrt(np.diag(Sig)) * 1.001 + 1e-6
        i0 = np.maximum(np.floor((mu[g] - ext - lo) / h - 0.5).astype(np.int64), 0)
        i1 = np.minimum(np.ceil((mu[g] + ext - lo) / h - 0.5).astype(np.int64), np.array(dims) - 1)
        if np.any(i1 < i0):
            continue
        ix, iy, iz = (np.arange(i0[a], i1[a] + 1) for a in range(3))
        X = np.stack(np.meshgrid(ix, iy, iz, indexing="ij"), -1)
        P = lo32 + (X.astype(F32) + F32(0.5)) * h32
        inside = occupied(R[g], s[g], mu[g], P, kappa)
        sel = X[inside]
        occ[sel[:, 2], sel[:, 1], sel[:, 0]] = True
    return occ


def hartmann_slice_ellipse(mu, R, s, kappa, z0):
    """The ellipse in which the plane z = z0 cuts the kappa-sigma ellipsoid,
    by Hartmann's construction (Eqs. 1-4, FP64).  The ellipsoid's inverse
    translation, rotation and scale take it to the unit sphere; the plane's
    normal becomes m = S R^T e_z / |S R^T e_z| and its distance from the
    centre p = (z0 - mu_z) / |S R^T e_z| (Eq. 1, S = kappa diag(s)).  The
    section is the circle of centre c0 = m p and radius r = sqrt(1 - p^2),
    c = c0 + c1 cos t + c2 sin t, with c1 = r (m_y, -m_x, 0) / |(m_x, m_y)|
    (r (1, 0, 0) when m = e_z) and c2 = m x c1 (Eqs. 2, 3; the printed factor
    in front of c1 is read as the circle's radius, which makes c the section
    circle); the ellipsoid's transformations map it back.  Returns (centre,
    e1, e2) in world coordinates, the ellipse being centre + e1 cos t +
    e2 sin t, or None when the plane misses the ellipsoid."""
    S = np.diag(kappa * np.asarray(s, np.float64))
    R = np.asarray(R, np.float64)
    n = np.array([0.0, 0.0, 1.0])
    sn = S @ R.T @ n
    norm = np.linalg.norm(sn)
    m = sn / norm
    p = (z0 - mu[2]) / norm
    if abs(p) >= 1.0:
        return None
    r = np.sqrt(1.0 - p * p)
    c0 = m * p
    if abs(m[2]) > 1.0 - 1e-12:
        c1 = np.array([r, 0.0, 0.0])
        c2 = np.array([0.0, r, 0.0])
    else:
        c1 = r * np.array([m[1], -m[0], 0.0]) / np.hypot(m[0], m[1])
        c2 = np.cross(m, c1)
    M = R @ S
    return np.asarray(mu, np.float64) + M @ c0, M @ c1, M @ c2


# --------------------------------------------------------------------------- closing
def _box_filter(a, r, op):
    """Separable cube filter of radius r: op = np.logical_or (dilation, outside
    empty) or np.logical_and (erosion, outside empty)."""
    out = a
    for axis in range(3):
        pad = [(0, 0)] * 3
        pad[axis] = (r, r)
        p = np.pad(out, pad, constant_values=False)
        n = out.shape[axis]
        acc = np.take(p, range(0, n), axis=axis)
        for k in range(1, 2 * r + 1):
            acc = op(acc, np.take(p, range(k, k + n), axis=axis))
        out = acc
    return out


def closing(occ, r):
    """Closing of the occupancy as a set in unbounded empty space: the grid
    padded by r empty layers, dilated, eroded, cropped back."""
    if r <= 0:
        return occ.copy()
    p = np.pad(occ, r, constant_values=False)
    c = _box_filter(_box_filter(p, r, np.logical_or), r, np.logical_and)
    return c[r:-r, r:-r, r:-r].copy()


# --------------------------------------------------------------------------- surface
CORNERS = np.array([(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)], np.int64)
# the 6 tetrahedra around the diagonal 0 -> 7: paths 0 -> e_a -> e_a + e_b -> 7
KUHN = []
for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
    c0 = 0
    c1 = c0 | (1 << perm[0])
    c2 = c1 | (1 << perm[1])
    KUHN.append((0, c1, c2, 7))


def _tet_triangles(inside):
    """Triangles (lists of (corner a, corner b) edges) of one tetrahedron
    with the given inside flags of its 4 corners, each edge an inside-outside
    pair; the triangles are oriented later."""
    ins = [k for k in range(4) if inside[k]]
    out = [k for k in range(4) if not inside[k]]
    if len(ins) in (0, 4):
        return []
    if len(ins) == 1:
        a = ins[0]
        return [[(a, b) for b in out]]
    if len(ins) == 3:
        b = out[0]
        return [[(a, b) for a in ins]]
    a0, a1 = ins
    b0, b1 = out
    # the quad a0b0, a0b1, a1b1, a1b0 in cyclic order, as two triangles
    return [[(a0, b0), (a0, b1), (a1, b1)], [(a0, b0), (a1, b1), (a1, b0)]]


def case_table():
    """For each of the 256 inside patterns of a cube's corners, its triangles as
    triples of cube-corner edges (corner a inside, corner b outside), from the
    Kuhn tetrahedra; generated, not stored."""
    table = []
    for case in range(256):
        tris = []
        for tet in KUHN:
            inside = [(case >> c) & 1 for c in tet]
            for t in _tet_triangles(inside):
                tris.append([(tet[a], tet[b]) for (a, b) in t])
        table.append(tris)
    return table


_TABLE = None


def surface(closed):
    """Triangle mesh of the boundary of the closed occupancy [nz, ny, nx]:
    returns (D [nv, 3] int64 doubled lattice coordinates, tris [nt, 3] int64),
    vertices numbered in ascending (Dz, Dy, Dx) order, triangles in cube
    order (z, y, x of the cube's corner 0, padded grid), then table order."""
    global _TABLE
    if _TABLE is None:
        _TABLE = case_table()
    nz, ny, nx = closed.shape
    pad = np.pad(closed, 1, constant_values=False)   # index i_padded = i + 1
    cases = np.zeros((nz + 1, ny + 1, nx + 1), np.int64)
    for c in range(8):
        dx, dy, dz = CORNERS[c]
        cases |= pad[dz:dz + nz + 1, dy:dy + ny + 1, dx:dx + nx + 1].astype(np.int64) << c
    tri_keys = []
    for z, y, x in np.argwhere((cases != 0) & (cases != 255)):
        case = int(cases[z, y, x])
        base = np.array([x - 1, y - 1, z - 1], np.int64)   # sample index of corner 0
        for t in _TABLE[case]:
            vs = []
            for (a, b) in t:
                Da = 2 * (base + CORNERS[a]) + 1
                Db = 2 * (base + CORNERS[b]) + 1
                vs.append((Da + Db) // 2)
            # orient from inside to outside: normal . (outside corner - inside corner) > 0
            (a, b) = t[0]
            dout = CORNERS[b] - CORNERS[a]
            nrm = np.cross(vs[1] - vs[0], vs[2] - vs[0])
            if int(nrm @ dout) < 0:
                vs = [vs[0], vs[2], vs[1]]
            tri_keys.append(vs)
    if not tri_keys:
        return np.zeros((0, 3), np.int64), np.zeros((0, 3), np.int64)
    K = np.array(tri_keys, np.int64).reshape(-1, 3)
    uniq, inv = np.unique(K[:, ::-1], axis=0, return_inverse=True)   # sort by (Dz, Dy, Dx)
    return uniq[:, ::-1].copy(), inv.reshape(-1, 3).astype(np.int64)


# --------------------------------------------------------------------------- simplification
def _plane_quadric(p0, p1, p2):
    """K = q q^T of the triangle's plane q = (n, -n.p0), |n| = 1, as the 10
    distinct entries (a2, ab, ac, ad, b2, bc, bd, c2, cd, d2); zero for a
    degenerate triangle."""
    e1 = (p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2])
    e2 = (p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2])
    nx = e1[1] * e2[2] - e1[2] * e2[1]
    ny = e1[2] * e2[0] - e1[0] * e2[2]
    nz = e1[0] * e2[1] - e1[1] * e2[0]
    ln = math.sqrt((nx * nx + ny * ny) + nz * nz)
    if ln == 0.0:
        return [0.0] * 10
    a, b, c = nx / ln, ny / ln, nz / ln
    d = -((a * p0[0] + b * p0[1]) + c * p0[2])
    return [a * a, a * b, a * c, a * d, b * b, b * c, b * d, c * c, c * d, d * d]


def _qadd(q, r):
    return [q[i] + r[i] for i in range(10)]


def _qeval(q, v):
    """v^T Q v for the homogeneous point (v, 1)."""
    x, y, z = v
    return (((q[0] * x * x + 2.0 * q[1] * x * y) + (2.0 * q[2] * x * z + 2.0 * q[3] * x))
            + ((q[4] * y * y + 2.0 * q[5] * y * z) + 2.0 * q[6] * y)
            + ((q[7] * z * z + 2.0 * q[8] * z) + q[9]))


def _qmin(q, va, vb):
    """The position minimising the quadric (Cramer's rule on its 3x3 system),
    or the midpoint of the edge when the system is (near) singular."""
    a11, a12, a13, a22, a23, a33 = q[0], q[1], q[2], q[4], q[5], q[7]
    b1, b2, b3 = -q[3], -q[6], -q[8]
    det = (a11 * (a22 * a33 - a23 * a23) - a12 * (a12 * a33 - a23 * a13)) + a13 * (a12 * a23 - a22 * a13)
    scale = (abs(a11) + abs(a22)) + abs(a33)
    if not abs(det) > 1e-12 * scale * scale * scale or scale == 0.0:
        return ((va[0] + vb[0]) * 0.5, (va[1] + vb[1]) * 0.5, (va[2] + vb[2]) * 0.5)
    x = (b1 * (a22 * a33 - a23 * a23) - a12 * (b2 * a33 - a23 * b3) + a13 * (b2 * a23 - a22 * b3)) / det
    y = (a11 * (b2 * a33 - a23 * b3) - b1 * (a12 * a33 - a23 * a13) + a13 * (a12 * b3 - b2 * a13)) / det
    z = (a11 * (a22 * b3 - b2 * a23) - a12 * (a12 * b3 - b2 * a13) + b1 * (a12 * a23 - a22 * a13)) / det
    return (x, y, z)


def qem_simplify(verts, tris, target):
    """Garland-Heckbert edge collapse to at most `target` triangles.  verts
    [nv, 3] float64, tris [nt, 3]; returns (verts, tris) compacted (vertex
    order kept, triangles in their original order)."""
    V = [tuple(float(c) for c in v) for v in np.asarray(verts, np.float64)]
    T = [list(map(int, t)) for t in np.asarray(tris)]
    alive_t = [True] * len(T)
    Q = [[0.0] * 10 for _ in V]
    vt = [set() for _ in V]            # vertex -> incident live triangles
    for i, t in enumerate(T):
        k = _plane_quadric(V[t[0]], V[t[1]], V[t[2]])
        for v in t:
            Q[v] = _qadd(Q[v], k)
            vt[v].add(i)
    stamp = [0] * len(V)
    alive_v = [True] * len(V)
    heap = []

    def push(a, b):
        a, b = (a, b) if a < b else (b, a)
        q = _qadd(Q[a], Q[b])
        p = _qmin(q, V[a], V[b])
        heapq.heappush(heap, (_qeval(q, p), a, b, stamp[a], stamp[b], p))

    edges = set()
    for t in T:
        for k in range(3):
            a, b = t[k], t[(k + 1) % 3]
            edges.add((min(a, b), max(a, b)))
    for (a, b) in sorted(edges):
        push(a, b)
    n_live = len(T)
    while n_live > target and heap:
        cost, a, b, sa, sb, p = heapq.heappop(heap)
        if not (alive_v[a] and alive_v[b]) or stamp[a] != sa or stamp[b] != sb:
            continue
        if not (vt[a] & vt[b]) and not any(b in T[i] for i in vt[a]):
            continue   # no longer an edge
        # collapse b into a, at p
        V[a] = p
        Q[a] = _qadd(Q[a], Q[b])
        alive_v[b] = False
        for i in sorted(vt[b]):
            t = T[i]
            if a in t:
                alive_t[i] = False
                n_live -= 1
                for v in t:
                    if v != b:
                        vt[v].discard(i)
            else:
                T[i] = [a if v == b else v for v in t]
                vt[a].add(i)
        vt[b] = set()
        stamp[a] += 1
        nb = set()
        for i in vt[a]:
            nb.update(T[i])
        nb.discard(a)
        for c in sorted(nb):
            push(a, c)
    keep = [i for i in range(len(T)) if alive_t[i]]
    used = sorted({v for i in keep for v in T[i]})
    remap = {v: k for k, v in enumerate(used)}
    nv = np.array([V[v] for v in used], np.float64).reshape(-1, 3)
    nt = np.array([[remap[v] for v in T[i]] for i in keep], np.int64).reshape(-1, 3)
    return nv, nt


# --------------------------------------------------------------------------- pages
def point_triangle_dist2(p, a, b, c):
    """Squared FP64 distance from points p [n,3] to the triangle (a, b, c): the
    closest point by Ericson's region tests (Real-Time Collision Detection,
    closest point on a triangle), in his order: vertex a, vertex b, edge ab,
    vertex c, edge ac, edge bc, interior; a zero-area triangle whose point
    falls through to the interior takes its nearest vertex.  The distance is
    (dx^2 + dy^2) + dz^2."""
    p = np.asarray(p, np.float64)
    a, b, c = (np.asarray(x, np.float64) for x in (a, b, c))
    ab, ac = b - a, c - a
    ap, bp, cp = p - a, p - b, p - c

    def dot(u, v):
        return (u[..., 0] * v[..., 0] + u[..., 1] * v[..., 1]) + u[..., 2] * v[..., 2]

    d1, d2 = dot(ap, ab), dot(ap, ac)
    d3, d4 = dot(bp, ab), dot(bp, ac)
    d5, d6 = dot(cp, ab), dot(cp, ac)
    vc = d1 * d4 - d3 * d2
    vb = d5 * d2 - d1 * d6
    va = d3 * d6 - d5 * d4
    out = np.empty((len(p), 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        den = (va + vb) + vc
        inv = 1.0 / den
        v, w = vb * inv, vc * inv
        out[:] = (a + ab * v[:, None]) + ac * w[:, None]
        z = den == 0
        if np.any(z):
            dd = np.stack([dot(p[z] - q, p[z] - q) for q in (a, b, c)], 1)
            out[z] = np.stack([a, b, c])[np.argmin(dd, 1)]
        # the earlier regions win: applied in reverse order
        m = (va <= 0) & ((d4 - d3) >= 0) & ((d5 - d6) >= 0)
        t = (d4 - d3) / ((d4 - d3) + (d5 - d6))
        out[m] = (b + (c - b) * t[:, None])[m]
        m = (vb <= 0) & (d2 >= 0) & (d6 <= 0)
        t = d2 / (d2 - d6)
        out[m] = (a + ac * t[:, None])[m]
        out[(d6 >= 0) & (d5 <= d6)] = c
        m = (vc <= 0) & (d1 >= 0) & (d3 <= 0)
        t = d1 / (d1 - d3)
        out[m] = (a + ab * t[:, None])[m]
    out[(d3 >= 0) & (d4 <= d3)] = b
    out[(d1 <= 0) & (d2 <= 0)] = a
    e = p - out
    return dot(e, e)


def nearest_triangle(p, verts, tris, chunk=4096):
    """Index of the nearest triangle of each point (ties: lower index)."""
    p = np.asarray(p, np.float64)
    best = np.full(len(p), np.inf)
    arg = np.zeros(len(p), np.int64)
    for t in range(len(tris)):
        a, b, c = verts[tris[t, 0]], verts[tris[t, 1]], verts[tris[t, 2]]
        d = point_triangle_dist2(p, a, b, c)
        better = d < best
        best[better] = d[better]
        arg[better] = t
    return arg


FUTILE_SPLITS = 16   # a chain of splits that separate nothing ends here


def assign_pages(mu, verts, tris, page_size):
    """Nearest-triangle assignment, subdivision and greedy merging.
    Returns dict(verts, tris, face_page [nt] (-1: no page), page_of [n] per
    mean, face_of [n], order [n] means in page order (page, triangle,
    index), counts [n_pages], parent [n_pages]: -1, or for the extra pages of
    an over-full triangle the page that triangle carries)."""
    V = [np.asarray(v, np.float64) for v in verts]
    T = [list(map(int, t)) for t in tris]
    mu = np.asarray(mu, np.float64)
    face = nearest_triangle(mu, np.array(V), np.array(T, np.int64).reshape(-1, 3))
    members = [[] for _ in T]
    for i, f in enumerate(face):
        members[f].append(i)
    fut = [0] * len(T)
    orig = list(range(len(T)))     # the input triangle each one lies in
    queue = [f for f in range(len(T)) if len(members[f]) > page_size]
    qi = 0
    while qi < len(queue):
        f = queue[qi]
        qi += 1
        v0, v1, v2 = T[f]
        m = len(V)
        V.append((V[v0] + V[v1]) * 0.5)
        T[f] = [v2, v0, m]
        T.append([v1, v2, m])
        g = len(T) - 1
        members.append([])
        pts = mu[members[f]]
        # the child of the nearer centroid: means sharing their nearest point
        # on the surface (a vertex) still separate
        c_f = (V[T[f][0]] + V[T[f][1]] + V[T[f][2]]) / 3.0
        c_g = (V[T[g][0]] + V[T[g][1]] + V[T[g][2]]) / 3.0
        d_f = _dist2(pts, c_f)
        d_g = _dist2(pts, c_g)
        old = members[f]
        members[f] = [i for i, a, b in zip(old, d_f, d_g) if a <= b]
        members[g] = [i for i, a, b in zip(old, d_f, d_g) if a > b]
        # splits that move every mean to one child count towards FUTILE_SPLITS
        ff = fut[f] + 1 if not members[g] else 0
        fg = fut[f] + 1 if not members[f] else 0
        fut[f] = ff
        fut.append(fg)
        orig.append(orig[f])
        for h in (f, g):
            if len(members[h]) > page_size and fut[h] < FUTILE_SPLITS:
                queue.append(h)
    nt = len(T)
    cnt = [len(members[f]) for f in range(nt)]
    # triangles sharing a vertex
    vfaces = {}
    for f, t in enumerate(T):
        for v in t:
            vfaces.setdefault(v, []).append(f)
    nbrs = [sorted({g for v in T[f] for g in vfaces[v] if g != f}) for f in range(nt)]
    cen = np.array([(V[t[0]] + V[t[1]] + V[t[2]]) / 3.0 for t in T]).reshape(-1, 3)
    page = [-1] * nt
    todo = [f for f in range(nt) if cnt[f] > 0]
    parent = []
    n_pages = 0
    next_base = None
    ti = 0
    while True:
        if next_base is None:
            while ti < len(todo) and page[todo[ti]] >= 0:
                ti += 1
            if ti == len(todo):
                break
            base = todo[ti]
        else:
            base = next_base
            next_base = None
        pid = n_pages
        n_pages += 1
        parent.append(-1)
        total = 0
        frontier = [base]
        seen = {base}
        while True:
            while frontier:
                f = frontier.pop(0)
                if page[f] >= 0 or cnt[f] == 0:
                    continue
                if total + cnt[f] > page_size and not (total == 0 and cnt[f] > page_size):
                    next_base = f
                    frontier = []
                    break
                page[f] = pid
                total += cnt[f]
                if cnt[f] > page_size:
                    # an over-full triangle: its means fill this page and the next ones
                    extra = (cnt[f] + page_size - 1) // page_size - 1
                    parent.extend([pid] * extra)
                    n_pages += extra
                for g in nbrs[f]:
                    if g not in seen and page[g] < 0:
                        seen.add(g)
                        frontier.append(g)
            if next_base is not None:
                break
            # no neighbour left: the unassigned triangle nearest the base continues the page
            rest = [f for f in todo if page[f] < 0 and f not in seen]
            if not rest:
                break
            d = ((cen[rest] - cen[base]) ** 2).sum(1)
            f = rest[int(np.argmin(d))]
            seen.add(f)
            frontier.append(f)
    face_page = np.array(page, np.int64)
    face_of = _member_face(members, len(mu))
    page_of = np.zeros(len(mu), np.int64)
    for f in range(nt):
        for k, i in enumerate(members[f]):
            page_of[i] = face_page[f] + k // page_size
    order = np.lexsort((np.arange(len(mu)), face_of, page_of))
    counts = np.bincount(page_of, minlength=n_pages)
    return dict(verts=np.array(V), tris=np.array(T, np.int64).reshape(-1, 3), face_page=face_page, page_of=page_of,
                face_of=face_of, order=order, counts=counts, n_pages=n_pages, parent=np.array(parent, np.int64),
                orig=np.array(orig, np.int64))


def _dist2(p, c):
    e = np.asarray(p, np.float64) - c
    return (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]


def _member_face(members, n):
    out = np.zeros(n, np.int64)
    for f, m in enumerate(members):
        out[m] = f
    return out


def mesh_links(mu, R, scale, own_page, vid, verts, tris, face_page, n_pages, n_samples, k_sigma, seed, parent=None):
    """Page links from the mesh (Sec. 3.3 "Page Linking"): K samples per
    Gaussian in its k-sigma ellipsoid (the sampling of the voxel proxy's links,
    link_uniforms), each mapped to its nearest triangle; a triangle whose page
    q differs from the Gaussian's page p gives the link q -> p; the extra
    pages of an over-full triangle are linked from its page (parent).
    Returns the CSR (link_ptr [n_pages + 1], link_col)."""
    from .build import link_uniforms
    lq, lp = [], []
    if n_samples > 0 and len(mu):
        u = link_uniforms(seed, np.asarray(vid, np.int64), n_samples)
        r, th, ph = u[..., 0], 2 * np.pi * u[..., 1], np.pi * u[..., 2]
        e = np.stack([r * np.sin(ph) * np.cos(th), r * np.sin(ph) * np.sin(th), r * np.cos(ph)], -1)
        loc = k_sigma * np.asarray(scale, np.float64)[:, None, :] * e
        x = np.asarray(mu, np.float64)[:, None, :] + np.einsum("gij,gsj->gsi", np.asarray(R, np.float64), loc)
        f = nearest_triangle(x.reshape(-1, 3), verts, tris).reshape(x.shape[:2])
        q = face_page[f]
        own = np.repeat(np.asarray(own_page, np.int64)[:, None], n_samples, 1)
        sel = (q >= 0) & (q != own)
        lq, lp = q[sel], own[sel]
    if parent is not None and np.any(np.asarray(parent) >= 0):
        extra = np.flatnonzero(np.asarray(parent) >= 0)
        lq = np.concatenate([np.asarray(lq, np.int64), np.asarray(parent)[extra]])
        lp = np.concatenate([np.asarray(lp, np.int64), extra])
    if len(lq):
        uniq = np.unique(np.asarray(lq, np.int64) * n_pages + np.asarray(lp, np.int64))
        lq, lp = uniq // n_pages, uniq % n_pages
    else:
        lq = lp = np.zeros(0, np.int64)
    link_ptr = np.zeros(n_pages + 1, np.int64)
    np.add.at(link_ptr, lq + 1, 1)
    return np.cumsum(link_ptr), lp.astype(np.int32)


def mesh_proxy(dec, lo, hi, h, kappa, op_min, closing_r, qem_ratio):
    """Sec. 3.1 end to end: occupancy -> closing -> surface -> simplification;
    returns dict(occ, closed, D, surf_tris, verts, tris)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    dims = tuple(int(np.ceil((hi[a] - lo[a]) / h)) for a in range(3))
    occ = occupancy(dec["pos"], dec["scale"], dec["rot"], dec["opacity"], lo, h, dims, kappa, op_min)
    closed = closing(occ, closing_r)
    D, st = surface(closed)
    pos = lo + D.astype(np.float64) * (0.5 * h)
    target = max(4, int(len(st) * qem_ratio))
    v, t = qem_simplify(pos, st, target) if len(st) else (pos, st)
    return dict(occ=occ, closed=closed, D=D, surf_tris=st, verts=v, tris=t, dims=dims)
