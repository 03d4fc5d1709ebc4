"""ORACLE (test infrastructure only): offline scene preparation in FP64 numpy.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; it shares no code with the CUDA library.

Steps, each following the paper (Sec. 3 "Preprocessing"):
  decode          Sec. 3.5 "Scene Storage": drop normals, decode opacity
                  (sigmoid) and scale (exp), normalise the quaternion, reorder
                  SH coefficient-major, keep only Gaussians inside the scene box.
  morton_pages    Morton order paging (the paper's suggested in-page order,
                  Sec. 5 "cache locality"), consecutive chunks, padded.
  octree_pages    Sec. 3.2 "Page Assignment": greedy merging of neighbouring
                  groups up to, never over, the page size, padding with
                  zero-property Gaussians.  Octree leaves in Morton order
                  stand in for the proxy-mesh faces.
  lod_build       Sec. 3.4 "Level of Detail": only Gaussians of one page merge;
                  each parent merges `fanout` consecutive children by moment
                  matching (mean, covariance), opacity averaged, SH weighted.
  lod_build_kmeans  the paper's own LOD of Sec. 3.4: k-means clusters of a
                  page's Gaussians in a scaled attribute space (position
                  first), each cluster averaged into one parent, the scale
                  enlarged by a fixed factor; `fanout` 2 halves per level.
  voxel_proxy     Sec. 3.1 "Mesh Extraction" stand-in: occupancy grid, one
                  closing, exposed voxel faces merged into rectangles, each
                  face marked with one page.
  links           Sec. 3.3 "Page Linking": random points in each ellipsoid,
                  uniform in spherical coordinates of the unit ball, then
                  scaled, rotated and translated; a sample whose nearest face
                  has another page links that page to the Gaussian's page;
                  unmarked faces take the page with most samples.

Readings where the paper is silent (each restated in the design notes):
quaternion order (w,x,y,z); SH stored [k][c]; Morton with 21 bits per axis
over the scene box; LOD weights opacity x volume; eigenvectors ordered by
descending eigenvalue, the largest-magnitude component of the first two
made positive, the third their cross product; quaternion sign w >= 0;
e_l(p) = largest parent sigma of page p at level l; occupancy = summed
opacity of the means in a voxel >= kappa; ellipsoid extent 2 sigma; the
sample generator is SplitMix64 keyed by (seed, virtual id, sample, axis).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


# --------------------------------------------------------------------------- decode
def decode(raw, lo, hi):
    """Decode raw Kerbl attributes to render-ready fp32 (Sec. 3.5).

    Returns dict of pos[n,3], scale[n,3], rot[n,4] (w,x,y,z unit), opacity[n],
    sh[n,K,3] and `src` (input index) for Gaussians with lo <= pos <= hi."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    p = raw.pos.astype(np.float64)
    keep = np.all((p >= lo) & (p <= hi), axis=1)
    idx = np.nonzero(keep)[0]
    scale = np.exp(raw.log_scale[idx].astype(np.float64)).astype(np.float32)
    q = raw.rot[idx].astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    opac = (1.0 / (1.0 + np.exp(-raw.op_logit[idx].astype(np.float64)))).astype(np.float32)
    K = (raw.sh_degree + 1) ** 2
    sh = np.empty((len(idx), K, 3), np.float32)
    sh[:, 0, :] = raw.f_dc[idx]
    if K > 1:
        sh[:, 1:, :] = np.transpose(raw.f_rest[idx], (0, 2, 1))
    return dict(pos=raw.pos[idx].astype(np.float32), scale=scale, rot=q.astype(np.float32), opacity=opac, sh=sh,
                src=idx.astype(np.int64))


# --------------------------------------------------------------------------- morton
def _spread3(v):
    """Spread the low 21 bits of v so bit b lands at 3b."""
    v = v.astype(np.uint64)
    out = np.zeros_like(v)
    for b in range(21):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton_codes(pos, lo, hi):
    """63-bit Morton code of each position over the box [lo, hi] (FP64 quantisation)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    q = np.floor((pos.astype(np.float64) - lo) / (hi - lo) * float(1 << 21))
    q = np.clip(q, 0, (1 << 21) - 1).astype(np.uint64)
    return _spread3(q[:, 0]) | (_spread3(q[:, 1]) << np.uint64(1)) | (_spread3(q[:, 2]) << np.uint64(2))


def morton_pages(codes, page_size):
    """Stable Morton order, then consecutive chunks of page_size.

    Returns (order, page_start, page_count): order[j] = decoded index at sorted
    position j; page p holds order[page_start[p] : page_start[p] + page_count[p]]."""
    order = np.argsort(codes, kind="stable")
    n = len(order)
    n_pages = (n + page_size - 1) // page_size
    starts = np.arange(n_pages, dtype=np.int64) * page_size
    counts = np.minimum(page_size, n - starts)
    return order, starts, counts


def octree_pages(codes, page_size, max_depth=21):
    """Octree leaves of at most page_size means (split while larger, depth <= 21),
    visited in Morton order, merged greedily: a leaf joins the current page if the
    sum stays <= page_size, else it starts a new page.  Empty leaves are skipped."""
    order = np.argsort(codes, kind="stable")
    sc = codes[order]
    leaves = []

    def rec(s, e, depth):
        if e - s == 0:
            return
        if e - s <= page_size or depth >= max_depth:
            leaves.append((s, e))
            return
        shift = 3 * (max_depth - depth - 1)
        base = (int(sc[s]) >> (shift + 3)) << (shift + 3)
        bounds = [s] + [s + int(np.searchsorted(sc[s:e], np.uint64(base + (c << shift)), side="left"))
                        for c in range(1, 8)] + [e]
        for c in range(8):
            rec(bounds[c], bounds[c + 1], depth + 1)

    rec(0, len(sc), 0)
    starts, counts = [], []
    cur_s, cur_n = None, 0
    for (s, e) in leaves:
        m = e - s
        if cur_s is not None and cur_n + m <= page_size:
            cur_n += m
        else:
            if cur_s is not None:
                starts.append(cur_s)
                counts.append(cur_n)
            cur_s, cur_n = s, m
    if cur_s is not None:
        starts.append(cur_s)
        counts.append(cur_n)
    return order, np.asarray(starts, np.int64), np.asarray(counts, np.int64)


# --------------------------------------------------------------------------- pages
def paged_arrays(dec, order, starts, counts, page_size):
    """Gather decoded Gaussians into [n_pages, page_size] arrays, zero padded."""
    n_pages = len(starts)
    slot = np.arange(page_size)[None, :]
    valid = slot < counts[:, None]
    gidx = np.where(valid, starts[:, None] + slot, 0)
    src = np.where(valid, order[gidx], -1)
    out = {}
    for k in ("pos", "scale", "rot", "opacity", "sh"):
        a = dec[k]
        arr = np.zeros((n_pages, page_size) + a.shape[1:], a.dtype)
        arr[valid] = a[src[valid]]
        out[k] = arr
    out["src"] = src
    out["count"] = counts.copy()
    return out


# --------------------------------------------------------------------------- LOD
def quat_to_rot(q):
    """Rotation matrices of unit quaternions (w,x,y,z), FP64, [..., 3, 3]."""
    q = q.astype(np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def rot_to_quat(R):
    """Unit quaternion (w,x,y,z), w >= 0, of rotation matrices (Shepperd's method)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return _rot_to_quat(np.asarray(R, np.float64))


def _rot_to_quat(R):
    tr = R[..., 0, 0] + R[..., 1, 1] + R[..., 2, 2]
    cands = np.stack([tr, R[..., 0, 0], R[..., 1, 1], R[..., 2, 2]], axis=-1)
    k = np.argmax(cands, axis=-1)
    q = np.empty(R.shape[:-2] + (4,))
    # case 0: w largest
    s = np.sqrt(np.maximum(1 + tr, 0)) * 2
    c0 = np.stack([0.25 * s, (R[..., 2, 1] - R[..., 1, 2]) / s, (R[..., 0, 2] - R[..., 2, 0]) / s,
                   (R[..., 1, 0] - R[..., 0, 1]) / s], -1)
    s1 = np.sqrt(np.maximum(1 + R[..., 0, 0] - R[..., 1, 1] - R[..., 2, 2], 0)) * 2
    c1 = np.stack([(R[..., 2, 1] - R[..., 1, 2]) / s1, 0.25 * s1, (R[..., 0, 1] + R[..., 1, 0]) / s1,
                   (R[..., 0, 2] + R[..., 2, 0]) / s1], -1)
    s2 = np.sqrt(np.maximum(1 + R[..., 1, 1] - R[..., 0, 0] - R[..., 2, 2], 0)) * 2
    c2 = np.stack([(R[..., 0, 2] - R[..., 2, 0]) / s2, (R[..., 0, 1] + R[..., 1, 0]) / s2, 0.25 * s2,
                   (R[..., 1, 2] + R[..., 2, 1]) / s2], -1)
    s3 = np.sqrt(np.maximum(1 + R[..., 2, 2] - R[..., 0, 0] - R[..., 1, 1], 0)) * 2
    c3 = np.stack([(R[..., 1, 0] - R[..., 0, 1]) / s3, (R[..., 0, 2] + R[..., 2, 0]) / s3,
                   (R[..., 1, 2] + R[..., 2, 1]) / s3, 0.25 * s3], -1)
    q = np.where((k == 0)[..., None], c0, np.where((k == 1)[..., None], c1, np.where((k == 2)[..., None], c2, c3)))
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    q = np.where(q[..., :1] < 0, -q, q)
    return q


def merge_moments(pos, scale, rot, opac, sh):
    """Moment-matched merge of groups of children.

    Inputs have a leading group axis and a child axis: pos[G,c,3] ... sh[G,c,K,3].
    Returns the parent Gaussians (fp32) and each parent's largest sigma (fp64).
    A group whose weights sum to zero yields a padding (all-zero) parent."""
    s = scale.astype(np.float64)
    o = opac.astype(np.float64)
    w = o * s[..., 0] * s[..., 1] * s[..., 2]                   # [G,c]
    W = w.sum(-1)                                               # [G]
    real = W > 0
    Ws = np.where(real, W, 1.0)
    mu = (w[..., None] * pos.astype(np.float64)).sum(1) / Ws[:, None]
    R = quat_to_rot(rot)                                        # [G,c,3,3]
    Sig_i = np.einsum("gcik,gck,gcjk->gcij", R, s * s, R)
    d = pos.astype(np.float64) - mu[:, None, :]
    Sig = (w[..., None, None] * (Sig_i + d[..., :, None] * d[..., None, :])).sum(1) / Ws[:, None, None]
    lam, vec = np.linalg.eigh(Sig)                               # ascending
    lam = lam[:, ::-1]
    vec = vec[:, :, ::-1]
    for col in (0, 1):
        v = vec[:, :, col]
        k = np.argmax(np.abs(v), axis=1)
        sgn = np.sign(v[np.arange(len(v)), k])
        sgn[sgn == 0] = 1
        vec[:, :, col] = v * sgn[:, None]
    vec[:, :, 2] = np.cross(vec[:, :, 0], vec[:, :, 1])
    lam = np.maximum(lam, 1e-30)
    p_scale = np.sqrt(lam)
    p_rot = rot_to_quat(vec)
    n_real = (o > 0).sum(-1)
    p_op = np.where(n_real > 0, (o * (o > 0)).sum(-1) / np.maximum(n_real, 1), 0.0)
    p_sh = (w[..., None, None] * sh.astype(np.float64)).sum(1) / Ws[:, None, None]
    z = ~real
    out = dict(pos=mu.astype(np.float32), scale=p_scale.astype(np.float32), rot=p_rot.astype(np.float32),
               opacity=p_op.astype(np.float32), sh=p_sh.astype(np.float32))
    for k in out:
        out[k][z] = 0
    sigma_max = np.where(real, p_scale[:, 0], 0.0)
    return out, sigma_max


def lod_build(pages, levels, fanout):
    """Levels 1..levels-1 of every page: parent j of level l+1 merges children
    fanout*j .. fanout*j+fanout-1 of level l.  Returns list of per-level dicts
    ([n_pages, m_l, ...] arrays) and err[n_pages, levels] (fp32, e_0 = 0)."""
    out = [{k: pages[k] for k in ("pos", "scale", "rot", "opacity", "sh")}]
    n_pages, m = pages["opacity"].shape
    err = np.zeros((n_pages, levels), np.float32)
    for l in range(1, levels):
        prev = out[-1]
        m_prev = prev["opacity"].shape[1]
        m_new = m_prev // fanout
        G = n_pages * m_new
        grp = {k: v.reshape((G, fanout) + v.shape[2:]) for k, v in prev.items()}
        par, smax = merge_moments(grp["pos"], grp["scale"], grp["rot"], grp["opacity"], grp["sh"])
        out.append({k: v.reshape((n_pages, m_new) + v.shape[1:]) for k, v in par.items()})
        err[:, l] = smax.reshape(n_pages, m_new).max(1).astype(np.float32)
    return out, err


# --------------------------------------------------------------------------- k-means LOD
def kmeans_features(pos, rot, opac, sh, attr_weight):
    """Clustering features [n, 11] (fp64) of one page's real Gaussians
    (Sec. 3.4, "Level of Detail": Gaussians are points in attribute space,
    attributes scaled to set their influence, position prioritised).
    Position is centred on the page mean and divided by the page's RMS
    radius (1 where that is 0); then the quaternion with w >= 0, the
    degree-0 SH colour and the opacity, each times attr_weight."""
    p = pos.astype(np.float64)
    n = len(p)
    mu = np.zeros(3)
    for i in range(n):
        mu += p[i]
    mu /= n
    r2 = 0.0
    for i in range(n):
        d = p[i] - mu
        r2 += d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
    rad = np.sqrt(r2 / n)
    if not rad > 0:
        rad = 1.0
    q = rot.astype(np.float64)
    q = np.where(q[:, :1] < 0, -q, q)
    return np.concatenate([(p - mu) / rad, attr_weight * q, attr_weight * sh[:, 0, :].astype(np.float64),
                           attr_weight * opac.astype(np.float64)[:, None]], 1)


def kmeans_lloyd(X, C0, iters):
    """Lloyd's iterations from the given centroids: assign every point to the
    nearest centroid (squared Euclidean distance, lowest index on a tie),
    then move each centroid to the mean of its points (a centroid without
    points stays).  Stops after `iters` rounds or when an assignment repeats
    the previous one (later rounds would change nothing).  Returns the last
    assignment and the centroids after it."""
    C = np.array(C0, np.float64)
    lab, prev = None, None
    for _ in range(iters):
        d = np.zeros((len(X), len(C)))
        for a in range(X.shape[1]):      # features summed in order
            t = X[:, None, a] - C[None, :, a]
            d += t * t
        lab = d.argmin(1)
        if prev is not None and np.array_equal(lab, prev):
            break
        for i in range(len(C)):
            mem = np.nonzero(lab == i)[0]
            if len(mem):
                acc = np.zeros(X.shape[1])
                for j in mem:
                    acc += X[j]
                C[i] = acc / len(mem)
        prev = lab
    return lab, C


def merge_cluster(pos, scale, rot, opac, sh, scale_factor):
    """One merged Gaussian from its members (Sec. 3.4): arithmetic means of
    position, opacity and SH; the quaternions averaged after each is turned
    to the first member's hemisphere, then normalised with w >= 0; the mean
    scale enlarged by the fixed factor when two or more members merge.
    Returns the fp64 attributes."""
    n = len(opac)
    q0 = rot[0].astype(np.float64)
    qs = np.zeros(4)
    for i in range(n):
        q = rot[i].astype(np.float64)
        qs += q if float(q @ q0) >= 0 else -q
    nq = np.sqrt(qs @ qs)
    q = qs / nq if nq > 0 else q0 / np.sqrt(q0 @ q0)
    if q[0] < 0:
        q = -q
    ps, sc, op, shs = np.zeros(3), np.zeros(3), 0.0, np.zeros(sh.shape[1:])
    for i in range(n):                   # members summed in order
        ps += pos[i].astype(np.float64)
        sc += scale[i].astype(np.float64)
        op += float(opac[i])
        shs += sh[i].astype(np.float64)
    sc = sc / n
    if n >= 2:
        sc = sc * scale_factor
    return dict(pos=ps / n, scale=sc, rot=q, opacity=op / n, sh=shs / n)


def lod_build_kmeans(pages, levels, fanout, iters=10, scale_factor=0.0, attr_weight=0.1):
    """Levels 1..levels-1 by k-means clustering inside each page (Sec. 3.4,
    Fig. "LOD generation": the Gaussians per page shrink by `fanout` per
    level, 2 in the paper).  Level l clusters the n real Gaussians of level
    l-1 into k = ceil(n / fanout) clusters seeded at children floor(i*n/k)
    (the page's Morton order), then merges each non-empty cluster into one
    parent; parents fill slots in cluster order, the rest is padding.
    scale_factor 0 means fanout^(1/3) (the volume of `fanout` equal
    Gaussians).  e_l(p) = max over parents and their members of
    |member mean - parent mean| + the member's largest scale.
    Returns the per-level dicts, err[n_pages, levels] (fp32) and the
    assignments labels[l][p] (cluster index per real child, in slot order)."""
    f = scale_factor if scale_factor > 0 else float(fanout) ** (1.0 / 3.0)
    out = [{k: pages[k] for k in ("pos", "scale", "rot", "opacity", "sh")}]
    n_pages, m = pages["opacity"].shape
    err = np.zeros((n_pages, levels), np.float32)
    labels = [None]
    for l in range(1, levels):
        prev = out[-1]
        m_new = prev["opacity"].shape[1] // fanout
        K = prev["sh"].shape[2]
        cur = dict(pos=np.zeros((n_pages, m_new, 3), np.float32), scale=np.zeros((n_pages, m_new, 3), np.float32),
                   rot=np.zeros((n_pages, m_new, 4), np.float32), opacity=np.zeros((n_pages, m_new), np.float32),
                   sh=np.zeros((n_pages, m_new, K, 3), np.float32))
        lab_l = []
        for p in range(n_pages):
            real = np.nonzero(prev["opacity"][p] > 0)[0]
            n = len(real)
            if n == 0:
                lab_l.append(np.zeros(0, np.int64))
                continue
            g = {k: prev[k][p][real] for k in ("pos", "scale", "rot", "opacity", "sh")}
            X = kmeans_features(g["pos"], g["rot"], g["opacity"], g["sh"], attr_weight)
            k = -(-n // fanout)
            C0 = X[[i * n // k for i in range(k)]]
            lab, _ = kmeans_lloyd(X, C0, iters)
            lab_l.append(lab)
            slot, emax = 0, 0.0
            for c in range(k):
                mem = np.nonzero(lab == c)[0]
                if len(mem) == 0:
                    continue
                par = merge_cluster(g["pos"][mem], g["scale"][mem], g["rot"][mem], g["opacity"][mem], g["sh"][mem], f)
                for k2 in cur:
                    cur[k2][p, slot] = par[k2]
                for j in mem:
                    d = g["pos"][j].astype(np.float64) - par["pos"]
                    emax = max(emax, float(np.sqrt(d @ d)) + float(g["scale"][j].astype(np.float64).max()))
                slot += 1
            err[p, l] = np.float32(emax)
        out.append(cur)
        labels.append(lab_l)
    return out, err, labels


# --------------------------------------------------------------------------- splitmix
def splitmix64(x):
    """SplitMix64 output for state x (uint64 numpy array): one 'next' step."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def link_uniforms(seed, vid, n_samples):
    """u[i, j, a] in [0,1): SplitMix64(seed xor ((vid*K + j)*4 + a)), top 53 bits."""
    vid = np.asarray(vid, np.uint64)
    j = np.arange(n_samples, dtype=np.uint64)
    a = np.arange(3, dtype=np.uint64)
    ctr = (vid[:, None, None] * np.uint64(n_samples) + j[None, :, None]) * np.uint64(4) + a[None, None, :]
    x = splitmix64(ctr ^ np.uint64(seed))
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------- proxy
@dataclass
class Grid:
    lo: np.ndarray
    h: float
    dims: tuple

    def index(self, p):
        """Voxel integer coordinates of points and an in-grid mask."""
        c = np.floor((np.asarray(p, np.float64) - self.lo) / self.h).astype(np.int64)
        ok = np.all((c >= 0) & (c < np.asarray(self.dims)), axis=-1)
        return c, ok

    def lin(self, c):
        nx, ny, nz = self.dims
        return (c[..., 2] * ny + c[..., 1]) * nx + c[..., 0]


def _shift_or(mask, fill):
    """3x3x3 neighbourhood OR (fill=False) / AND (fill=True) of a [nz,ny,nx] bool grid."""
    nz, ny, nx = mask.shape
    pad = np.pad(mask, 1, constant_values=fill)
    acc = np.zeros_like(mask) if not fill else np.ones_like(mask)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = pad[dz:dz + nz, dy:dy + ny, dx:dx + nx]
                acc = (acc | sl) if not fill else (acc & sl)
    return acc


def majority(keys, vals):
    """For each distinct key, the most frequent value (ties: smallest value)."""
    if len(keys) == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    pair, cnt = np.unique(np.stack([keys, vals], 1), axis=0, return_counts=True)
    order = np.lexsort((pair[:, 1], -cnt, pair[:, 0]))
    pair = pair[order]
    first = np.ones(len(pair), bool)
    first[1:] = pair[1:, 0] != pair[:-1, 0]
    return pair[first, 0], pair[first, 1]


FACE_DIRS = [(0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)]


def voxel_proxy_and_links(page_pos, page_rot, page_scale, page_op, counts, page_size, lo, hi, h, kappa, closing,
                          n_samples, k_sigma, seed, use_links=True):
    """Voxel proxy (faces carry page ids) and the page-link CSR.

    page_* are [n_pages, page_size, ...] L0 arrays; counts[n_pages] the real
    Gaussians per page.  Returns dict with verts, tris, face_page, link_ptr,
    link_col, and the voxel grid state for inspection."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    dims = tuple(int(np.ceil((hi[a] - lo[a]) / h)) for a in range(3))
    grid = Grid(lo, float(h), dims)
    nx, ny, nz = dims
    n_pages = page_pos.shape[0]
    slot = np.arange(page_size)[None, :]
    valid = slot < counts[:, None]
    pg = np.broadcast_to(np.arange(n_pages)[:, None], valid.shape)[valid]
    vid = (np.arange(n_pages)[:, None] * page_size + slot)[valid].astype(np.int64)
    mu = page_pos[valid].astype(np.float64)
    op = page_op[valid].astype(np.float64)
    c, ok = grid.index(mu)
    lin_mu = grid.lin(c)
    # occupancy: summed opacity of the means in the voxel
    occ_sum = np.zeros(nx * ny * nz)
    np.add.at(occ_sum, lin_mu[ok], op[ok])
    occ = (occ_sum >= kappa).reshape(nz, ny, nx)
    closed = _shift_or(_shift_or(occ, False), True) if closing else occ
    # exposed faces
    cl = np.pad(closed, 1, constant_values=False)
    face_mask = {}
    for (a, s) in FACE_DIRS:
        sh = [0, 0, 0]
        sh[2 - a] = s
        nb = cl[1 + sh[0]:1 + sh[0] + nz, 1 + sh[1]:1 + sh[1] + ny, 1 + sh[2]:1 + sh[2] + nx]
        face_mask[(a, s)] = closed & ~nb
    face_vox = np.zeros_like(closed)
    for m in face_mask.values():
        face_vox |= m
    # voxel pages from the means (majority, ties -> smaller page)
    vpage = np.full(nx * ny * nz, -1, np.int64)
    keys, vals = majority(lin_mu[ok], pg[ok])
    vpage[keys] = vals
    vpage[~closed.reshape(-1)] = -1
    # link samples
    fv = face_vox.reshape(-1)
    pairs_q, pairs_p = [], []
    if n_samples > 0:
        R = quat_to_rot(page_rot[valid])
        sc = page_scale[valid].astype(np.float64)
        chunk = 1 << 18
        cand_all = []
        for s0 in range(0, len(vid), chunk):
            sl = slice(s0, s0 + chunk)
            u = link_uniforms(seed, vid[sl], n_samples)
            r, th, ph = u[..., 0], 2 * np.pi * u[..., 1], np.pi * u[..., 2]
            e = np.stack([r * np.sin(ph) * np.cos(th), r * np.sin(ph) * np.sin(th), r * np.cos(ph)], -1)
            loc = k_sigma * sc[sl][:, None, :] * e
            x = mu[sl][:, None, :] + np.einsum("gij,gsj->gsi", R[sl], loc)
            cand_all.append(_nearest_face_voxel(grid, fv, x))
        cand = np.concatenate(cand_all, 0)               # [n, K] linear voxel or -1
        own = np.repeat(pg[:, None], n_samples, 1)
        has = cand >= 0
        # unmarked face voxels take the page with most samples in them
        unmarked = has & (vpage[np.where(has, cand, 0)] < 0)
        k2, v2 = majority(cand[unmarked], own[unmarked])
        vpage[k2] = v2
        q = np.where(has, vpage[np.where(has, cand, 0)], -1)
        lk = has & (q >= 0) & (q != own)
        pairs_q.append(q[lk])
        pairs_p.append(own[lk])
    # co-located pages in a face voxel are linked from the voxel's page
    fmu = ok & fv[np.where(ok, lin_mu, 0)]
    q2 = vpage[lin_mu[fmu]]
    p2 = pg[fmu]
    sel = (q2 >= 0) & (q2 != p2)
    pairs_q.append(q2[sel])
    pairs_p.append(p2[sel])
    if use_links and pairs_q:
        pq = np.concatenate(pairs_q).astype(np.int64)
        pp = np.concatenate(pairs_p).astype(np.int64)
        if len(pq):
            uniq = np.unique(pq * n_pages + pp)
            lq, lp = uniq // n_pages, uniq % n_pages
        else:
            lq = lp = np.zeros(0, np.int64)
    else:
        lq = lp = np.zeros(0, np.int64)
    link_ptr = np.zeros(n_pages + 1, np.int64)
    np.add.at(link_ptr, lq + 1, 1)
    link_ptr = np.cumsum(link_ptr)
    link_col = lp.astype(np.int32)
    verts, tris, fpage = _greedy_quads(grid, face_mask, vpage.reshape(nz, ny, nx))
    return dict(verts=verts, tris=tris, face_page=fpage, link_ptr=link_ptr, link_col=link_col, grid=grid,
                occ=occ, closed=closed, vpage=vpage)


_NB26 = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                  if not (dx == 0 and dy == 0 and dz == 0)], np.int64)


def _nearest_face_voxel(grid, face_vox_flat, x):
    """Face voxel a sample belongs to: its own voxel if that is a face voxel,
    else the face voxel of the 26-neighbourhood whose centre is nearest
    (ties: smallest linear index), else -1 (also for samples outside the grid)."""
    shp = x.shape[:-1]
    x = x.reshape(-1, 3)
    c, ok = grid.index(x)
    lin = grid.lin(c)
    out = np.full(len(x), -1, np.int64)
    own = ok & face_vox_flat[np.where(ok, lin, 0)]
    out[own] = lin[own]
    rest = np.nonzero(ok & ~own)[0]
    if len(rest):
        cc = c[rest][:, None, :] + _NB26[None, :, :]
        inb = np.all((cc >= 0) & (cc < np.asarray(grid.dims)), -1)
        ll = grid.lin(cc)
        isf = inb & face_vox_flat[np.where(inb, ll, 0)]
        centre = grid.lo + (cc + 0.5) * grid.h
        d2 = ((centre - x[rest][:, None, :]) ** 2).sum(-1)
        d2 = np.where(isf, d2, np.inf)
        big = np.iinfo(np.int64).max
        # nearest centre first, then the smallest linear index
        mind = d2.min(1)
        tie = (d2 == mind[:, None]) & isf
        pick = np.where(tie, ll, big).min(1)
        found = np.isfinite(mind)
        out[rest[found]] = pick[found]
    return out.reshape(shp)


def _greedy_quads(grid, face_mask, vpage):
    """Merge exposed faces of equal page into rectangles, per (axis, side, layer):
    rows of the second in-plane axis outer, first in-plane axis inner; a
    rectangle grows along the first axis, then row by row.  Each rectangle
    becomes two triangles (c00,c10,c11), (c00,c11,c01)."""
    nx, ny, nz = grid.dims
    verts, tris, fpage = [], [], []
    for (a, s) in FACE_DIRS:
        u_ax, w_ax = (a + 1) % 3, (a + 2) % 3
        m = face_mask[(a, s)]                               # [nz,ny,nx]
        mt = np.transpose(m, (2 - a, 2 - w_ax, 2 - u_ax))    # [layer, w, u]
        pt = np.transpose(vpage, (2 - a, 2 - w_ax, 2 - u_ax))
        layers = np.nonzero(mt.reshape(mt.shape[0], -1).any(1))[0]
        for k in layers:
            face = mt[k]
            page = np.where(face, pt[k], -2)
            used = np.zeros_like(face)
            W_, U_ = face.shape
            rows, cols = np.nonzero(face)
            for (w0, u0) in zip(rows, cols):
                if used[w0, u0]:
                    continue
                q = page[w0, u0]
                u1 = u0 + 1
                while u1 < U_ and page[w0, u1] == q and not used[w0, u1]:
                    u1 += 1
                w1 = w0 + 1
                while w1 < W_ and np.all(page[w1, u0:u1] == q) and not used[w1, u0:u1].any():
                    w1 += 1
                used[w0:w1, u0:u1] = True
                plane = grid.lo[a] + grid.h * (k + (1 if s > 0 else 0))
                corners = []
                for (uu, ww) in ((u0, w0), (u1, w0), (u1, w1), (u0, w1)):
                    v = [0.0, 0.0, 0.0]
                    v[a] = plane
                    v[u_ax] = grid.lo[u_ax] + grid.h * uu
                    v[w_ax] = grid.lo[w_ax] + grid.h * ww
                    corners.append(v)
                b = len(verts)
                verts.extend(corners)
                tris.append((b, b + 1, b + 2))
                tris.append((b, b + 2, b + 3))
                fpage.extend([q, q])
    return (np.asarray(verts, np.float64).astype(np.float32).reshape(-1, 3), np.asarray(tris, np.int32).reshape(-1, 3),
            np.asarray(fpage, np.int32))


# --------------------------------------------------------------------------- scene
@dataclass
class BuildParams:
    page_size: int = 256
    paging: str = "morton"          # or "octree"
    lod_levels: int = 1
    lod_fanout: int = 8
    lo: tuple = (-5.0, -5.0, -5.0)
    hi: tuple = (5.0, 5.0, 5.0)
    voxel: float = 10.0 / 32
    kappa: float = 0.5
    closing: bool = True
    link_samples: int = 8
    link_sigma: float = 2.0
    seed: int = 77
    links: bool = True
    lod_method: str = "moment"      # or "kmeans"
    kmeans_iters: int = 10
    kmeans_scale: float = 0.0       # 0: fanout^(1/3)
    kmeans_attr_weight: float = 0.1
    # paging "mesh": the proxy of Sec. 3.1 (ellipsoid slices, closing,
    # surface, QEM) and pages by nearest triangle (Sec. 3.2)
    mesh_kappa: float = 2.0          # ellipsoid of mesh_kappa sigma
    mesh_op_min: float = 0.1         # Gaussians below this opacity do not occupy
    mesh_closing: int = 1            # closing radius in voxels
    mesh_qem_ratio: float = 0.25     # triangles kept by the simplification


@dataclass
class Scene:
    params: BuildParams
    n_pages: int
    levels: list                     # per level dict of [n_pages, m_l, ...] arrays
    err: np.ndarray                  # [n_pages, L] f32
    count: np.ndarray                # [n_pages] real Gaussians at L0
    src: np.ndarray                  # [n_pages, page_size] decoded index (-1 padding)
    dec_src: np.ndarray              # decoded index -> raw input index
    verts: np.ndarray
    tris: np.ndarray
    face_page: np.ndarray
    link_ptr: np.ndarray
    link_col: np.ndarray
    proxy: dict = field(default_factory=dict)

    def m(self, l):
        return self.levels[l]["opacity"].shape[1]


def build_scene(raw, bp: BuildParams) -> Scene:
    dec = decode(raw, bp.lo, bp.hi)
    if bp.paging == "mesh":
        return _build_scene_mesh(dec, bp)
    codes = morton_codes(dec["pos"], bp.lo, bp.hi)
    if bp.paging == "morton":
        order, starts, counts = morton_pages(codes, bp.page_size)
    else:
        order, starts, counts = octree_pages(codes, bp.page_size)
    pages = paged_arrays(dec, order, starts, counts, bp.page_size)
    if bp.lod_method == "kmeans":
        levels, err, _ = lod_build_kmeans(pages, bp.lod_levels, bp.lod_fanout, bp.kmeans_iters, bp.kmeans_scale,
                                          bp.kmeans_attr_weight)
    else:
        levels, err = lod_build(pages, bp.lod_levels, bp.lod_fanout)
    px = voxel_proxy_and_links(pages["pos"], pages["rot"], pages["scale"], pages["opacity"], counts, bp.page_size,
                               bp.lo, bp.hi, bp.voxel, bp.kappa, bp.closing, bp.link_samples, bp.link_sigma,
                               bp.seed, bp.links)
    return Scene(bp, len(starts), levels, err, counts, pages["src"], dec["src"], px["verts"], px["tris"],
                 px["face_page"], px["link_ptr"], px["link_col"], px)


def _build_scene_mesh(dec, bp):
    """Paging "mesh": the proxy of Sec. 3.1, pages by nearest triangle with
    subdivision and merging (Sec. 3.2), links from the mesh (Sec. 3.3), then
    the LOD of the other pagings."""
    from . import mesh as om
    mp = om.mesh_proxy(dec, bp.lo, bp.hi, bp.voxel, bp.mesh_kappa, bp.mesh_op_min, bp.mesh_closing,
                       bp.mesh_qem_ratio)
    asg = om.assign_pages(dec["pos"], mp["verts"], mp["tris"], bp.page_size)
    counts = asg["counts"].astype(np.int64)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    pages = paged_arrays(dec, asg["order"], starts, counts, bp.page_size)
    if bp.lod_method == "kmeans":
        levels, err, _ = lod_build_kmeans(pages, bp.lod_levels, bp.lod_fanout, bp.kmeans_iters, bp.kmeans_scale,
                                          bp.kmeans_attr_weight)
    else:
        levels, err = lod_build(pages, bp.lod_levels, bp.lod_fanout)
    n_pages = len(counts)
    slot = np.arange(bp.page_size)[None, :]
    valid = slot < counts[:, None]
    own = np.broadcast_to(np.arange(n_pages)[:, None], valid.shape)[valid]
    vid = (np.arange(n_pages)[:, None] * bp.page_size + slot)[valid].astype(np.int64)
    R = quat_to_rot(pages["rot"][valid])
    if bp.links:
        link_ptr, link_col = om.mesh_links(pages["pos"][valid], R, pages["scale"][valid], own, vid, asg["verts"],
                                           asg["tris"], asg["face_page"], n_pages, bp.link_samples, bp.link_sigma,
                                           bp.seed, asg["parent"])
    else:
        link_ptr, link_col = np.zeros(n_pages + 1, np.int64), np.zeros(0, np.int32)
    px = dict(mesh=mp, assign=asg)
    return Scene(bp, n_pages, levels, err, counts, pages["src"], dec["src"], asg["verts"].astype(np.float32),
                 asg["tris"].astype(np.int32), asg["face_page"].astype(np.int32), link_ptr, link_col, px)


# --------------------------------------------------------------------------- SH codebook (compressed pages)
def sh_rest(sh):
    """The view-dependent SH coefficients of [..., K, 3] arrays as vectors of
    3 (K - 1) values in (coefficient, channel) order."""
    return sh[..., 1:, :].reshape(sh.shape[:-2] + (3 * (sh.shape[-2] - 1),))


def nearest_code(X, cb):
    """Index of the nearest codeword (squared Euclidean distance in FP64, the
    features summed in order, lowest index on a tie) for every row of X."""
    C = cb.astype(np.float64)
    d = np.zeros((len(X), len(C)))
    for a in range(X.shape[1]):
        t = X[:, None, a] - C[None, :, a]
        d += t * t
    return d.argmin(1)


def quantize_sh(levels, n_codes, iters=10, n_train=65536):
    """Vector quantisation of the view-dependent SH coefficients (bands 1..3)
    into a codebook of n_codes vectors: the compression Sec. 6 leaves to
    future work (codebooks of quantised attributes kept in GPU memory, so
    that pages carry an index instead of the coefficients; the k-means
    quantisation of SH is the related work of Sec. 2, Compression).
      training set  the real (opacity > 0) level-0 Gaussians in slot order;
                    when there are more than n_train, the ones at positions
                    floor(j T / n_train), j < n_train
      codebook      Lloyd's iterations (kmeans_lloyd) from the training
                    vectors at positions floor(j T' / n_codes), rounded to fp32
      codes         every Gaussian of every level (padding included) gets the
                    nearest fp32 codeword (nearest_code)
    Returns (codebook [n_codes, 3 (K - 1)] f32, codes: per level an int32
    array [n_pages, m_l])."""
    L0 = levels[0]
    K = L0["sh"].shape[2]
    if K < 2:
        raise ValueError("SH degree 0: no view-dependent coefficients to quantise")
    X0 = sh_rest(L0["sh"]).reshape(-1, 3 * (K - 1)).astype(np.float64)
    T_all = X0[L0["opacity"].reshape(-1) > 0]
    T = len(T_all)
    nt = min(T, int(n_train))
    if nt < n_codes or n_codes < 1:
        raise ValueError("fewer training Gaussians than codes")
    train = T_all[[j * T // nt for j in range(nt)]]
    _, C = kmeans_lloyd(train, train[[j * nt // n_codes for j in range(n_codes)]], iters)
    cb = C.astype(np.float32)
    codes = []
    for L in levels:
        n_pages, m = L["opacity"].shape
        X = sh_rest(L["sh"]).reshape(-1, 3 * (K - 1)).astype(np.float64)
        codes.append(nearest_code(X, cb).astype(np.int32).reshape(n_pages, m))
    return cb, codes


def vq_levels(levels, cb, codes):
    """The attributes a VQ page record carries, decoded: position and opacity
    fp32; scale, rotation and the SH band 0 rounded to fp16; bands 1..3 the
    Gaussian's codeword."""
    out = []
    for L, c in zip(levels, codes):
        L = dict(L)
        K = L["sh"].shape[2]
        sh = np.empty_like(L["sh"])
        sh[:, :, 0, :] = L["sh"][:, :, 0, :].astype(np.float16).astype(np.float32)
        sh[:, :, 1:, :] = cb[c].reshape(c.shape + (K - 1, 3))
        L["sh"] = sh
        for k in ("scale", "rot"):
            L[k] = L[k].astype(np.float16).astype(np.float32)
        out.append(L)
    return out
