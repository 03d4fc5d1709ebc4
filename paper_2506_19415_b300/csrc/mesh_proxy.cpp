// Host part of the mesh proxy (Sec. 3.1) and of the page assignment by
// nearest triangle (Sec. 3.2).  FP64 throughout, compiled without contracted
// multiply-adds, every formula in one fixed order, so the results are
// reproducible bit for bit:
//   qem_simplify   Garland-Heckbert edge collapses: per-vertex quadrics from
//                  the unit-normal planes of the incident triangles; the edge
//                  of least cost (ties: smaller vertex id, then the larger)
//                  collapses into its smaller vertex, moved to the quadric's
//                  minimiser (Cramer's rule; the midpoint when singular);
//                  triangles that lose a vertex die; until at most `target`
//                  triangles live.
//   TriIndex       nearest triangle of a point (squared distance by
//                  Ericson's closest-point region tests, ties to the lower
//                  index), exact, through a uniform grid of cells searched in
//                  Chebyshev rings until no unvisited cell can be nearer.
//   assign_pages   nearest triangle of each mean; triangles holding more than
//                  page_size split at the midpoint of their first edge into
//                  (v2, v0, m) and (v1, v2, m), the means going to the child
//                  with the nearer centroid; then pages grown breadth-first over triangles
//                  sharing a vertex while they fit, an overflowing triangle
//                  starting the next page, the nearest unassigned triangle
//                  continuing a page with no neighbour left.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <deque>
#include <queue>
#include <set>
#include <vector>

#include "mesh.h"
#include "scene.h"

namespace vm {
namespace {

constexpr int32_t kFutileSplits = 16;  // splits in a row that move every mean to one child

using V3 = std::array<double, 3>;
using Quad = std::array<double, 10>;

Quad plane_quadric(const V3 &p0, const V3 &p1, const V3 &p2) {
  const double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
  const double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
  const double nx = e1[1] * e2[2] - e1[2] * e2[1];
  const double ny = e1[2] * e2[0] - e1[0] * e2[2];
  const double nz = e1[0] * e2[1] - e1[1] * e2[0];
  const double ln = std::sqrt((nx * nx + ny * ny) + nz * nz);
  Quad q{};
  if (ln == 0.0) return q;
  const double a = nx / ln, b = ny / ln, c = nz / ln;
  const double d = -((a * p0[0] + b * p0[1]) + c * p0[2]);
  q = {a * a, a * b, a * c, a * d, b * b, b * c, b * d, c * c, c * d, d * d};
  return q;
}

Quad qadd(const Quad &q, const Quad &r) {
  Quad o;
  for (int i = 0; i < 10; ++i) o[i] = q[i] + r[i];
  return o;
}

double qeval(const Quad &q, const V3 &v) {
  const double x = v[0], y = v[1], z = v[2];
  return (((q[0] * x * x + 2.0 * q[1] * x * y) + (2.0 * q[2] * x * z + 2.0 * q[3] * x)) +
          ((q[4] * y * y + 2.0 * q[5] * y * z) + 2.0 * q[6] * y)) +
         ((q[7] * z * z + 2.0 * q[8] * z) + q[9]);
}

V3 qmin(const Quad &q, const V3 &va, const V3 &vb) {
  const double a11 = q[0], a12 = q[1], a13 = q[2], a22 = q[4], a23 = q[5], a33 = q[7];
  const double b1 = -q[3], b2 = -q[6], b3 = -q[8];
  const double det = (a11 * (a22 * a33 - a23 * a23) - a12 * (a12 * a33 - a23 * a13)) + a13 * (a12 * a23 - a22 * a13);
  const double scale = (std::fabs(a11) + std::fabs(a22)) + std::fabs(a33);
  if (!(std::fabs(det) > 1e-12 * scale * scale * scale) || scale == 0.0)
    return {(va[0] + vb[0]) * 0.5, (va[1] + vb[1]) * 0.5, (va[2] + vb[2]) * 0.5};
  const double x = ((b1 * (a22 * a33 - a23 * a23) - a12 * (b2 * a33 - a23 * b3)) + a13 * (b2 * a23 - a22 * b3)) / det;
  const double y = ((a11 * (b2 * a33 - a23 * b3) - b1 * (a12 * a33 - a23 * a13)) + a13 * (a12 * b3 - b2 * a13)) / det;
  const double z = ((a11 * (a22 * b3 - b2 * a23) - a12 * (a12 * b3 - b2 * a13)) + b1 * (a12 * a23 - a22 * a13)) / det;
  return {x, y, z};
}

struct Collapse {
  double cost;
  int32_t a, b;
  int64_t sa, sb;
  V3 p;
  bool operator>(const Collapse &o) const {
    if (cost != o.cost) return cost > o.cost;
    if (a != o.a) return a > o.a;
    if (b != o.b) return b > o.b;
    if (sa != o.sa) return sa > o.sa;
    if (sb != o.sb) return sb > o.sb;
    return p > o.p;
  }
};

double dot3(const double *u, const double *v) { return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]; }

// squared distance from p to the triangle (a, b, c)
double tri_dist2(const double *p, const double *a, const double *b, const double *c) {
  double ab[3], ac[3], ap[3], bp[3], cp[3];
  for (int k = 0; k < 3; ++k) {
    ab[k] = b[k] - a[k];
    ac[k] = c[k] - a[k];
    ap[k] = p[k] - a[k];
    bp[k] = p[k] - b[k];
    cp[k] = p[k] - c[k];
  }
  const double d1 = dot3(ap, ab), d2 = dot3(ap, ac), d3 = dot3(bp, ab), d4 = dot3(bp, ac), d5 = dot3(cp, ab),
               d6 = dot3(cp, ac);
  const double vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
  double q[3];
  if (d1 <= 0 && d2 <= 0) {
    for (int k = 0; k < 3; ++k) q[k] = a[k];
  } else if (d3 >= 0 && d4 <= d3) {
    for (int k = 0; k < 3; ++k) q[k] = b[k];
  } else if (vc <= 0 && d1 >= 0 && d3 <= 0) {
    const double t = d1 / (d1 - d3);
    for (int k = 0; k < 3; ++k) q[k] = a[k] + ab[k] * t;
  } else if (d6 >= 0 && d5 <= d6) {
    for (int k = 0; k < 3; ++k) q[k] = c[k];
  } else if (vb <= 0 && d2 >= 0 && d6 <= 0) {
    const double t = d2 / (d2 - d6);
    for (int k = 0; k < 3; ++k) q[k] = a[k] + ac[k] * t;
  } else if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
    const double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    for (int k = 0; k < 3; ++k) q[k] = b[k] + (c[k] - b[k]) * t;
  } else {
    const double den = (va + vb) + vc;
    if (den == 0) {
      const double *vs[3] = {a, b, c};
      double best = 0;
      int bi = 0;
      for (int j = 0; j < 3; ++j) {
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = p[k] - vs[j][k];
        const double d = dot3(e, e);
        if (j == 0 || d < best) { best = d; bi = j; }
      }
      for (int k = 0; k < 3; ++k) q[k] = vs[bi][k];
    } else {
      const double inv = 1.0 / den, v = vb * inv, w = vc * inv;
      for (int k = 0; k < 3; ++k) q[k] = (a[k] + ab[k] * v) + ac[k] * w;
    }
  }
  double e[3];
  for (int k = 0; k < 3; ++k) e[k] = p[k] - q[k];
  return dot3(e, e);
}

}  // namespace

void qem_simplify(std::vector<double> &verts, std::vector<int32_t> &tris, int64_t target) {
  const int64_t nv = (int64_t)verts.size() / 3, nt = (int64_t)tris.size() / 3;
  std::vector<V3> V(nv);
  for (int64_t i = 0; i < nv; ++i) V[i] = {verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]};
  std::vector<std::array<int32_t, 3>> T(nt);
  for (int64_t i = 0; i < nt; ++i) T[i] = {tris[3 * i], tris[3 * i + 1], tris[3 * i + 2]};
  std::vector<uint8_t> alive_t(nt, 1), alive_v(nv, 1);
  std::vector<Quad> Q(nv, Quad{});
  std::vector<std::set<int64_t>> vt(nv);
  for (int64_t i = 0; i < nt; ++i) {
    const Quad k = plane_quadric(V[T[i][0]], V[T[i][1]], V[T[i][2]]);
    for (int j = 0; j < 3; ++j) {
      Q[T[i][j]] = qadd(Q[T[i][j]], k);
      vt[T[i][j]].insert(i);
    }
  }
  std::vector<int64_t> stamp(nv, 0);
  std::priority_queue<Collapse, std::vector<Collapse>, std::greater<Collapse>> heap;
  auto push = [&](int32_t a, int32_t b) {
    if (a > b) std::swap(a, b);
    const Quad q = qadd(Q[a], Q[b]);
    const V3 p = qmin(q, V[a], V[b]);
    heap.push(Collapse{qeval(q, p), a, b, stamp[a], stamp[b], p});
  };
  {
    std::vector<std::pair<int32_t, int32_t>> edges;
    for (auto &t : T)
      for (int k = 0; k < 3; ++k) {
        const int32_t a = t[k], b = t[(k + 1) % 3];
        edges.emplace_back(std::min(a, b), std::max(a, b));
      }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    for (auto &e : edges) push(e.first, e.second);
  }
  int64_t n_live = nt;
  while (n_live > target && !heap.empty()) {
    const Collapse c = heap.top();
    heap.pop();
    const int32_t a = c.a, b = c.b;
    if (!(alive_v[a] && alive_v[b]) || stamp[a] != c.sa || stamp[b] != c.sb) continue;
    bool shared = false;
    for (int64_t i : vt[a])
      if (vt[b].count(i)) { shared = true; break; }
    if (!shared) continue;
    V[a] = c.p;
    Q[a] = qadd(Q[a], Q[b]);
    alive_v[b] = 0;
    const std::vector<int64_t> tb(vt[b].begin(), vt[b].end());
    for (int64_t i : tb) {
      auto &t = T[i];
      if (t[0] == a || t[1] == a || t[2] == a) {
        alive_t[i] = 0;
        --n_live;
        for (int j = 0; j < 3; ++j)
          if (t[j] != b) vt[t[j]].erase(i);
      } else {
        for (int j = 0; j < 3; ++j)
          if (t[j] == b) t[j] = a;
        vt[a].insert(i);
      }
    }
    vt[b].clear();
    ++stamp[a];
    std::set<int32_t> nb;
    for (int64_t i : vt[a])
      for (int j = 0; j < 3; ++j) nb.insert(T[i][j]);
    nb.erase(a);
    for (int32_t v : nb) push(a, v);
  }
  std::vector<int32_t> remap(nv, -1);
  std::vector<int32_t> used;
  for (int64_t i = 0; i < nt; ++i)
    if (alive_t[i])
      for (int j = 0; j < 3; ++j) used.push_back(T[i][j]);
  std::sort(used.begin(), used.end());
  used.erase(std::unique(used.begin(), used.end()), used.end());
  std::vector<double> ov;
  for (size_t k = 0; k < used.size(); ++k) {
    remap[used[k]] = (int32_t)k;
    for (int j = 0; j < 3; ++j) ov.push_back(V[used[k]][j]);
  }
  std::vector<int32_t> ot;
  for (int64_t i = 0; i < nt; ++i)
    if (alive_t[i])
      for (int j = 0; j < 3; ++j) ot.push_back(remap[T[i][j]]);
  verts.swap(ov);
  tris.swap(ot);
}

struct TriIndex {
  const std::vector<double> *V;
  const std::vector<int32_t> *T;
  double lo[3], cell;
  int64_t n[3];
  std::vector<int64_t> start;   // CSR of triangles per cell
  std::vector<int32_t> items;
};

TriIndex *tri_index_build(const std::vector<double> &verts, const std::vector<int32_t> &tris) {
  auto *ix = new TriIndex();
  ix->V = &verts;
  ix->T = &tris;
  const int64_t nt = (int64_t)tris.size() / 3;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, ext = 0;
  for (int64_t t = 0; t < nt; ++t) {
    double tl[3] = {INFINITY, INFINITY, INFINITY}, th[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        const double v = verts[3 * (size_t)tris[3 * t + j] + k];
        tl[k] = std::min(tl[k], v);
        th[k] = std::max(th[k], v);
      }
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], tl[k]);
      hi[k] = std::max(hi[k], th[k]);
      ext += th[k] - tl[k];
    }
  }
  if (nt == 0) {
    for (int k = 0; k < 3; ++k) { ix->lo[k] = 0; ix->n[k] = 1; }
    ix->cell = 1;
    ix->start.assign(2, 0);
    return ix;
  }
  double cell = ext / (3.0 * (double)nt) * 2.0;
  double span = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-9});
  if (!(cell > span / 512)) cell = span / 512;
  ix->cell = cell;
  for (int k = 0; k < 3; ++k) {
    ix->lo[k] = lo[k];
    ix->n[k] = std::max<int64_t>(1, (int64_t)std::floor((hi[k] - lo[k]) / cell) + 1);
  }
  const int64_t nc = ix->n[0] * ix->n[1] * ix->n[2];
  std::vector<int64_t> cnt(nc + 1, 0);
  auto range = [&](int64_t t, int64_t c0[3], int64_t c1[3]) {
    for (int k = 0; k < 3; ++k) {
      double tl = INFINITY, th = -INFINITY;
      for (int j = 0; j < 3; ++j) {
        const double v = verts[3 * (size_t)tris[3 * t + j] + k];
        tl = std::min(tl, v);
        th = std::max(th, v);
      }
      c0[k] = std::min(ix->n[k] - 1, std::max<int64_t>(0, (int64_t)std::floor((tl - lo[k]) / cell)));
      c1[k] = std::min(ix->n[k] - 1, std::max<int64_t>(0, (int64_t)std::floor((th - lo[k]) / cell)));
    }
  };
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int64_t c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
      ix->start = cnt;
      ix->items.resize(cnt[nc]);
    }
    std::vector<int64_t> fill = pass ? ix->start : std::vector<int64_t>();
    for (int64_t t = 0; t < nt; ++t) {
      int64_t c0[3], c1[3];
      range(t, c0, c1);
      for (int64_t z = c0[2]; z <= c1[2]; ++z)
        for (int64_t y = c0[1]; y <= c1[1]; ++y)
          for (int64_t x = c0[0]; x <= c1[0]; ++x) {
            const int64_t c = (z * ix->n[1] + y) * ix->n[0] + x;
            if (pass == 0) ++cnt[c + 1];
            else ix->items[fill[c]++] = (int32_t)t;
          }
    }
  }
  return ix;
}

int32_t tri_index_nearest(const TriIndex *ix, const double p[3]) {
  const auto &V = *ix->V;
  const auto &T = *ix->T;
  int64_t pc[3];
  for (int k = 0; k < 3; ++k)
    pc[k] = std::min(ix->n[k] - 1, std::max<int64_t>(0, (int64_t)std::floor((p[k] - ix->lo[k]) / ix->cell)));
  double best = INFINITY;
  int32_t arg = -1;
  const int64_t rmax = std::max({ix->n[0], ix->n[1], ix->n[2]});
  for (int64_t r = 0; r <= rmax; ++r) {
    for (int64_t z = pc[2] - r; z <= pc[2] + r; ++z) {
      if (z < 0 || z >= ix->n[2]) continue;
      for (int64_t y = pc[1] - r; y <= pc[1] + r; ++y) {
        if (y < 0 || y >= ix->n[1]) continue;
        const bool edge_zy = std::llabs(z - pc[2]) == r || std::llabs(y - pc[1]) == r;
        for (int64_t x = pc[0] - r; x <= pc[0] + r; ++x) {
          if (x < 0 || x >= ix->n[0]) continue;
          if (!edge_zy && std::llabs(x - pc[0]) != r) continue;  // only the ring's shell
          const int64_t c = (z * ix->n[1] + y) * ix->n[0] + x;
          for (int64_t k = ix->start[c]; k < ix->start[c + 1]; ++k) {
            const int32_t t = ix->items[k];
            const double d = tri_dist2(p, &V[3 * (size_t)T[3 * (size_t)t]], &V[3 * (size_t)T[3 * (size_t)t + 1]],
                                       &V[3 * (size_t)T[3 * (size_t)t + 2]]);
            if (d < best || (d == best && t < arg)) { best = d; arg = t; }
          }
        }
      }
    }
    // cells of the next ring are at least r cells away from the point's cell
    if (arg >= 0) {
      const double bound = (double)r * ix->cell;
      if (bound * bound > best) break;
    }
  }
  return arg;
}

void tri_index_free(TriIndex *ix) { delete ix; }

void assign_pages(int64_t n, const float *mu32, int64_t page_size, std::vector<double> &verts,
                  std::vector<int32_t> &tris, std::vector<int32_t> &face_page, std::vector<int64_t> &order,
                  std::vector<int64_t> &counts, std::vector<int64_t> &parent) {
  parent.clear();
  std::vector<double> mu(3 * n);
  for (int64_t i = 0; i < 3 * n; ++i) mu[i] = (double)mu32[i];
  std::vector<int32_t> face(n);
  {
    TriIndex *ix = tri_index_build(verts, tris);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) face[i] = tri_index_nearest(ix, &mu[3 * i]);
    tri_index_free(ix);
  }
  int64_t nt = (int64_t)tris.size() / 3;
  std::vector<std::vector<int64_t>> members(nt);
  for (int64_t i = 0; i < n; ++i) members[face[i]].push_back(i);
  std::deque<int64_t> queue;
  std::vector<int32_t> fut(nt, 0);  // consecutive splits that moved all means to this child
  for (int64_t f = 0; f < nt; ++f)
    if ((int64_t)members[f].size() > page_size) queue.push_back(f);
  auto dist_to = [&](int64_t i, int64_t f) {
    return tri_dist2(&mu[3 * i], &verts[3 * (size_t)tris[3 * f]], &verts[3 * (size_t)tris[3 * f + 1]],
                     &verts[3 * (size_t)tris[3 * f + 2]]);
  };
  while (!queue.empty()) {
    const int64_t f = queue.front();
    queue.pop_front();
    const int32_t v0 = tris[3 * f], v1 = tris[3 * f + 1], v2 = tris[3 * f + 2];
    const int32_t m = (int32_t)(verts.size() / 3);
    for (int k = 0; k < 3; ++k) verts.push_back((verts[3 * (size_t)v0 + k] + verts[3 * (size_t)v1 + k]) * 0.5);
    tris[3 * f] = v2; tris[3 * f + 1] = v0; tris[3 * f + 2] = m;
    tris.push_back(v1); tris.push_back(v2); tris.push_back(m);
    const int64_t g = nt++;
    members.emplace_back();
    // the child of the nearer centroid (means sharing their nearest point on
    // the surface, a vertex, still separate)
    double cf[3], cg[3];
    for (int k = 0; k < 3; ++k) {
      cf[k] = ((verts[3 * (size_t)tris[3 * f] + k] + verts[3 * (size_t)tris[3 * f + 1] + k]) +
               verts[3 * (size_t)tris[3 * f + 2] + k]) / 3.0;
      cg[k] = ((verts[3 * (size_t)tris[3 * g] + k] + verts[3 * (size_t)tris[3 * g + 1] + k]) +
               verts[3 * (size_t)tris[3 * g + 2] + k]) / 3.0;
    }
    std::vector<int64_t> old;
    old.swap(members[f]);
    for (int64_t i : old) {
      double ef[3], eg[3];
      for (int k = 0; k < 3; ++k) { ef[k] = mu[3 * i + k] - cf[k]; eg[k] = mu[3 * i + k] - cg[k]; }
      if (dot3(ef, ef) <= dot3(eg, eg)) members[f].push_back(i);
      else members[g].push_back(i);
    }
    // a chain of kFutileSplits splits that separate nothing ends there
    const int32_t ff = members[g].empty() ? fut[f] + 1 : 0, fg = members[f].empty() ? fut[f] + 1 : 0;
    fut[f] = ff;
    fut.push_back(fg);
    if ((int64_t)members[f].size() > page_size && fut[f] < kFutileSplits) queue.push_back(f);
    if ((int64_t)members[g].size() > page_size && fut[g] < kFutileSplits) queue.push_back(g);
  }
  // merging
  std::vector<int64_t> cnt(nt);
  for (int64_t f = 0; f < nt; ++f) cnt[f] = (int64_t)members[f].size();
  const int64_t nv = (int64_t)verts.size() / 3;
  std::vector<std::vector<int64_t>> vfaces(nv);
  for (int64_t f = 0; f < nt; ++f)
    for (int j = 0; j < 3; ++j) vfaces[tris[3 * f + j]].push_back(f);
  std::vector<std::vector<int64_t>> nbrs(nt);
  for (int64_t f = 0; f < nt; ++f) {
    auto &nb = nbrs[f];
    for (int j = 0; j < 3; ++j)
      for (int64_t g : vfaces[tris[3 * f + j]])
        if (g != f) nb.push_back(g);
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
  }
  std::vector<double> cen(3 * nt);
  for (int64_t f = 0; f < nt; ++f)
    for (int k = 0; k < 3; ++k)
      cen[3 * f + k] = ((verts[3 * (size_t)tris[3 * f] + k] + verts[3 * (size_t)tris[3 * f + 1] + k]) +
                        verts[3 * (size_t)tris[3 * f + 2] + k]) / 3.0;
  std::vector<int64_t> page(nt, -1), todo;
  for (int64_t f = 0; f < nt; ++f)
    if (cnt[f] > 0) todo.push_back(f);
  int64_t n_pages = 0, next_base = -1;
  size_t ti = 0;
  std::vector<int64_t> seen_stamp(nt, -1);
  for (;;) {
    int64_t base;
    if (next_base < 0) {
      while (ti < todo.size() && page[todo[ti]] >= 0) ++ti;
      if (ti == todo.size()) break;
      base = todo[ti];
    } else {
      base = next_base;
      next_base = -1;
    }
    const int64_t pid = n_pages++;
    parent.push_back(-1);
    int64_t total = 0;
    std::deque<int64_t> frontier{base};
    seen_stamp[base] = pid;
    for (;;) {
      while (!frontier.empty()) {
        const int64_t f = frontier.front();
        frontier.pop_front();
        if (page[f] >= 0 || cnt[f] == 0) continue;
        if (total + cnt[f] > page_size && !(total == 0 && cnt[f] > page_size)) {
          next_base = f;
          frontier.clear();
          break;
        }
        page[f] = pid;
        total += cnt[f];
        if (cnt[f] > page_size) {  // an over-full triangle: its means fill this page and the next ones
          const int64_t extra = (cnt[f] + page_size - 1) / page_size - 1;
          for (int64_t k = 0; k < extra; ++k) parent.push_back(pid);
          n_pages += extra;
        }
        for (int64_t g : nbrs[f])
          if (seen_stamp[g] != pid && page[g] < 0) {
            seen_stamp[g] = pid;
            frontier.push_back(g);
          }
      }
      if (next_base >= 0) break;
      int64_t pick = -1;
      double bd = 0;
      for (int64_t f : todo) {
        if (page[f] >= 0 || seen_stamp[f] == pid) continue;
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = cen[3 * f + k] - cen[3 * base + k];
        const double d = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
        if (pick < 0 || d < bd) { pick = f; bd = d; }
      }
      if (pick < 0) break;
      seen_stamp[pick] = pid;
      frontier.push_back(pick);
    }
  }
  face_page.assign(nt, -1);
  for (int64_t f = 0; f < nt; ++f) face_page[f] = (int32_t)page[f];
  counts.assign(n_pages, 0);
  std::vector<std::array<int64_t, 3>> key(n);
  for (int64_t f = 0; f < nt; ++f)
    for (size_t k = 0; k < members[f].size(); ++k) {
      const int64_t i = members[f][k];
      key[i] = {page[f] + (int64_t)k / page_size, f, i};
    }
  order.resize(n);
  for (int64_t i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  for (int64_t i = 0; i < n; ++i) counts[key[i][0]]++;
}

}  // namespace vm

// ------------------------------------------------------------ inspection calls
using namespace vm;

extern "C" int vm3dgs_mesh_simplify(double *verts, int64_t nv, int32_t *tris, int64_t nt, int64_t target,
                                    int64_t *nv_out, int64_t *nt_out) {
  if ((!verts && nv) || (!tris && nt) || nv < 0 || nt < 0 || !nv_out || !nt_out)
    return fail(VM3DGS_E_INVAL, "bad mesh arrays");
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tris[i] < 0 || tris[i] >= nv) return fail(VM3DGS_E_INVAL, "triangle index out of range");
  std::vector<double> V(verts, verts + 3 * nv);
  std::vector<int32_t> T(tris, tris + 3 * nt);
  qem_simplify(V, T, target);
  std::copy(V.begin(), V.end(), verts);
  std::copy(T.begin(), T.end(), tris);
  *nv_out = (int64_t)V.size() / 3;
  *nt_out = (int64_t)T.size() / 3;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_mesh_assign_pages(int64_t n, const float *mu, int64_t page_size, const double *verts,
                                        int64_t nv, const int32_t *tris, int64_t nt, int64_t cap_v, double *verts_out,
                                        int64_t cap_t, int32_t *tris_out, int32_t *face_page_out, int64_t *order_out,
                                        int64_t *counts_out, int64_t *parent_out, int64_t *sizes_out) {
  if (n < 0 || (!mu && n) || page_size <= 0 || (!verts && nv) || (!tris && nt) || !sizes_out || !order_out ||
      !counts_out || !verts_out || !tris_out || !face_page_out)
    return fail(VM3DGS_E_INVAL, "bad arguments");
  if (nt == 0 && n > 0) return fail(VM3DGS_E_INVAL, "no triangles");
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tris[i] < 0 || tris[i] >= nv) return fail(VM3DGS_E_INVAL, "triangle index out of range");
  std::vector<double> V(verts, verts + 3 * nv);
  std::vector<int32_t> T(tris, tris + 3 * nt), fp;
  std::vector<int64_t> order, counts, parent;
  assign_pages(n, mu, page_size, V, T, fp, order, counts, parent);
  sizes_out[0] = (int64_t)V.size() / 3;
  sizes_out[1] = (int64_t)T.size() / 3;
  sizes_out[2] = (int64_t)counts.size();
  if (sizes_out[0] > cap_v || sizes_out[1] > cap_t) return fail(VM3DGS_E_CAPACITY, "output arrays too small");
  std::copy(V.begin(), V.end(), verts_out);
  std::copy(T.begin(), T.end(), tris_out);
  std::copy(fp.begin(), fp.end(), face_page_out);
  std::copy(order.begin(), order.end(), order_out);
  std::copy(counts.begin(), counts.end(), counts_out);
  if (parent_out) std::copy(parent.begin(), parent.end(), parent_out);
  return VM3DGS_OK;
}
