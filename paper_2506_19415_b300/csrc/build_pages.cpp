// Offline scene preparation on the host (Sec. 3 of the paper), OpenMP
// parallel.  Produces the page blocks the renderer streams, the per-level
// geometric errors that drive LOD choice, the page-marked proxy mesh for the
// visibility buffer and the page links.
//
//   decode      Sec. 3.5: normals dropped, opacity = logistic(logit),
//               scale = exp(log scale), quaternion normalised, SH stored
//               coefficient-major, Gaussians outside the scene box dropped.
//   paging      Sec. 3.2: pages of at most page_size Gaussians, padded with
//               zero-opacity Gaussians.  Mode 0: Morton order in chunks.
//               Mode 1: octree leaves (split while > page_size) in Morton
//               order, merged greedily up to, never over, the page size.
//   LOD         Sec. 3.4: only Gaussians of one page merge.  Method 0: parent
//               j of level l+1 merges children fanout*j.. of level l by moment
//               matching (weights opacity x volume); opacity is the mean of
//               the real children; the page's error at level l is its largest
//               parent standard deviation.  Method 1, the paper's own: k-means
//               clusters of the page's Gaussians in a scaled attribute space,
//               each averaged into one parent (kmeans_level).
//   proxy       Sec. 3.1 stand-in: voxels whose means' opacities sum to
//               kappa, one 3x3x3 closing, exposed faces marked with the
//               majority page of the voxel and merged into rectangles.
//   links       Sec. 3.3: random points in each 2-sigma ellipsoid, uniform in
//               the spherical coordinates of the unit ball, nearest face
//               voxel; unmarked face voxels take the page with most samples;
//               a face of page q hit by a sample of page p != q links q -> p,
//               as do co-located means of other pages in a face voxel.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <parallel/algorithm>
#include <utility>
#include <vector>

#include "mesh.h"
#include "scene.h"

namespace {

using std::int64_t;
using std::uint64_t;

uint64_t spread3(uint64_t v) {
  uint64_t out = 0;
  for (int b = 0; b < 21; ++b) out |= ((v >> b) & 1ull) << (3 * b);
  return out;
}

uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void quat_to_rot(const double *q, double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

// symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations
void jacobi3(const double A_in[3][3], double lam[3], double V[3][3]) {
  double A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) { A[i][j] = A_in[i][j]; V[i][j] = i == j; }
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-36 * dia || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2 * A[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        double c = 1 / std::sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) lam[i] = A[i][i];
}

// rotation matrix -> unit quaternion (w,x,y,z), w >= 0 (Shepperd's method)
void rot_to_quat(const double R[3][3], double *q) {
  double tr = R[0][0] + R[1][1] + R[2][2];
  double cand[4] = {tr, R[0][0], R[1][1], R[2][2]};
  int k = 0;
  for (int i = 1; i < 4; ++i)
    if (cand[i] > cand[k]) k = i;
  if (k == 0) {
    double s = std::sqrt(std::max(1 + tr, 0.0)) * 2;
    q[0] = 0.25 * s; q[1] = (R[2][1] - R[1][2]) / s; q[2] = (R[0][2] - R[2][0]) / s; q[3] = (R[1][0] - R[0][1]) / s;
  } else if (k == 1) {
    double s = std::sqrt(std::max(1 + R[0][0] - R[1][1] - R[2][2], 0.0)) * 2;
    q[0] = (R[2][1] - R[1][2]) / s; q[1] = 0.25 * s; q[2] = (R[0][1] + R[1][0]) / s; q[3] = (R[0][2] + R[2][0]) / s;
  } else if (k == 2) {
    double s = std::sqrt(std::max(1 + R[1][1] - R[0][0] - R[2][2], 0.0)) * 2;
    q[0] = (R[0][2] - R[2][0]) / s; q[1] = (R[0][1] + R[1][0]) / s; q[2] = 0.25 * s; q[3] = (R[1][2] + R[2][1]) / s;
  } else {
    double s = std::sqrt(std::max(1 + R[2][2] - R[0][0] - R[1][1], 0.0)) * 2;
    q[0] = (R[1][0] - R[0][1]) / s; q[1] = (R[0][2] + R[2][0]) / s; q[2] = (R[1][2] + R[2][1]) / s; q[3] = 0.25 * s;
  }
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double sg = q[0] < 0 ? -1.0 : 1.0;
  for (int i = 0; i < 4; ++i) q[i] = sg * q[i] / n;
}

}  // namespace

// IEEE binary32 -> binary16, round to nearest even (handles subnormals, overflow to inf)
uint16_t vm::f32_to_f16(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  uint32_t sign = (x >> 16) & 0x8000u;
  uint32_t mant = x & 0x7FFFFFu;
  int exp = (int)((x >> 23) & 0xFF);
  if (exp == 0xFF) return (uint16_t)(sign | 0x7C00u | (mant ? 0x200u : 0));
  int e = exp - 127 + 15;
  if (e >= 31) return (uint16_t)(sign | 0x7C00u);
  if (e <= 0) {
    if (e < -10) return (uint16_t)sign;
    mant |= 0x800000u;
    int shift = 14 - e;                  // 24-bit significand -> (11 + e - 1) bits
    uint32_t h = mant >> shift;
    uint32_t rem = mant & ((1u << shift) - 1);
    uint32_t half = 1u << (shift - 1);
    if (rem > half || (rem == half && (h & 1))) ++h;
    return (uint16_t)(sign | h);
  }
  uint32_t h = ((uint32_t)e << 10) | (mant >> 13);
  uint32_t rem = mant & 0x1FFFu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1))) ++h;   // may carry into the exponent: still correct
  return (uint16_t)(sign | h);
}

namespace {
using vm::f32_to_f16;

struct Decoded {
  int64_t n = 0;
  int K = 1;
  std::vector<float> pos, scale, rot, opac, sh;  // sh [n][K][3]
  std::vector<int64_t> src;
};

Decoded decode(const vm3dgs_gaussians &in, const double lo[3], const double hi[3]) {
  Decoded d;
  d.K = (in.sh_degree + 1) * (in.sh_degree + 1);
  const int K = d.K;
  std::vector<uint8_t> keep(in.n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < in.n; ++i) {
    bool k = true;
    for (int a = 0; a < 3; ++a) {
      double p = in.pos[3 * i + a];
      k = k && p >= lo[a] && p <= hi[a];
    }
    keep[i] = k;
  }
  for (int64_t i = 0; i < in.n; ++i)
    if (keep[i]) d.src.push_back(i);
  d.n = (int64_t)d.src.size();
  d.pos.resize(3 * d.n); d.scale.resize(3 * d.n); d.rot.resize(4 * d.n); d.opac.resize(d.n);
  d.sh.resize((size_t)d.n * K * 3);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < d.n; ++j) {
    const int64_t i = d.src[j];
    for (int a = 0; a < 3; ++a) {
      d.pos[3 * j + a] = in.pos[3 * i + a];
      d.scale[3 * j + a] = (float)std::exp((double)in.log_scale[3 * i + a]);
    }
    double q[4] = {in.rot[4 * i], in.rot[4 * i + 1], in.rot[4 * i + 2], in.rot[4 * i + 3]};
    double nn = std::sqrt(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    for (int a = 0; a < 4; ++a) d.rot[4 * j + a] = (float)(q[a] / nn);
    d.opac[j] = (float)(1.0 / (1.0 + std::exp(-(double)in.op_logit[i])));
    for (int c = 0; c < 3; ++c) d.sh[((size_t)j * K + 0) * 3 + c] = in.f_dc[3 * i + c];
    for (int k = 1; k < K; ++k)
      for (int c = 0; c < 3; ++c)
        d.sh[((size_t)j * K + k) * 3 + c] = in.f_rest[((size_t)i * 3 + c) * (K - 1) + (k - 1)];
  }
  return d;
}

void octree_leaves(const std::vector<uint64_t> &sc, int64_t s, int64_t e, int depth, int64_t ps,
                   std::vector<std::pair<int64_t, int64_t>> &out) {
  if (e - s == 0) return;
  if (e - s <= ps || depth >= 21) { out.emplace_back(s, e); return; }
  const int shift = 3 * (21 - depth - 1);
  const uint64_t base = (sc[s] >> (shift + 3)) << (shift + 3);
  int64_t b[9];
  b[0] = s; b[8] = e;
  for (int c = 1; c < 8; ++c)
    b[c] = std::lower_bound(sc.begin() + s, sc.begin() + e, base + ((uint64_t)c << shift)) - sc.begin();
  for (int c = 0; c < 8; ++c) octree_leaves(sc, b[c], b[c + 1], depth + 1, ps, out);
}

struct Grid {
  double lo[3], h;
  int64_t n[3];
  int64_t total() const { return n[0] * n[1] * n[2]; }
  int64_t lin(int64_t x, int64_t y, int64_t z) const { return (z * n[1] + y) * n[0] + x; }
  bool cell(const double *p, int64_t c[3]) const {
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      c[a] = (int64_t)std::floor((p[a] - lo[a]) / h);
      ok = ok && c[a] >= 0 && c[a] < n[a];
    }
    return ok;
  }
};

// majority value per key over (key, value) pairs; ties -> smallest value
void majority(std::vector<std::pair<int64_t, int64_t>> &kv, std::vector<int64_t> &dst) {
  __gnu_parallel::sort(kv.begin(), kv.end());
  size_t i = 0;
  while (i < kv.size()) {
    size_t j = i;
    int64_t best_v = -1, best_c = 0;
    while (j < kv.size() && kv[j].first == kv[i].first) {
      size_t k = j;
      while (k < kv.size() && kv[k].first == kv[j].first && kv[k].second == kv[j].second) ++k;
      int64_t c = (int64_t)(k - j);
      if (c > best_c) { best_c = c; best_v = kv[j].second; }
      j = k;
    }
    dst[kv[i].first] = best_v;
    i = j;
  }
}


// One LOD level of one page by k-means (Sec. 3.4): the real children of the
// level above (opacity > 0, slot order) are clustered into ceil(n / F)
// clusters in a position-first attribute space and every non-empty cluster
// becomes one parent.  Every sum runs in member order and every distance in
// feature order, in double, so the result is a fixed sequence of IEEE
// operations.
//   features  (pos - page mean) / page RMS radius (1 if 0); then aw times
//             the quaternion with w >= 0, the degree-0 SH colour, opacity
//   seeds     children floor(i * n / k), i < k
//   Lloyd     nearest centroid (lowest index on a tie), then each centroid
//             to its points' mean (one without points stays); at most
//             `iters` rounds, ending early when an assignment repeats
//   merge     means of position, opacity and SH; quaternions turned to the
//             first member's hemisphere, summed, normalised, w >= 0; mean
//             scale times sfac for two or more members
//   error     max over members of |member - parent position| + the
//             member's largest scale
// pb/cb are the SoA blocks (attribute row a at [a * m + g]); cb is zeroed by
// the caller.  Returns the page's error at this level.
// Nearest centroid of every point (lowest index on a tie).  X is [n][D],
// C is feature-major [D][k]; each distance sums its D squared differences in
// feature order, so vectorising across centroids leaves every value as is.
template <int D>
__attribute__((target_clones("avx2", "default"))) void assign_nearest(const double *__restrict X, int n,
                                                                      const double *__restrict C, int k,
                                                                      double *__restrict dist, int *__restrict lab) {
  for (int i = 0; i < n; ++i) {
    const double *x = X + (size_t)i * D;
    for (int j = 0; j < k; ++j) dist[j] = 0.0;
    for (int a = 0; a < D; ++a) {
      const double xa = x[a];
      const double *__restrict ca = C + (size_t)a * k;
      for (int j = 0; j < k; ++j) {
        const double t = xa - ca[j];
        dist[j] += t * t;
      }
    }
    int best = 0;
    for (int j = 1; j < k; ++j)
      if (dist[j] < dist[best]) best = j;
    lab[i] = best;
  }
}

double kmeans_level(const float *pb, int64_t mp, float *cb, int64_t mn, int K, int F, int iters, double sfac,
                    double aw) {
  constexpr int D = 11;
  std::vector<int> real;
  for (int64_t g = 0; g < mp; ++g)
    if (pb[10 * mp + g] > 0) real.push_back((int)g);
  const int n = (int)real.size();
  if (n == 0) return 0.0;
  auto at = [&](int row, int i) { return (double)pb[row * mp + real[i]]; };
  double mu[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) mu[a] += at(a, i);
  for (int a = 0; a < 3; ++a) mu[a] /= n;
  double r2 = 0;
  for (int i = 0; i < n; ++i) {
    const double d0 = at(0, i) - mu[0], d1 = at(1, i) - mu[1], d2 = at(2, i) - mu[2];
    const double t = d0 * d0 + d1 * d1 + d2 * d2;
    r2 += t;
  }
  double rad = std::sqrt(r2 / n);
  if (!(rad > 0)) rad = 1.0;
  std::vector<double> X((size_t)n * D);
  for (int i = 0; i < n; ++i) {
    double *x = &X[(size_t)i * D];
    for (int a = 0; a < 3; ++a) x[a] = (at(a, i) - mu[a]) / rad;
    const bool flip = at(6, i) < 0;
    for (int a = 0; a < 4; ++a) x[3 + a] = aw * (flip ? -at(6 + a, i) : at(6 + a, i));
    for (int c = 0; c < 3; ++c) x[7 + c] = aw * at(11 + c, i);
    x[10] = aw * at(10, i);
  }
  const int k = (n + F - 1) / F;
  // centroids feature-major [D][k] so the distance loop runs along centroids
  std::vector<double> C((size_t)D * k), acc((size_t)D * k), dist(k);
  for (int j = 0; j < k; ++j) {
    const double *x = &X[(size_t)((int64_t)j * n / k) * D];
    for (int a = 0; a < D; ++a) C[(size_t)a * k + j] = x[a];
  }
  std::vector<int> lab(n), prev(n), cnt(k);
  for (int it = 0; it < iters; ++it) {
    assign_nearest<D>(X.data(), n, C.data(), k, dist.data(), lab.data());
    if (it > 0 && lab == prev) break;
    std::fill(acc.begin(), acc.end(), 0.0);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int i = 0; i < n; ++i) {
      const int j = lab[i];
      ++cnt[j];
      for (int a = 0; a < D; ++a) acc[(size_t)a * k + j] += X[(size_t)i * D + a];
    }
    for (int j = 0; j < k; ++j)
      if (cnt[j] > 0)
        for (int a = 0; a < D; ++a) C[(size_t)a * k + j] = acc[(size_t)a * k + j] / cnt[j];
    prev = lab;
  }
  // members of each cluster in slot order
  std::vector<int> head(k + 1, 0), mem(n);
  for (int i = 0; i < n; ++i) ++head[lab[i] + 1];
  for (int j = 0; j < k; ++j) head[j + 1] += head[j];
  {
    std::vector<int> fill(head.begin(), head.end() - 1);
    for (int i = 0; i < n; ++i) mem[fill[lab[i]]++] = i;
  }
  std::vector<double> shs(3 * K);
  double emax = 0.0;
  int64_t slot = 0;
  for (int j = 0; j < k; ++j) {
    const int b = head[j], e = head[j + 1], cn = e - b;
    if (cn == 0) continue;
    double q0[4], qs[4] = {0, 0, 0, 0}, ps[3] = {0, 0, 0}, sc[3] = {0, 0, 0}, op = 0;
    for (int a = 0; a < 4; ++a) q0[a] = at(6 + a, mem[b]);
    std::fill(shs.begin(), shs.end(), 0.0);
    for (int t = b; t < e; ++t) {
      const int i = mem[t];
      double q[4];
      for (int a = 0; a < 4; ++a) q[a] = at(6 + a, i);
      const double dq = q[0] * q0[0] + q[1] * q0[1] + q[2] * q0[2] + q[3] * q0[3];
      for (int a = 0; a < 4; ++a) qs[a] += dq >= 0 ? q[a] : -q[a];
      for (int a = 0; a < 3; ++a) ps[a] += at(a, i);
      for (int a = 0; a < 3; ++a) sc[a] += at(3 + a, i);
      op += at(10, i);
      for (int c = 0; c < 3 * K; ++c) shs[c] += at(11 + c, i);
    }
    const double nq = std::sqrt(qs[0] * qs[0] + qs[1] * qs[1] + qs[2] * qs[2] + qs[3] * qs[3]);
    double q[4];
    if (nq > 0) {
      for (int a = 0; a < 4; ++a) q[a] = qs[a] / nq;
    } else {
      const double n0 = std::sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
      for (int a = 0; a < 4; ++a) q[a] = q0[a] / n0;
    }
    if (q[0] < 0)
      for (int a = 0; a < 4; ++a) q[a] = -q[a];
    double pos[3];
    for (int a = 0; a < 3; ++a) pos[a] = ps[a] / cn;
    for (int a = 0; a < 3; ++a) {
      double s = sc[a] / cn;
      if (cn >= 2) s = s * sfac;
      cb[(3 + a) * mn + slot] = (float)s;
      cb[a * mn + slot] = (float)pos[a];
    }
    for (int a = 0; a < 4; ++a) cb[(6 + a) * mn + slot] = (float)q[a];
    cb[10 * mn + slot] = (float)(op / cn);
    for (int c = 0; c < 3 * K; ++c) cb[(11 + c) * mn + slot] = (float)(shs[c] / cn);
    for (int t = b; t < e; ++t) {
      const int i = mem[t];
      const double d0 = at(0, i) - pos[0], d1 = at(1, i) - pos[1], d2 = at(2, i) - pos[2];
      const double smax = std::max(std::max(at(3, i), at(4, i)), at(5, i));
      emax = std::max(emax, std::sqrt(d0 * d0 + d1 * d1 + d2 * d2) + smax);
    }
    ++slot;
  }
  return emax;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" int vm3dgs_build_pages(const vm3dgs_gaussians *in, const vm3dgs_build_params *bp, vm3dgs_scene **out) {
  using namespace vm;
  if (!in || !bp || !out) return fail(VM3DGS_E_INVAL, "null argument");
  *out = nullptr;
  if (in->n < 0 || in->sh_degree < 0 || in->sh_degree > 3 || !in->pos || !in->log_scale || !in->rot ||
      !in->op_logit || !in->f_dc || (in->sh_degree > 0 && !in->f_rest))
    return fail(VM3DGS_E_INVAL, "bad Gaussian arrays");
  if (bp->page_size <= 0 || bp->lod_levels < 1 || bp->lod_levels > kMaxLevels || bp->lod_fanout < 2 ||
      bp->voxel <= 0 || bp->link_samples < 0 || bp->paging < 0 || bp->paging > 2)
    return fail(VM3DGS_E_INVAL, "bad build parameters");
  if (bp->paging == 2 && (!(bp->mesh_kappa > 0) || bp->mesh_closing < 0 || !(bp->mesh_qem_ratio > 0) ||
                          !(bp->mesh_qem_ratio <= 1)))
    return fail(VM3DGS_E_INVAL, "bad mesh proxy parameters");
  for (int a = 0; a < 3 && bp->paging == 2; ++a)
    if (std::ceil((bp->hi[a] - bp->lo[a]) / bp->voxel) > 1000000.0)
      return fail(VM3DGS_E_INVAL, "mesh proxy grid too fine (more than 1e6 samples along an axis)");
  if (bp->lod_method < 0 || bp->lod_method > 1 ||
      (bp->lod_method == 1 && (bp->kmeans_iters < 1 || !(bp->kmeans_scale >= 0) || !(bp->kmeans_attr_weight >= 0))))
    return fail(VM3DGS_E_INVAL, "bad LOD method parameters");
  {
    int64_t m = bp->page_size;
    for (int l = 1; l < bp->lod_levels; ++l) {
      if (m % bp->lod_fanout) return fail(VM3DGS_E_INVAL, "page_size must divide by fanout^(levels-1)");
      m /= bp->lod_fanout;
    }
  }
  for (int a = 0; a < 3; ++a)
    if (!(bp->hi[a] > bp->lo[a])) return fail(VM3DGS_E_INVAL, "empty scene box");
  if (bp->n_threads > 0) omp_set_num_threads(bp->n_threads);

  auto *S = new (std::nothrow) vm3dgs_scene();
  if (!S) return fail(VM3DGS_E_NOMEM, "scene");
  const int64_t ps = bp->page_size;
  Decoded d = decode(*in, bp->lo, bp->hi);
  const int K = d.K;
  S->page_size = (int32_t)ps; S->levels = bp->lod_levels; S->fanout = bp->lod_fanout;
  S->sh_degree = in->sh_degree; S->K = K; S->n_gauss = d.n;
  S->rec32 = rec_bytes32(K);
  S->rec16 = bp->fp16 ? rec_bytes16(K) : 0;

  // ---- paging
  std::vector<int64_t> starts, counts;
  std::vector<int64_t> order(d.n);
  std::vector<double> mverts;           // paging 2: the mesh proxy (Sec. 3.1) and its triangles' pages
  std::vector<int32_t> mtris, mface;
  std::vector<int64_t> mparent;         // extra pages of an over-full triangle: the page it carries
  if (bp->paging == 2) {
    MeshGrid g;
    for (int a = 0; a < 3; ++a) {
      g.lo[a] = bp->lo[a];
      g.n[a] = (int64_t)std::ceil((bp->hi[a] - bp->lo[a]) / bp->voxel);
    }
    g.h = bp->voxel;
    std::vector<uint8_t> closed;
    std::vector<int32_t> D;
    std::string err;
    if (!mesh_occupancy(g, d.n, d.pos.data(), d.scale.data(), d.rot.data(), d.opac.data(), (float)bp->mesh_kappa,
                        bp->mesh_op_min, bp->mesh_closing, closed, nullptr, err) ||
        !mesh_surface(g, closed, D, mtris, err)) {
      delete S;
      return fail(VM3DGS_E_CUDA, "mesh proxy: " + err);
    }
    mverts.resize(D.size());
    for (size_t i = 0; i < D.size(); ++i) mverts[i] = g.lo[i % 3] + (double)D[i] * (0.5 * g.h);
    const int64_t ntri = (int64_t)mtris.size() / 3;
    if (ntri > 0) qem_simplify(mverts, mtris, std::max<int64_t>(4, (int64_t)((double)ntri * bp->mesh_qem_ratio)));
    if (mtris.empty() && d.n > 0) {
      delete S;
      return fail(VM3DGS_E_INVAL, "mesh proxy is empty (no Gaussian occupies a sample point)");
    }
    assign_pages(d.n, d.pos.data(), ps, mverts, mtris, mface, order, counts, mparent);
    int64_t acc = 0;
    for (int64_t c : counts) { starts.push_back(acc); acc += c; }
  } else {
  // ---- Morton codes and paging
  std::vector<uint64_t> code(d.n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < d.n; ++i) {
    uint64_t q[3];
    for (int a = 0; a < 3; ++a) {
      double v = std::floor(((double)d.pos[3 * i + a] - bp->lo[a]) / (bp->hi[a] - bp->lo[a]) * 2097152.0);
      v = std::min(std::max(v, 0.0), 2097151.0);
      q[a] = (uint64_t)v;
    }
    code[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
  }
  std::vector<std::pair<uint64_t, int64_t>> ci(d.n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < d.n; ++i) ci[i] = {code[i], i};
  __gnu_parallel::sort(ci.begin(), ci.end());
  std::vector<uint64_t> sc(d.n);
  for (int64_t i = 0; i < d.n; ++i) { order[i] = ci[i].second; sc[i] = ci[i].first; }
  std::vector<std::pair<uint64_t, int64_t>>().swap(ci);
  if (bp->paging == 0) {
    for (int64_t s = 0; s < d.n; s += ps) { starts.push_back(s); counts.push_back(std::min(ps, d.n - s)); }
  } else {
    std::vector<std::pair<int64_t, int64_t>> leaves;
    octree_leaves(sc, 0, d.n, 0, ps, leaves);
    int64_t cs = -1, cn = 0;
    for (auto &lf : leaves) {
      int64_t m = lf.second - lf.first;
      if (cs >= 0 && cn + m <= ps) cn += m;
      else {
        if (cs >= 0) { starts.push_back(cs); counts.push_back(cn); }
        cs = lf.first; cn = m;
      }
    }
    if (cs >= 0) { starts.push_back(cs); counts.push_back(cn); }
  }
  }
  const int64_t NP = (int64_t)starts.size();
  S->n_pages = (int32_t)NP;
  S->count = counts;
  S->src.assign(NP * ps, -1);
  for (int64_t p = 0; p < NP; ++p)
    for (int64_t s = 0; s < counts[p]; ++s) S->src[p * ps + s] = d.src[order[starts[p] + s]];

  // ---- page blocks, all levels
  const int NA = n_attr32(K);
  int64_t total32 = 0;
  for (int l = 0; l < S->levels; ++l) { S->off32[l] = total32; total32 += NP * (int64_t)S->m(l) * S->rec32; }
  S->bytes32 = total32;
  S->data32 = (uint8_t *)std::aligned_alloc(4096, (size_t)((total32 + 4095) / 4096 * 4096));
  if (!S->data32) { delete S; return fail(VM3DGS_E_NOMEM, "page data"); }
  // level 0 gather
  {
    float *L0 = (float *)(S->data32 + S->off32[0]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < NP; ++p) {
      float *blk = L0 + p * ps * NA;
      std::memset(blk, 0, sizeof(float) * ps * NA);
      for (int64_t s = 0; s < counts[p]; ++s) {
        const int64_t j = order[starts[p] + s];
        for (int a = 0; a < 3; ++a) blk[(0 + a) * ps + s] = d.pos[3 * j + a];
        for (int a = 0; a < 3; ++a) blk[(3 + a) * ps + s] = d.scale[3 * j + a];
        for (int a = 0; a < 4; ++a) blk[(6 + a) * ps + s] = d.rot[4 * j + a];
        blk[10 * ps + s] = d.opac[j];
        for (int k = 0; k < 3 * K; ++k) blk[(11 + k) * ps + s] = d.sh[(size_t)j * K * 3 + k];
      }
    }
  }
  // LOD levels and errors
  S->err.assign(NP * S->levels, 0.0f);
  if (bp->lod_method == 1) {
    const double sfac = bp->kmeans_scale > 0 ? bp->kmeans_scale : std::pow((double)S->fanout, 1.0 / 3.0);
    for (int l = 1; l < S->levels; ++l) {
      const int64_t mp = S->m(l - 1), mn = S->m(l);
      const float *prev = (const float *)(S->data32 + S->off32[l - 1]);
      float *cur = (float *)(S->data32 + S->off32[l]);
#pragma omp parallel for schedule(dynamic, 1)
      for (int64_t p = 0; p < NP; ++p) {
        float *cb = cur + p * mn * NA;
        std::memset(cb, 0, sizeof(float) * mn * NA);
        S->err[p * S->levels + l] = (float)kmeans_level(prev + p * mp * NA, mp, cb, mn, K, S->fanout,
                                                        bp->kmeans_iters, sfac, bp->kmeans_attr_weight);
      }
    }
  }
  for (int l = 1; l < S->levels && bp->lod_method != 1; ++l) {
    const int64_t mp = S->m(l - 1), mn = S->m(l), F = S->fanout;
    const float *prev = (const float *)(S->data32 + S->off32[l - 1]);
    float *cur = (float *)(S->data32 + S->off32[l]);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < NP; ++p) {
      const float *pb = prev + p * mp * NA;
      float *cb = cur + p * mn * NA;
      std::memset(cb, 0, sizeof(float) * mn * NA);
      double emax = 0.0;
      for (int64_t j = 0; j < mn; ++j) {
        double w[64], W = 0;
        int nreal = 0;
        double osum = 0;
        for (int64_t c = 0; c < F; ++c) {
          const int64_t g = j * F + c;
          double o = pb[10 * mp + g];
          w[c] = o * (double)pb[3 * mp + g] * (double)pb[4 * mp + g] * (double)pb[5 * mp + g];
          W += w[c];
          if (o > 0) { ++nreal; osum += o; }
        }
        if (!(W > 0)) continue;  // padding parent: stays zero
        double mu[3] = {0, 0, 0};
        for (int64_t c = 0; c < F; ++c)
          for (int a = 0; a < 3; ++a) mu[a] += w[c] * pb[a * mp + j * F + c];
        for (int a = 0; a < 3; ++a) mu[a] /= W;
        double Sig[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int64_t c = 0; c < F; ++c) {
          const int64_t g = j * F + c;
          double q[4] = {pb[6 * mp + g], pb[7 * mp + g], pb[8 * mp + g], pb[9 * mp + g]};
          double R[3][3];
          quat_to_rot(q, R);
          double s2[3];
          for (int a = 0; a < 3; ++a) s2[a] = (double)pb[(3 + a) * mp + g] * (double)pb[(3 + a) * mp + g];
          double dx[3];
          for (int a = 0; a < 3; ++a) dx[a] = (double)pb[a * mp + g] - mu[a];
          for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
              double si = R[r][0] * s2[0] * R[cc][0] + R[r][1] * s2[1] * R[cc][1] + R[r][2] * s2[2] * R[cc][2];
              Sig[r][cc] += w[c] * (si + dx[r] * dx[cc]);
            }
        }
        for (int r = 0; r < 3; ++r)
          for (int cc = 0; cc < 3; ++cc) Sig[r][cc] /= W;
        double lam[3], V[3][3];
        jacobi3(Sig, lam, V);
        int idx[3] = {0, 1, 2};
        std::sort(idx, idx + 3, [&](int a, int b) { return lam[a] > lam[b] || (lam[a] == lam[b] && a < b); });
        double Rm[3][3], ls[3];
        for (int k = 0; k < 3; ++k) {
          ls[k] = lam[idx[k]];
          for (int r = 0; r < 3; ++r) Rm[r][k] = V[r][idx[k]];
        }
        for (int k = 0; k < 2; ++k) {
          int am = 0;
          for (int r = 1; r < 3; ++r)
            if (std::fabs(Rm[r][k]) > std::fabs(Rm[am][k])) am = r;
          if (Rm[am][k] < 0)
            for (int r = 0; r < 3; ++r) Rm[r][k] = -Rm[r][k];
        }
        Rm[0][2] = Rm[1][0] * Rm[2][1] - Rm[2][0] * Rm[1][1];
        Rm[1][2] = Rm[2][0] * Rm[0][1] - Rm[0][0] * Rm[2][1];
        Rm[2][2] = Rm[0][0] * Rm[1][1] - Rm[1][0] * Rm[0][1];
        double q[4];
        rot_to_quat(Rm, q);
        for (int a = 0; a < 3; ++a) cb[a * mn + j] = (float)mu[a];
        for (int a = 0; a < 3; ++a) cb[(3 + a) * mn + j] = (float)std::sqrt(std::max(ls[a], 1e-30));
        for (int a = 0; a < 4; ++a) cb[(6 + a) * mn + j] = (float)q[a];
        cb[10 * mn + j] = (float)(nreal > 0 ? osum / nreal : 0.0);
        for (int k = 0; k < 3 * K; ++k) {
          double acc = 0;
          for (int64_t c = 0; c < F; ++c) acc += w[c] * pb[(11 + k) * mp + j * F + c];
          cb[(11 + k) * mn + j] = (float)(acc / W);
        }
        emax = std::max(emax, std::sqrt(std::max(ls[0], 1e-30)));
      }
      S->err[p * S->levels + l] = (float)emax;
    }
  }
  // fp16 records
  if (bp->fp16) {
    const int NH = n_half16(K);
    int64_t total16 = 0;
    for (int l = 0; l < S->levels; ++l) { S->off16[l] = total16; total16 += NP * (int64_t)S->m(l) * S->rec16; }
    S->bytes16 = total16;
    S->data16 = (uint8_t *)std::aligned_alloc(4096, (size_t)((total16 + 4095) / 4096 * 4096));
    if (!S->data16) { delete S; return fail(VM3DGS_E_NOMEM, "fp16 page data"); }
    for (int l = 0; l < S->levels; ++l) {
      const int64_t m = S->m(l);
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < NP; ++p) {
        const float *src = (const float *)(S->data32 + S->off32[l]) + p * m * NA;
        uint8_t *dst = S->data16 + S->off16[l] + p * m * S->rec16;
        float *f = (float *)dst;
        uint16_t *h = (uint16_t *)(dst + 16 * m);
        for (int64_t g = 0; g < m; ++g) {
          for (int a = 0; a < 3; ++a) f[a * m + g] = src[a * m + g];
          f[3 * m + g] = src[10 * m + g];
          for (int a = 0; a < 3; ++a) h[a * m + g] = f32_to_f16(src[(3 + a) * m + g]);
          for (int a = 0; a < 4; ++a) h[(3 + a) * m + g] = f32_to_f16(src[(6 + a) * m + g]);
          for (int k = 0; k < 3 * K; ++k) h[(7 + k) * m + g] = f32_to_f16(src[(11 + k) * m + g]);
          for (int k = 7 + 3 * K; k < NH; ++k) h[k * m + g] = 0;
        }
      }
    }
  }

  const float *L0 = (const float *)(S->data32 + S->off32[0]);
  // ---- link samples
  const int KS = bp->link_samples;
  const double twopi = 2.0 * 3.14159265358979323846, pi = 3.14159265358979323846;
  auto sample_point = [&](int64_t p, int64_t s, int j, double *x) {
    const float *blk = L0 + p * ps * NA;
    const uint64_t vid = (uint64_t)(p * ps + s);
    double u[3];
    for (int a = 0; a < 3; ++a)
      u[a] = (double)(splitmix64(((vid * (uint64_t)KS + (uint64_t)j) * 4ull + (uint64_t)a) ^ bp->seed) >> 11) *
             (1.0 / 9007199254740992.0);
    double r = u[0], th = twopi * u[1], ph = pi * u[2];
    double e[3] = {r * std::sin(ph) * std::cos(th), r * std::sin(ph) * std::sin(th), r * std::cos(ph)};
    double q[4] = {blk[6 * ps + s], blk[7 * ps + s], blk[8 * ps + s], blk[9 * ps + s]};
    double R[3][3];
    quat_to_rot(q, R);
    double loc[3];
    for (int a = 0; a < 3; ++a) loc[a] = bp->link_sigma * (double)blk[(3 + a) * ps + s] * e[a];
    for (int a = 0; a < 3; ++a) x[a] = (double)blk[a * ps + s] + ((R[a][0] * loc[0] + R[a][1] * loc[1]) + R[a][2] * loc[2]);
  };
  if (bp->paging == 2) {
    // ---- links from the mesh (Sec. 3.3): the nearest triangle of each sample
    std::vector<uint64_t> mpairs;
    if (bp->links && KS > 0) {
      TriIndex *ix = tri_index_build(mverts, mtris);
      std::vector<std::vector<uint64_t>> tl(omp_get_max_threads());
#pragma omp parallel for schedule(dynamic, 4)
      for (int64_t p = 0; p < NP; ++p) {
        auto &mine = tl[omp_get_thread_num()];
        for (int64_t s = 0; s < counts[p]; ++s)
          for (int j = 0; j < KS; ++j) {
            double x[3];
            sample_point(p, s, j, x);
            const int32_t f = tri_index_nearest(ix, x);
            const int32_t q = f >= 0 ? mface[f] : -1;
            if (q >= 0 && q != p) mine.push_back((uint64_t)q * (uint64_t)NP + (uint64_t)p);
          }
      }
      tri_index_free(ix);
      for (auto &t : tl) mpairs.insert(mpairs.end(), t.begin(), t.end());
    }
    if (bp->links) {
      for (int64_t q = 0; q < NP; ++q)
        if (mparent[q] >= 0) mpairs.push_back((uint64_t)mparent[q] * (uint64_t)NP + (uint64_t)q);
      __gnu_parallel::sort(mpairs.begin(), mpairs.end());
      mpairs.erase(std::unique(mpairs.begin(), mpairs.end()), mpairs.end());
    }
    S->link_ptr.assign(NP + 1, 0);
    S->link_col.resize(mpairs.size());
    for (size_t i = 0; i < mpairs.size(); ++i) {
      S->link_ptr[mpairs[i] / NP + 1]++;
      S->link_col[i] = (int32_t)(mpairs[i] % NP);
    }
    for (int64_t p = 0; p < NP; ++p) S->link_ptr[p + 1] += S->link_ptr[p];
    S->verts.resize(mverts.size());
    for (size_t i = 0; i < mverts.size(); ++i) S->verts[i] = (float)mverts[i];
    S->tris = mtris;
    S->face_page = mface;
    finish_scene(S);
    *out = S;
    return VM3DGS_OK;
  }

  // ---- voxel proxy
  Grid G;
  for (int a = 0; a < 3; ++a) { G.lo[a] = bp->lo[a]; G.n[a] = (int64_t)std::ceil((bp->hi[a] - bp->lo[a]) / bp->voxel); }
  G.h = bp->voxel;
  const int64_t NV = G.total();
  // real Gaussians in (page, slot) order
  std::vector<int64_t> gstart(NP + 1, 0);
  for (int64_t p = 0; p < NP; ++p) gstart[p + 1] = gstart[p] + counts[p];
  const int64_t NG = gstart[NP];
  std::vector<int64_t> gvox(NG);
  std::vector<int32_t> gpage(NG);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t p = 0; p < NP; ++p)
    for (int64_t s = 0; s < counts[p]; ++s) {
      const float *blk = L0 + p * ps * NA;
      double mu[3] = {blk[0 * ps + s], blk[1 * ps + s], blk[2 * ps + s]};
      int64_t c[3];
      const int64_t g = gstart[p] + s;
      gvox[g] = G.cell(mu, c) ? G.lin(c[0], c[1], c[2]) : -1;
      gpage[g] = (int32_t)p;
    }
  // voxel-sorted Gaussians: occupancy sums in (page, slot) order per voxel, majority page
  std::vector<std::pair<int64_t, int64_t>> vg;
  vg.reserve(NG);
  for (int64_t g = 0; g < NG; ++g)
    if (gvox[g] >= 0) vg.emplace_back(gvox[g], g);
  __gnu_parallel::sort(vg.begin(), vg.end());
  std::vector<uint8_t> occ(NV, 0);
  std::vector<int32_t> vpage(NV, -1);
  {
    std::vector<size_t> runs;
    for (size_t i = 0; i < vg.size(); ++i)
      if (i == 0 || vg[i].first != vg[i - 1].first) runs.push_back(i);
    runs.push_back(vg.size());
    const int64_t nruns = (int64_t)runs.size() - 1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nruns; ++r) {
      double sum = 0;
      const int64_t v = vg[runs[r]].first;
      std::vector<int32_t> pgs;
      for (size_t i = runs[r]; i < runs[r + 1]; ++i) {
        const int64_t g = vg[i].second;
        const int64_t p = gpage[g], s = g - gstart[p];
        sum += (double)L0[p * ps * NA + 10 * ps + s];
        pgs.push_back((int32_t)p);
      }
      occ[v] = sum >= bp->kappa;
      std::sort(pgs.begin(), pgs.end());
      int32_t best = -1;
      size_t bc = 0;
      for (size_t i = 0; i < pgs.size();) {
        size_t j = i;
        while (j < pgs.size() && pgs[j] == pgs[i]) ++j;
        if (j - i > bc) { bc = j - i; best = pgs[i]; }
        i = j;
      }
      vpage[v] = best;
    }
  }
  // closing: dilation (outside = empty) then erosion (outside = full), separable per axis
  std::vector<uint8_t> closed(occ);
  if (bp->closing) {
    auto pass = [&](std::vector<uint8_t> &m, int axis, bool dil) {
      std::vector<uint8_t> o(m.size());
      const int64_t nx = G.n[0], ny = G.n[1], nz = G.n[2];
#pragma omp parallel for schedule(static)
      for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
          for (int64_t x = 0; x < nx; ++x) {
            int64_t c[3] = {x, y, z};
            uint8_t acc = dil ? 0 : 1;
            for (int dlt = -1; dlt <= 1; ++dlt) {
              int64_t cc[3] = {x, y, z};
              cc[axis] += dlt;
              uint8_t v;
              if (cc[axis] < 0 || cc[axis] >= G.n[axis]) v = dil ? 0 : 1;
              else v = m[G.lin(cc[0], cc[1], cc[2])];
              acc = dil ? (acc | v) : (acc & v);
            }
            o[G.lin(c[0], c[1], c[2])] = acc;
          }
      m.swap(o);
    };
    for (int a = 0; a < 3; ++a) pass(closed, a, true);
    for (int a = 0; a < 3; ++a) pass(closed, a, false);
  }
  for (int64_t v = 0; v < NV; ++v)
    if (!closed[v]) vpage[v] = -1;
  auto is_closed = [&](int64_t x, int64_t y, int64_t z) -> bool {
    if (x < 0 || y < 0 || z < 0 || x >= G.n[0] || y >= G.n[1] || z >= G.n[2]) return false;
    return closed[G.lin(x, y, z)] != 0;
  };
  static const int DIRS[6][2] = {{0, -1}, {0, 1}, {1, -1}, {1, 1}, {2, -1}, {2, 1}};
  std::vector<uint8_t> facebits(NV, 0);
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < G.n[2]; ++z)
    for (int64_t y = 0; y < G.n[1]; ++y)
      for (int64_t x = 0; x < G.n[0]; ++x) {
        if (!closed[G.lin(x, y, z)]) continue;
        uint8_t b = 0;
        for (int f = 0; f < 6; ++f) {
          int64_t c[3] = {x, y, z};
          c[DIRS[f][0]] += DIRS[f][1];
          if (!is_closed(c[0], c[1], c[2])) b |= (uint8_t)(1u << f);
        }
        facebits[G.lin(x, y, z)] = b;
      }
  auto face_cell = [&](const double *xp) -> int64_t {
    int64_t c[3];
    if (!G.cell(xp, c)) return -1;
    const int64_t own = G.lin(c[0], c[1], c[2]);
    if (facebits[own]) return own;
    double best_d = INFINITY;
    int64_t best = -1;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          int64_t cc[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
          if (cc[0] < 0 || cc[1] < 0 || cc[2] < 0 || cc[0] >= G.n[0] || cc[1] >= G.n[1] || cc[2] >= G.n[2]) continue;
          const int64_t l = G.lin(cc[0], cc[1], cc[2]);
          if (!facebits[l]) continue;
          double d2 = 0;
          for (int a = 0; a < 3; ++a) {
            double ctr = G.lo[a] + ((double)cc[a] + 0.5) * G.h;
            d2 += (ctr - xp[a]) * (ctr - xp[a]);
          }
          if (d2 < best_d || (d2 == best_d && l < best)) { best_d = d2; best = l; }
        }
    return best;
  };
  if (KS > 0) {
    // unmarked face voxels take the page with the most samples in them
    std::vector<std::vector<std::pair<int64_t, int64_t>>> tl(omp_get_max_threads());
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < NP; ++p) {
      auto &mine = tl[omp_get_thread_num()];
      for (int64_t s = 0; s < counts[p]; ++s)
        for (int j = 0; j < KS; ++j) {
          double x[3];
          sample_point(p, s, j, x);
          int64_t v = face_cell(x);
          if (v >= 0 && vpage[v] < 0) mine.emplace_back(v, p);
        }
    }
    std::vector<std::pair<int64_t, int64_t>> all;
    for (auto &t : tl) all.insert(all.end(), t.begin(), t.end());
    std::vector<int64_t> maj(NV, -2);
    if (!all.empty()) {
      majority(all, maj);
      for (auto &kv : all)
        if (maj[kv.first] >= 0) vpage[kv.first] = (int32_t)maj[kv.first];
    }
  }
  std::vector<uint64_t> pairs;
  if (bp->links) {
    std::vector<std::vector<uint64_t>> tl(omp_get_max_threads());
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < NP; ++p) {
      auto &mine = tl[omp_get_thread_num()];
      const float *blk = L0 + p * ps * NA;
      for (int64_t s = 0; s < counts[p]; ++s) {
        for (int j = 0; j < KS; ++j) {
          double x[3];
          sample_point(p, s, j, x);
          int64_t v = face_cell(x);
          if (v >= 0 && vpage[v] >= 0 && vpage[v] != p) mine.push_back((uint64_t)vpage[v] * (uint64_t)NP + (uint64_t)p);
        }
        double mu[3] = {blk[0 * ps + s], blk[1 * ps + s], blk[2 * ps + s]};
        int64_t c[3];
        if (G.cell(mu, c)) {
          const int64_t v = G.lin(c[0], c[1], c[2]);
          if (facebits[v] && vpage[v] >= 0 && vpage[v] != p) mine.push_back((uint64_t)vpage[v] * (uint64_t)NP + (uint64_t)p);
        }
        if (mine.size() > (1u << 22)) {
          std::sort(mine.begin(), mine.end());
          mine.erase(std::unique(mine.begin(), mine.end()), mine.end());
        }
      }
    }
    for (auto &t : tl) pairs.insert(pairs.end(), t.begin(), t.end());
    __gnu_parallel::sort(pairs.begin(), pairs.end());
    pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  }
  S->link_ptr.assign(NP + 1, 0);
  S->link_col.resize(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) {
    S->link_ptr[pairs[i] / NP + 1]++;
    S->link_col[i] = (int32_t)(pairs[i] % NP);
  }
  for (int64_t p = 0; p < NP; ++p) S->link_ptr[p + 1] += S->link_ptr[p];

  // ---- greedy rectangles per (axis, side, layer)
  struct Slab { int f; int64_t k; };
  std::vector<Slab> slabs;
  for (int f = 0; f < 6; ++f)
    for (int64_t k = 0; k < G.n[DIRS[f][0]]; ++k) slabs.push_back({f, k});
  std::vector<std::vector<float>> sv(slabs.size());
  std::vector<std::vector<int32_t>> sp(slabs.size());
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t si = 0; si < (int64_t)slabs.size(); ++si) {
    const int f = slabs[si].f, a = DIRS[f][0], sgn = DIRS[f][1];
    const int64_t k = slabs[si].k;
    const int ua = (a + 1) % 3, wa = (a + 2) % 3;
    const int64_t U = G.n[ua], W = G.n[wa];
    std::vector<int32_t> pg(U * W, -2);
    bool any = false;
    for (int64_t w = 0; w < W; ++w)
      for (int64_t u = 0; u < U; ++u) {
        int64_t c[3];
        c[a] = k; c[ua] = u; c[wa] = w;
        const int64_t l = G.lin(c[0], c[1], c[2]);
        if (facebits[l] & (1u << f)) { pg[w * U + u] = vpage[l]; any = true; }
      }
    if (!any) continue;
    std::vector<uint8_t> used(U * W, 0);
    const double plane = G.lo[a] + G.h * (double)(k + (sgn > 0 ? 1 : 0));
    for (int64_t w0 = 0; w0 < W; ++w0)
      for (int64_t u0 = 0; u0 < U; ++u0) {
        const int32_t q = pg[w0 * U + u0];
        if (q == -2 || used[w0 * U + u0]) continue;
        int64_t u1 = u0 + 1;
        while (u1 < U && pg[w0 * U + u1] == q && !used[w0 * U + u1]) ++u1;
        int64_t w1 = w0 + 1;
        while (w1 < W) {
          bool ok = true;
          for (int64_t u = u0; u < u1 && ok; ++u) ok = pg[w1 * U + u] == q && !used[w1 * U + u];
          if (!ok) break;
          ++w1;
        }
        for (int64_t w = w0; w < w1; ++w)
          for (int64_t u = u0; u < u1; ++u) used[w * U + u] = 1;
        const int64_t cu[4] = {u0, u1, u1, u0}, cw[4] = {w0, w0, w1, w1};
        for (int c4 = 0; c4 < 4; ++c4) {
          double v[3];
          v[a] = plane;
          v[ua] = G.lo[ua] + G.h * (double)cu[c4];
          v[wa] = G.lo[wa] + G.h * (double)cw[c4];
          for (int t = 0; t < 3; ++t) sv[si].push_back((float)v[t]);
        }
        sp[si].push_back(q);
      }
  }
  for (size_t si = 0; si < slabs.size(); ++si) {
    for (size_t qd = 0; qd < sp[si].size(); ++qd) {
      const int32_t b = (int32_t)(S->verts.size() / 3);
      for (int t = 0; t < 12; ++t) S->verts.push_back(sv[si][12 * qd + t]);
      const int32_t tri[6] = {b, b + 1, b + 2, b, b + 2, b + 3};
      S->tris.insert(S->tris.end(), tri, tri + 6);
      S->face_page.push_back(sp[si][qd]);
      S->face_page.push_back(sp[si][qd]);
    }
  }
  finish_scene(S);
  *out = S;
  return VM3DGS_OK;
}
