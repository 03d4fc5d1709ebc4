// Page determination (Sec. 4.1 "Page Determination"; evaluation "Page
// determination details"): the proxy mesh, each face marked with a page id,
// is rasterised into a low-resolution visibility buffer, then every pixel
// raises the request word of its page, and of the pages its page links to
// (Sec. 3.3), to a code that decreases with depth (atomic max).
//
// Compiled with -fmad=false.  Conventions (the paper uses the graphics
// hardware and states none): triangles crossing z = 0.2 are clipped
// (Sutherland-Hodgman) and fanned; positions are clamped to +-4e6 px and
// snapped to 1/256 px (round half to even); coverage uses 64-bit integer edge
// functions at pixel centres with an ownership rule (an edge owns the centres
// on it if it runs up, or right when horizontal) so that shared edges cover
// once; depth is the perspective-correct z, E_sum / sum_k E_k w_k with the
// per-vertex w_k = 1 / z_k; the visibility word is
// (bits(z) << 32) | (page + 1), minimum per pixel, all ones when empty.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "renderer.cuh"

namespace vm {
namespace {

struct V3 { float x, y, z; };

__device__ __forceinline__ V3 to_cam(const float *V, float4 p) {
  V3 r;
  r.x = ((V[0] * p.x + V[1] * p.y) + V[2] * p.z) + V[3];
  r.y = ((V[4] * p.x + V[5] * p.y) + V[6] * p.z) + V[7];
  r.z = ((V[8] * p.x + V[9] * p.y) + V[10] * p.z) + V[11];
  return r;
}

// Triangle t of the de-indexed proxy: three planes of ntri float4 vertices
// (x, y, z, w), the face's page id in the w of the first.
__device__ __forceinline__ void load_tri(const float4 *tv, int64_t ntri, int64_t t, float4 (&p)[3]) {
  p[0] = __ldg(tv + t);
  p[1] = __ldg(tv + ntri + t);
  p[2] = __ldg(tv + 2 * ntri + t);
}

__device__ __forceinline__ int64_t floordiv256(int64_t a) { return a >= 0 ? a / 256 : -((-a + 255) / 256); }

__device__ __forceinline__ bool owns(int64_t dx, int64_t dy) { return dy < 0 || (dy == 0 && dx > 0); }

// A snapped, oriented (area > 0) triangle with its clamped pixel box and the
// inverse view depths of its vertices.
struct Tri {
  int32_t X[3], Y[3];
  float W[3];
  uint32_t page1;
  int32_t i0, i1, j0, j1;
};
// Queued triangles are Tri records; a huge one is split into bands of kBand
// rows, each band a 64-bit entry (slot << 32 | band) of the band list.
using QTri = Tri;
static_assert(sizeof(QTri) <= kRasterRecord, "raster record");
constexpr uint64_t kNoBand = ~0ull;
constexpr int kBand = 4;

// coverage test and depth write of pixel (i, j)
__device__ __forceinline__ void shade(const Tri &t, const int64_t *dxe, const int64_t *dye, const bool *own,
                                      float farea, int64_t i, int64_t j, int Wf, uint64_t *fb) {
  const int ea[3] = {1, 2, 0};
  const int64_t px = i * 256 + 128, py = j * 256 + 128;
  int64_t E[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    E[k] = dxe[k] * (py - (int64_t)t.Y[ea[k]]) - dye[k] * (px - (int64_t)t.X[ea[k]]);
    if (!(E[k] > 0 || (E[k] == 0 && own[k]))) return;
  }
  const float s = (__ll2float_rn(E[0]) * t.W[0] + __ll2float_rn(E[1]) * t.W[1]) + __ll2float_rn(E[2]) * t.W[2];
  const float zp = farea / s;
  const uint64_t key = ((uint64_t)__float_as_uint(zp) << 32) | t.page1;
  atomicMin(reinterpret_cast<unsigned long long *>(fb + j * Wf + i), (unsigned long long)key);
}

// The edge functions at the centre of pixel (i, j), as shade() computes them.
__device__ __forceinline__ void edge_values(const Tri &t, const int64_t *dxe, const int64_t *dye, int64_t i, int64_t j,
                                            int64_t *E) {
  const int ea[3] = {1, 2, 0};
  const int64_t px = i * 256 + 128, py = j * 256 + 128;
#pragma unroll
  for (int k = 0; k < 3; ++k) E[k] = dxe[k] * (py - (int64_t)t.Y[ea[k]]) - dye[k] * (px - (int64_t)t.X[ea[k]]);
}

// shade() with the pixel's edge values already known (equal to those
// shade() would compute: the edge functions are exact integer affine maps,
// so stepping them by integer increments gives the same values)
__device__ __forceinline__ void shade_e(const Tri &t, const int64_t *E, const bool *own, float farea, int64_t i,
                                        int64_t j, int Wf, uint64_t *fb) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (!(E[k] > 0 || (E[k] == 0 && own[k]))) return;
  const float s = (__ll2float_rn(E[0]) * t.W[0] + __ll2float_rn(E[1]) * t.W[1]) + __ll2float_rn(E[2]) * t.W[2];
  const float zp = farea / s;
  const uint64_t key = ((uint64_t)__float_as_uint(zp) << 32) | t.page1;
  atomicMin(reinterpret_cast<unsigned long long *>(fb + j * Wf + i), (unsigned long long)key);
}

__device__ __forceinline__ void edges(const Tri &t, int64_t *dxe, int64_t *dye, bool *own, float *farea) {
  const int ea[3] = {1, 2, 0}, eb[3] = {2, 0, 1};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dxe[k] = (int64_t)t.X[eb[k]] - t.X[ea[k]];
    dye[k] = (int64_t)t.Y[eb[k]] - t.Y[ea[k]];
    own[k] = owns(dxe[k], dye[k]);
  }
  const int64_t area = dxe[2] * ((int64_t)t.Y[2] - t.Y[0]) - dye[2] * ((int64_t)t.X[2] - t.X[0]);
  *farea = __ll2float_rn(area);
}

// serial coverage of a whole triangle's pixel box by the calling thread
__device__ void raster_serial(const Tri &t, int Wf, uint64_t *fb) {
  int64_t dxe[3], dye[3];
  bool own[3];
  float farea;
  edges(t, dxe, dye, own, &farea);
  for (int64_t j = t.j0; j <= t.j1; ++j)
    for (int64_t i = t.i0; i <= t.i1; ++i) shade(t, dxe, dye, own, farea, i, j, Wf, fb);
}

struct RasterQueues {
  QTri *queue;         // medium triangles from the front, huge ones from the back
  uint64_t *bands;     // bands of the huge triangles
  uint32_t *count;     // [0] medium, [1] listed, [2] huge, [3] bands, [4] to clip
  uint32_t qcap, bcap;
};
constexpr int64_t kSmallPx = 16, kMediumPx = 1024;

// Snaps and orients one (clipped) triangle into t.  Returns the number of
// pixels of its clamped box, 0 when it has none (zero area, off the buffer).
// Boxes of at most kSmallPx pixels are rasterised by the warp's lanes
// together, up to kMediumPx by a warp each, larger ones in bands.
__device__ int64_t setup_tri(const V3 *c, uint32_t page1, float fxf, float fyf, float cxf, float cyf, int Wf, int Hf,
                             Tri &t) {
  int64_t X[3], Y[3];
  float Z[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float xs = fxf * (c[k].x / c[k].z) + cxf;
    float ys = fyf * (c[k].y / c[k].z) + cyf;
    xs = fminf(fmaxf(xs, -4.0e6f), 4.0e6f);
    ys = fminf(fmaxf(ys, -4.0e6f), 4.0e6f);
    X[k] = __float2ll_rn(xs * 256.0f);
    Y[k] = __float2ll_rn(ys * 256.0f);
    Z[k] = c[k].z;
  }
  int64_t area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
  if (area == 0) return 0;
  if (area < 0) {
    int64_t tmp = X[1]; X[1] = X[2]; X[2] = tmp;
    tmp = Y[1]; Y[1] = Y[2]; Y[2] = tmp;
    float tf = Z[1]; Z[1] = Z[2]; Z[2] = tf;
  }
  int64_t xmin = min(X[0], min(X[1], X[2])), xmax = max(X[0], max(X[1], X[2]));
  int64_t ymin = min(Y[0], min(Y[1], Y[2])), ymax = max(Y[0], max(Y[1], Y[2]));
  int64_t i0 = floordiv256(xmin - 128 + 255), i1 = floordiv256(xmax - 128);
  int64_t j0 = floordiv256(ymin - 128 + 255), j1 = floordiv256(ymax - 128);
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 > Wf - 1) i1 = Wf - 1;
  if (j1 > Hf - 1) j1 = Hf - 1;
  if (i1 < i0 || j1 < j0) return 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) { t.X[k] = (int32_t)X[k]; t.Y[k] = (int32_t)Y[k]; t.W[k] = 1.0f / Z[k]; }
  t.page1 = page1;
  t.i0 = (int32_t)i0; t.i1 = (int32_t)i1; t.j0 = (int32_t)j0; t.j1 = (int32_t)j1;
  return (i1 - i0 + 1) * (j1 - j0 + 1);
}

// a medium triangle into queue slot q (rasterised in place when full)
__device__ __forceinline__ void queue_medium(const Tri &t, uint32_t q, const RasterQueues &rq, int Wf, uint64_t *fb) {
  if (q < rq.qcap / 2) rq.queue[q] = t;
  else raster_serial(t, Wf, fb);
}

// a huge triangle from the back of the queue, its bands to the band list
__device__ void queue_huge(const Tri &t, const RasterQueues &rq, int Wf, uint64_t *fb) {
  const uint32_t nb = (uint32_t)((t.j1 - t.j0) / kBand + 1);
  const uint32_t q = atomicAdd(rq.count + 2, 1u);
  bool queued = false;
  if (q < rq.qcap / 2) {
    const uint32_t b0 = atomicAdd(rq.count + 3, nb);
    if ((uint64_t)b0 + nb <= rq.bcap) {
      rq.queue[rq.qcap - 1 - q] = t;
      for (uint32_t k = 0; k < nb; ++k) rq.bands[b0 + k] = ((uint64_t)q << 32) | k;
      queued = true;
    } else {
      for (uint32_t k = 0; b0 + k < rq.bcap && k < nb; ++k) rq.bands[b0 + k] = kNoBand;
    }
  }
  if (!queued) raster_serial(t, Wf, fb);  // queue or band list full
}

// The lanes of a warp rasterise their small triangles (lane l's in wtri[l],
// npx pixels, 0 for none) together: each lane takes one (triangle, pixel)
// pair of the warp's list in turn, found by a binary search over the
// inclusive pixel counts.
__device__ __forceinline__ void raster_warp(int npx, const Tri *wtri, int Wf, uint64_t *fb) {
  const int lane = threadIdx.x & 31;
  int incl = npx;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  for (int g0 = 0; g0 < total; g0 += 32) {
    const int g = g0 + lane;
    // owner = number of lanes whose inclusive count is <= g
    int L = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const int v = __shfl_sync(0xffffffffu, incl, min(L + s - 1, 31));
      if (L + s <= 32 && v <= g) L += s;
    }
    const int L_incl = __shfl_sync(0xffffffffu, incl, min(L, 31));
    const int L_npx = __shfl_sync(0xffffffffu, npx, min(L, 31));
    if (g < total) {
      const Tri &t = wtri[L];
      const int q = g - (L_incl - L_npx);
      const int bw = t.i1 - t.i0 + 1;
      int64_t dxe[3], dye[3];
      bool own[3];
      float farea;
      edges(t, dxe, dye, own, &farea);
      shade(t, dxe, dye, own, farea, t.i0 + q % bw, t.j0 + q / bw, Wf, fb);
    }
  }
  __syncwarp();
}

// False only if the triangle (all vertices in front of the near plane)
// covers no pixel centre: its screen box, from reciprocal-based positions
// widened by more than their distance to the exact ones (division, snapping
// to 1/256 px), holds no centre i + 1/2.
__device__ __forceinline__ bool may_cover(const V3 *q, float fxf, float fyf, float cxf, float cyf) {
  float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f, mag = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float r = __frcp_rn(q[k].z);
    const float ux = fxf * (q[k].x * r), uy = fyf * (q[k].y * r);
    const float x = ux + cxf, y = uy + cyf;
    xlo = fminf(xlo, x); xhi = fmaxf(xhi, x);
    ylo = fminf(ylo, y); yhi = fmaxf(yhi, y);
    mag = fmaxf(mag, fmaxf(fabsf(ux), fabsf(uy)));
  }
  if (!(mag < 1.0e6f)) return true;  // far outside or not finite: leave it to the exact test
  const float m = 1e-6f * (mag + fabsf(cxf) + fabsf(cyf)) + 1.0f / 128.0f;
  return floorf(xhi + m - 0.5f) >= ceilf(xlo - m - 0.5f) && floorf(yhi + m - 0.5f) >= ceilf(ylo - m - 0.5f);
}

// Smallest value over the box [lo, hi] of n.p + d, and a bound on its
// rounding error.
__device__ __forceinline__ void box_min(const float *n, float d, const float *lo, const float *hi, float &mn,
                                        float &err) {
  mn = d;
  float mag = fabsf(d);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mn += fminf(n[a] * lo[a], n[a] * hi[a]);
    mag += fabsf(n[a]) * fmaxf(fabsf(lo[a]), fabsf(hi[a]));
  }
  err = 1e-5f * mag + 1e-2f;
}

// The five culling planes of a camera as n.p + d > 0 on the culled side:
// x > kr z, x < kl z, y > kb z, y < kt z (planes through the eye 2 pixels
// beyond each side of the buffer) and z < zn.
struct CullPlanes {
  float n[5][3], d[5];
  float kr, kl, kb, kt, fxf, fyf, cxf, cyf;
};

__device__ __forceinline__ CullPlanes cull_planes(const vm3dgs_camera &cam, int ds) {
  CullPlanes P;
  const int Wf = (cam.width + ds - 1) / ds, Hf = (cam.height + ds - 1) / ds;
  const float fds = (float)ds;
  P.fxf = cam.fx / fds; P.fyf = cam.fy / fds; P.cxf = cam.cx / fds; P.cyf = cam.cy / fds;
  P.kr = ((float)Wf + 2.0f - P.cxf) / P.fxf; P.kl = (-2.0f - P.cxf) / P.fxf;
  P.kb = ((float)Hf + 2.0f - P.cyf) / P.fyf; P.kt = (-2.0f - P.cyf) / P.fyf;
  const float *V = cam.view;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P.n[0][a] = V[a] - P.kr * V[8 + a];
    P.n[1][a] = P.kl * V[8 + a] - V[a];
    P.n[2][a] = V[4 + a] - P.kb * V[8 + a];
    P.n[3][a] = P.kt * V[8 + a] - V[4 + a];
    P.n[4][a] = -V[8 + a];
  }
  P.d[0] = V[3] - P.kr * V[11];
  P.d[1] = P.kl * V[11] - V[3];
  P.d[2] = V[7] - P.kb * V[11];
  P.d[3] = P.kt * V[11] - V[7];
  P.d[4] = 0.2f - V[11];
  return P;
}

// Pass 1a: a thread per cluster.  A cluster is dropped when its box lies,
// with a margin larger than the rounding of either test, behind the near
// plane or beyond one of the side planes (planes through the eye, so every
// triangle inside is beyond it too and covers no pixel centre); the others
// are appended (warp-aggregated, in no particular order) to the live list.
__global__ void __launch_bounds__(256) cluster_cull_kernel(const Cluster *cl, int64_t ncl, vm3dgs_camera cam, int ds,
                                                           uint32_t *live, uint32_t *nlive) {
  __shared__ uint32_t s_cnt[8], s_base;
  const CullPlanes P = cull_planes(cam, ds);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // CTA-uniform rounds: one list reservation per CTA and round
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < ncl; b0 += stride) {
    const int64_t ci = b0 + threadIdx.x;
    bool keep = false;
    if (ci < ncl) {
      const float4 *c4 = reinterpret_cast<const float4 *>(cl + ci);
      const float4 u = __ldg(c4), w = __ldg(c4 + 1);
      const float lo[3] = {u.x, u.y, u.z}, hi[3] = {w.x, w.y, w.z};
      keep = true;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        float mn, err;
        box_min(P.n[k], P.d[k], lo, hi, mn, err);
        if (mn > err) keep = false;
      }
    }
    const uint32_t km = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_cnt[warp] = (uint32_t)__popc(km);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < 8; ++w) { const uint32_t c = s_cnt[w]; s_cnt[w] = tot; tot += c; }
      s_base = tot ? atomicAdd(nlive, tot) : 0u;
    }
    __syncthreads();
    if (keep) live[s_base + s_cnt[warp] + __popc(km & ((1u << lane) - 1u))] = (uint32_t)ci;
    __syncthreads();  // s_cnt and s_base are rewritten next round
  }
}

// Pass 1b: a warp per live cluster, a triangle per lane.  Triangles entirely
// behind the near plane, entirely more than 2 pixels beyond one side of the
// buffer, or in front of it with a screen box that holds no pixel centre,
// cover no pixel centre; the others in front of it are appended to a dense
// list so that pass 2 runs without idle lanes (each warp gathers them in
// shared memory and reserves list space once per kCullBuf entries, not once
// per cluster: the list counter is a single contended word), those crossing
// it to the clipping list.
constexpr int kCullBuf = 256;
__global__ void __launch_bounds__(256) raster_cull_kernel(const float4 *tv, int64_t ntri, const Cluster *cl,
                                                          const uint32_t *live, const uint32_t *nlive,
                                                          vm3dgs_camera cam, int ds, uint32_t *vis, uint32_t *nvis,
                                                          uint32_t *clip, uint32_t *nclip) {
  __shared__ uint32_t s_buf[8][kCullBuf];
  __shared__ uint32_t s_cnt[8], s_base;
  const int warp = threadIdx.x >> 5;
  uint32_t *buf = s_buf[warp];
  int nbuf = 0;  // warp-uniform
  const CullPlanes P = cull_planes(cam, ds);
  const float zn = 0.2f;
  const float *V = cam.view;
  const int lane = threadIdx.x & 31;
  const int64_t n = *nlive;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = w0; q < n; q += nw) {
    const uint32_t ci = live[q];
    const uint32_t first = cl[ci].first, count = cl[ci].count;
    const int64_t t = (int64_t)first + lane;
    bool keep = false;
    if ((uint32_t)lane < count) {
      float4 p[3];
      load_tri(tv, ntri, t, p);
      V3 c[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) c[k] = to_cam(V, p[k]);
      int nin = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) nin += c[k].z >= zn;
      if (nin > 0 && nin < 3) clip[atomicAdd(nclip, 1u)] = (uint32_t)t;
      if (nin == 3) {
        bool o1 = true, o2 = true, o3 = true, o4 = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          o1 = o1 && c[k].x > P.kr * c[k].z;
          o2 = o2 && c[k].x < P.kl * c[k].z;
          o3 = o3 && c[k].y > P.kb * c[k].z;
          o4 = o4 && c[k].y < P.kt * c[k].z;
        }
        keep = !(o1 || o2 || o3 || o4) && may_cover(c, P.fxf, P.fyf, P.cxf, P.cyf);
      }
    }
    const uint32_t km = __ballot_sync(0xffffffffu, keep);
    if (nbuf + __popc(km) > kCullBuf) {  // flush the warp's buffer
      uint32_t off = 0;
      if (lane == 0) off = atomicAdd(nvis, (uint32_t)nbuf);
      off = __shfl_sync(0xffffffffu, off, 0);
      for (int k = lane; k < nbuf; k += 32) vis[off + k] = buf[k];
      __syncwarp();
      nbuf = 0;
    }
    if (keep) buf[nbuf + __popc(km & ((1u << lane) - 1u))] = (uint32_t)t;
    nbuf += __popc(km);
    __syncwarp();
  }
  // one reservation for the rest of the CTA's buffers
  if (lane == 0) s_cnt[warp] = (uint32_t)nbuf;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < 8; ++w) { const uint32_t c = s_cnt[w]; s_cnt[w] = tot; tot += c; }
    s_base = tot ? atomicAdd(nvis, tot) : 0u;
  }
  __syncthreads();
  for (int k = lane; k < nbuf; k += 32) vis[s_base + s_cnt[warp] + k] = buf[k];
}

// Pass 2: snap and rasterise the listed triangles (small ones by the warp
// together, medium ones queued with one counter update per warp, huge ones
// in bands); each lane's triangle is set up directly in the warp's shared
// slots.
// Medium triangles gather per warp in shared memory (kMedBuf records) and
// reach the queue through one reservation per CTA at the end (the queue
// counter is a single contended word); a full buffer is flushed at once.
constexpr int kMedBuf = 32;
__device__ __forceinline__ void copy_tris(Tri *dst, const Tri *src, int n, int lane) {
  const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
  uint32_t *d = reinterpret_cast<uint32_t *>(dst);
  constexpr int W = sizeof(Tri) / 4;
  for (int k = lane; k < n * W; k += 32) d[k] = s[k];
}

__global__ void __launch_bounds__(256, 4) raster_setup_kernel(const float4 *tv, int64_t ntri, const uint32_t *vis,
                                                           const uint32_t *nvis, vm3dgs_camera cam, int ds,
                                                           uint64_t *fb, RasterQueues rq) {
  static_assert(sizeof(Tri) % 4 == 0, "Tri is copied as words");
  __shared__ Tri s_tri[8][32];
  __shared__ Tri s_med[8][kMedBuf];
  __shared__ uint32_t s_cnt[8], s_base;
  const int warp = threadIdx.x >> 5;
  Tri *wtri = s_tri[warp];
  Tri *mbuf = s_med[warp];
  int nmed = 0;  // warp-uniform
  const int Wf = (cam.width + ds - 1) / ds, Hf = (cam.height + ds - 1) / ds;
  const float fds = (float)ds;
  const float fxf = cam.fx / fds, fyf = cam.fy / fds, cxf = cam.cx / fds, cyf = cam.cy / fds;
  const int64_t n = *nvis;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t q = base + lane;
    int64_t npx = 0;
    if (q < n) {
      const int64_t t = vis[q];
      float4 p[3];
      load_tri(tv, ntri, t, p);
      V3 c[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) c[k] = to_cam(cam.view, p[k]);
      npx = setup_tri(c, (uint32_t)(__float_as_int(p[0].w) + 1), fxf, fyf, cxf, cyf, Wf, Hf, wtri[lane]);
      if (npx > kMediumPx) {
        queue_huge(wtri[lane], rq, Wf, fb);
        npx = 0;
      }
    }
    const bool med = npx > kSmallPx;
    const uint32_t mm = __ballot_sync(0xffffffffu, med);
    if (mm) {
      if (nmed + __popc(mm) > kMedBuf) {  // flush the warp's buffer now
        uint32_t q0 = 0;
        if (lane == 0) q0 = atomicAdd(rq.count, (uint32_t)nmed);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        const int fit = q0 < rq.qcap / 2 ? (int)min((uint32_t)nmed, rq.qcap / 2 - q0) : 0;
        copy_tris(rq.queue + q0, mbuf, fit, lane);
        __syncwarp();
        for (int k = fit + lane; k < nmed; k += 32) raster_serial(mbuf[k], Wf, fb);  // queue full
        __syncwarp();
        nmed = 0;
      }
      if (med) mbuf[nmed + __popc(mm & ((1u << lane) - 1u))] = wtri[lane];
      nmed += __popc(mm);
    }
    __syncwarp();
    raster_warp(med ? 0 : (int)npx, wtri, Wf, fb);
  }
  // one reservation for the CTA's buffered medium triangles
  if (lane == 0) s_cnt[warp] = (uint32_t)nmed;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < 8; ++w) { const uint32_t c = s_cnt[w]; s_cnt[w] = tot; tot += c; }
    s_base = tot ? atomicAdd(rq.count, tot) : 0u;
  }
  __syncthreads();
  if (nmed) {
    const uint32_t q0 = s_base + s_cnt[warp];
    const int fit = q0 < rq.qcap / 2 ? (int)min((uint32_t)nmed, rq.qcap / 2 - q0) : 0;
    copy_tris(rq.queue + q0, mbuf, fit, lane);
    for (int k = fit + lane; k < nmed; k += 32) raster_serial(mbuf[k], Wf, fb);  // queue full
  }
}

// Pass 2b: triangles crossing z = zn, clipped against that plane into a
// triangle (one vertex in front) or a quad (two) fanned from its first
// vertex; small pieces are rasterised by the thread, larger ones queued.
__global__ void __launch_bounds__(256) raster_clip_kernel(const float4 *tv, int64_t ntri, const uint32_t *clip,
                                                          const uint32_t *nclip, vm3dgs_camera cam, int ds,
                                                          uint64_t *fb, RasterQueues rq) {
  const int Wf = (cam.width + ds - 1) / ds, Hf = (cam.height + ds - 1) / ds;
  const float fds = (float)ds;
  const float fxf = cam.fx / fds, fyf = cam.fy / fds, cxf = cam.cx / fds, cyf = cam.cy / fds;
  const float zn = 0.2f;
  const int64_t n = *nclip;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int64_t t = clip[q];
    float4 p[3];
    load_tri(tv, ntri, t, p);
    V3 c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = to_cam(cam.view, p[k]);
    const uint32_t page1 = (uint32_t)(__float_as_int(p[0].w) + 1);
    bool inside[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) inside[k] = c[k].z >= zn;
    V3 poly[4];
    int m = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const V3 a = c[k], b = c[(k + 1) % 3];
      const bool ia = inside[k], ib = inside[(k + 1) % 3];
      if (ia) poly[m++] = a;
      if (ia != ib) {
        const float tt = (zn - a.z) / (b.z - a.z);
        V3 p;
        p.x = a.x + tt * (b.x - a.x);
        p.y = a.y + tt * (b.y - a.y);
        p.z = zn;
        poly[m++] = p;
      }
    }
    for (int k = 1; k + 1 < m; ++k) {
      const V3 tri[3] = {poly[0], poly[k], poly[k + 1]};
      Tri tr;
      const int64_t npx = setup_tri(tri, page1, fxf, fyf, cxf, cyf, Wf, Hf, tr);
      if (npx > kMediumPx) queue_huge(tr, rq, Wf, fb);
      else if (npx > kSmallPx) queue_medium(tr, atomicAdd(rq.count, 1u), rq, Wf, fb);
      else if (npx > 0) raster_serial(tr, Wf, fb);
    }
  }
}

// medium triangles: one warp each, lanes over the pixel box (a static split:
// taking them from a shared counter cost more in contended atomics than the
// tail it removed)
__global__ void __launch_bounds__(256) raster_medium_kernel(const QTri *queue, const uint32_t *qcount, uint32_t qcap,
                                                            int Wf, uint64_t *fb) {
  const uint32_t n = min(qcount[0], qcap / 2);
  const int lane = threadIdx.x & 31;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t q = w0; q < n; q += nw) {
    const Tri t = queue[q];
    int64_t dxe[3], dye[3];
    bool own[3];
    float farea;
    edges(t, dxe, dye, own, &farea);
    // (a medium box holds at most kMediumPx pixels: 32-bit indices) the
    // lane's pixels p = lane, lane + 32, ... as (column, row), stepped by
    // 32 = s_dy rows + s_dx columns with one carry, without a division a pixel
    // The edge values step with the pixel: a pixel (di, dj) further adds
    // 256 (dxe dj - dye di) to each.
    const int bw = t.i1 - t.i0 + 1, npx = bw * (t.j1 - t.j0 + 1);
    const int s_dy = 32 / bw, s_dx = 32 - s_dy * bw;
    int dy = lane / bw, dx = lane - dy * bw;
    int64_t E[3], dstep[3], dcarry[3];
    edge_values(t, dxe, dye, t.i0 + dx, t.j0 + dy, E);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dstep[k] = 256 * (dxe[k] * s_dy - dye[k] * s_dx);
      dcarry[k] = 256 * (dxe[k] + dye[k] * bw);
    }
    for (int p = lane; p < npx; p += 32) {
      shade_e(t, E, own, farea, t.i0 + dx, t.j0 + dy, Wf, fb);
      dx += s_dx;
      dy += s_dy;
#pragma unroll
      for (int k = 0; k < 3; ++k) E[k] += dstep[k];
      if (dx >= bw) {
        dx -= bw;
        ++dy;
#pragma unroll
        for (int k = 0; k < 3; ++k) E[k] += dcarry[k];
      }
    }
  }
}

__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) {  // b > 0
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Huge triangles in bands of kBand rows, one band per warp task; in each row
// only the pixels that can pass all three edge tests (E_k >= 0, a superset of
// the covered centres) are tested, with the same test as everywhere else.
__global__ void __launch_bounds__(256) raster_huge_kernel(const QTri *queue, const uint64_t *bands,
                                                          const uint32_t *qcount, uint32_t qcap, uint32_t bcap, int Wf,
                                                          uint64_t *fb) {
  const int64_t nb = min(qcount[3], bcap);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ea[3] = {1, 2, 0};
  for (int64_t b = w0; b < nb; b += nw) {
    const uint64_t e = bands[b];
    if (e == kNoBand) continue;
    const Tri t = queue[qcap - 1 - (uint32_t)(e >> 32)];
    int64_t dxe[3], dye[3];
    bool own[3];
    float farea;
    edges(t, dxe, dye, own, &farea);
    const int64_t ja = t.j0 + (int64_t)(uint32_t)e * kBand, jb = min((int64_t)t.j1, ja + kBand - 1);
    for (int64_t j = ja; j <= jb; ++j) {
      // E_k(i) = A_k - B_k i at the centre of pixel (i, j)
      const int64_t py = j * 256 + 128;
      int64_t lo_i = t.i0, hi_i = t.i1;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int64_t A = dxe[k] * (py - (int64_t)t.Y[ea[k]]) - dye[k] * (128 - (int64_t)t.X[ea[k]]);
        const int64_t B = 256 * dye[k];
        if (B == 0) {
          if (A < 0) hi_i = lo_i - 1;
        } else if (B > 0) {
          hi_i = min(hi_i, floordiv(A, B));
        } else {
          lo_i = max(lo_i, -floordiv(A, -B));
        }
      }
      if (lo_i + lane <= hi_i) {
        int64_t E[3];
        edge_values(t, dxe, dye, lo_i + lane, j, E);
        for (int64_t i = lo_i + lane; i <= hi_i; i += 32) {
          shade_e(t, E, own, farea, i, j, Wf, fb);
#pragma unroll
          for (int k = 0; k < 3; ++k) E[k] -= dye[k] * (256 * 32);
        }
      }
    }
  }
}

// The visibility buffer to "empty", the raster counters to 0, and (when req
// is given: the first view of a page determination) the request words,
// direct flags and per-page gathering words to 0.
__global__ void clear_kernel(uint64_t *fb, int64_t n, uint32_t *qcount, uint32_t *req, uint8_t *direct, uint32_t *dreq,
                             int64_t NP) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = t; i < n; i += stride) fb[i] = ~0ull;
  if (t < 8) qcount[t] = 0;
  if (req)
    for (int64_t i = t; i < NP; i += stride) {
      req[i] = 0;
      direct[i] = 0;
      if (dreq) dreq[i] = 0;
    }
}

// Per pixel: the code of its page goes to dst (atomic max, once per page
// and warp), and the page is marked direct.  With links dst is a separate
// per-page word, spread to the page and its linked pages afterwards.
__global__ void __launch_bounds__(256) reduce_kernel(const uint64_t *fb, int64_t npix, uint32_t *dst, uint8_t *direct) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < npix; base += stride) {
    const int64_t i = base + lane;
    const uint64_t key = i < npix ? fb[i] : ~0ull;
    const uint32_t low = (uint32_t)(key & 0xFFFFFFFFull);
    const bool valid = key != ~0ull && low != 0u;
    const int page = valid ? (int)(low - 1u) : -1;
    const uint32_t enc = valid ? 0xFFFFFFFFu - (uint32_t)(key >> 32) : 0u;
    const uint32_t peers = __match_any_sync(0xffffffffu, page);
    const uint32_t mx = __reduce_max_sync(peers, enc);
    if (!valid || (peers & ((1u << lane) - 1u)) != 0u) continue;
    atomicMax(dst + page, mx);
    direct[page] = 1;
  }
}

// Links (Sec. 3.3): a page seen directly raises its own request word and
// those of the pages it links to to its code (a thread per page, so each
// page's links are walked once a frame).
__global__ void __launch_bounds__(256) link_kernel(const uint32_t *dreq, int64_t NP, const int64_t *link_ptr,
                                                   const int32_t *link_col, uint32_t *req) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += stride) {
    const uint32_t v = dreq[p];
    if (v == 0u) continue;
    atomicMax(req + p, v);
    for (int64_t k = link_ptr[p]; k < link_ptr[p + 1]; ++k) atomicMax(req + link_col[k], v);
  }
}

__global__ void request_all_kernel(uint32_t *req, uint8_t *direct, int64_t NP) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += stride) {
    req[p] = 0xFFFFFFFFu;
    direct[p] = 1;
  }
}

}  // namespace

void launch_feedback_clear(uint64_t *fb, int64_t n, uint32_t *qcount, uint32_t *req, uint8_t *direct, uint32_t *dreq,
                           int64_t NP, cudaStream_t st) {
  const int64_t m = n > NP ? n : NP;
  clear_kernel<<<wave_grid((const void *)clear_kernel, 256, 0, m, 256), 256, 0, st>>>(fb, n, qcount, req, direct, dreq,
                                                                                     NP);
}

void launch_feedback_raster(const float4 *tv, const Cluster *cl, int64_t ncl, int64_t ntri,
                            const vm3dgs_camera &cam, int ds, uint64_t *fb, void *queue,
                            uint32_t *qcount, uint32_t qcap, uint64_t *bands, uint32_t bcap, uint32_t *vis,
                            uint32_t *clip, uint32_t *live, cudaStream_t st) {
  if (ntri <= 0 || ncl <= 0) return;
  // qcount (zeroed by the clear): [0] queued medium triangles, [1] listed
  // triangles, [2] queued huge triangles, [3] their bands, [4] triangles to
  // clip, [5] live clusters
  const RasterQueues rq{reinterpret_cast<QTri *>(queue), bands, qcount, qcap, bcap};
  cluster_cull_kernel<<<wave_grid((const void *)cluster_cull_kernel, 256, 0, ncl, 256), 256, 0, st>>>(
      cl, ncl, cam, ds, live, qcount + 5);
  // one full wave each: the list lengths are known only on the device
  raster_cull_kernel<<<full_wave((const void *)raster_cull_kernel, 256, 0), 256, 0, st>>>(
      tv, ntri, cl, live, qcount + 5, cam, ds, vis, qcount + 1, clip, qcount + 4);
  raster_setup_kernel<<<full_wave((const void *)raster_setup_kernel, 256, 0), 256, 0, st>>>(
      tv, ntri, vis, qcount + 1, cam, ds, fb, rq);
  raster_clip_kernel<<<148, 128, 0, st>>>(tv, ntri, clip, qcount + 4, cam, ds, fb, rq);
  const int Wf = (cam.width + ds - 1) / ds;
  raster_medium_kernel<<<full_wave((const void *)raster_medium_kernel, 256, 0), 256, 0, st>>>(rq.queue, qcount, qcap,
                                                                                              Wf, fb);
  raster_huge_kernel<<<full_wave((const void *)raster_huge_kernel, 256, 0), 256, 0, st>>>(rq.queue, bands, qcount, qcap,
                                                                                          bcap, Wf, fb);
}

void launch_feedback_reduce(const uint64_t *fb, int64_t npix, uint32_t *dst, uint8_t *direct, cudaStream_t st) {
  reduce_kernel<<<wave_grid((const void *)reduce_kernel, 256, 0, npix, 256), 256, 0, st>>>(fb, npix, dst, direct);
}

void launch_feedback_links(const uint32_t *dreq, int64_t NP, const int64_t *link_ptr, const int32_t *link_col,
                           uint32_t *req, cudaStream_t st) {
  link_kernel<<<wave_grid((const void *)link_kernel, 256, 0, NP, 256), 256, 0, st>>>(dreq, NP, link_ptr, link_col, req);
}

void launch_request_all(uint32_t *req, uint8_t *direct, int64_t NP, cudaStream_t st) {
  int64_t b = (NP + 255) / 256;
  if (b > 148 * 4) b = 148 * 4;
  request_all_kernel<<<(unsigned)(b > 0 ? b : 1), 256, 0, st>>>(req, direct, NP);
}

int64_t build_clusters(const float *verts, const int32_t *tris, const int32_t *face_page, int64_t ntri, int64_t NP,
                       float *tv_out, Cluster *cl_out) {
  // stable counting sort by page (ids outside [0, NP) sort last, together)
  std::vector<int64_t> start((size_t)NP + 2, 0);
  auto bucket = [&](int64_t t) { const int32_t p = face_page[t]; return (p >= 0 && p < NP) ? (int64_t)p : NP; };
  for (int64_t t = 0; t < ntri; ++t) ++start[(size_t)bucket(t) + 1];
  for (int64_t b = 0; b <= NP; ++b) start[(size_t)b + 1] += start[(size_t)b];
  std::vector<int64_t> pos(start.begin(), start.end() - 1);
  std::vector<int64_t> order((size_t)ntri);
  for (int64_t t = 0; t < ntri; ++t) order[(size_t)pos[(size_t)bucket(t)]++] = t;
  // vertex c of sorted triangle k at tv_out[4 * (c * ntri + k)], page id bits in w of vertex 0
  for (int64_t k = 0; k < ntri; ++k) {
    const int64_t t = order[(size_t)k];
    for (int c = 0; c < 3; ++c) {
      const float *p = verts + 3 * (int64_t)tris[3 * t + c];
      float *o = tv_out + 4 * ((int64_t)c * ntri + k);
      o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
      o[3] = 0.0f;
      if (c == 0) std::memcpy(o + 3, face_page + t, 4);
    }
  }
  int64_t ncl = 0;
  for (int64_t b = 0; b <= NP; ++b) {
    for (int64_t k0 = start[(size_t)b]; k0 < start[(size_t)b + 1]; k0 += 32) {
      const int64_t k1 = std::min(k0 + 32, start[(size_t)b + 1]);
      Cluster c;
      for (int a = 0; a < 3; ++a) { c.lo[a] = INFINITY; c.hi[a] = -INFINITY; }
      for (int64_t k = k0; k < k1; ++k)
        for (int v = 0; v < 3; ++v) {
          const float *p = tv_out + 4 * ((int64_t)v * ntri + k);
          for (int a = 0; a < 3; ++a) { c.lo[a] = std::min(c.lo[a], p[a]); c.hi[a] = std::max(c.hi[a], p[a]); }
        }
      c.first = (uint32_t)k0;
      c.count = (uint32_t)(k1 - k0);
      cl_out[ncl++] = c;
    }
  }
  return ncl;
}

}  // namespace vm
