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
// once; depth is perspective-correct z; the visibility word is
// (bits(z) << 32) | (page + 1), minimum per pixel, all ones when empty.
#include "renderer.cuh"

namespace vm {
namespace {

struct V3 { float x, y, z; };

__device__ __forceinline__ V3 to_cam(const float *V, const float *p) {
  V3 r;
  r.x = ((V[0] * p[0] + V[1] * p[1]) + V[2] * p[2]) + V[3];
  r.y = ((V[4] * p[0] + V[5] * p[1]) + V[6] * p[2]) + V[7];
  r.z = ((V[8] * p[0] + V[9] * p[1]) + V[10] * p[2]) + V[11];
  return r;
}

__device__ __forceinline__ int64_t floordiv256(int64_t a) { return a >= 0 ? a / 256 : -((-a + 255) / 256); }

__device__ __forceinline__ bool owns(int64_t dx, int64_t dy) { return dy < 0 || (dy == 0 && dx > 0); }

// A snapped, oriented (area > 0) triangle with its clamped pixel box.
struct Tri {
  int32_t X[3], Y[3];
  float Z[3];
  uint32_t page1;
  int32_t i0, i1, j0, j1;
};

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
  float b0 = __ll2float_rn(E[0]) / farea, b1 = __ll2float_rn(E[1]) / farea, b2 = __ll2float_rn(E[2]) / farea;
  float s = (b0 / t.Z[0] + b1 / t.Z[1]) + b2 / t.Z[2];
  float zp = 1.0f / s;
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

// Snaps and orients one (clipped) triangle; small ones are rasterised by the
// calling thread, larger ones go to the queue for whole-CTA rasterisation.
__device__ void setup_tri(const V3 *c, uint32_t page1, float fxf, float fyf, float cxf, float cyf, int Wf, int Hf,
                          uint64_t *fb, Tri *queue, uint32_t *qcount, uint32_t qcap) {
  // queue layout: medium triangles (17..1024 pixels) from the front, huge ones
  // (more) from the back; qcount[0], qcount[1] count them
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
  if (area == 0) return;
  if (area < 0) {
    int64_t t = X[1]; X[1] = X[2]; X[2] = t;
    t = Y[1]; Y[1] = Y[2]; Y[2] = t;
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
  if (i1 < i0 || j1 < j0) return;
  Tri t;
#pragma unroll
  for (int k = 0; k < 3; ++k) { t.X[k] = (int32_t)X[k]; t.Y[k] = (int32_t)Y[k]; t.Z[k] = Z[k]; }
  t.page1 = page1;
  t.i0 = (int32_t)i0; t.i1 = (int32_t)i1; t.j0 = (int32_t)j0; t.j1 = (int32_t)j1;
  const int64_t bw = i1 - i0 + 1, npx = bw * (j1 - j0 + 1);
  if (npx > 16) {
    const bool huge = npx > 1024;
    const uint32_t q = atomicAdd(qcount + (huge ? 1 : 0), 1u);
    if (q < qcap / 2) { queue[huge ? qcap - 1 - q : q] = t; return; }
  }
  int64_t dxe[3], dye[3];
  bool own[3];
  float farea;
  edges(t, dxe, dye, own, &farea);
  for (int64_t q = 0; q < npx; ++q) shade(t, dxe, dye, own, farea, i0 + q % bw, j0 + q / bw, Wf, fb);
}

// Pass 1: triangles entirely behind the near plane, or entirely more than 2
// pixels beyond one side of the buffer, cover no pixel centre; the others are
// appended (warp-aggregated) to a dense list so that pass 2 runs without idle
// lanes.
__global__ void __launch_bounds__(256) raster_cull_kernel(const float *verts, const int32_t *tris, int64_t ntri,
                                                          vm3dgs_camera cam, int ds, uint32_t *vis,
                                                          uint32_t *nvis) {
  const int Wf = (cam.width + ds - 1) / ds, Hf = (cam.height + ds - 1) / ds;
  const float fds = (float)ds;
  const float fxf = cam.fx / fds, fyf = cam.fy / fds, cxf = cam.cx / fds, cyf = cam.cy / fds;
  const float zn = 0.2f;
  const float kr = ((float)Wf + 2.0f - cxf) / fxf, kl = (-2.0f - cxf) / fxf;
  const float kb = ((float)Hf + 2.0f - cyf) / fyf, kt = (-2.0f - cyf) / fyf;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < ntri; base += stride) {
    const int64_t t = base + lane;
    bool keep = false;
    if (t < ntri) {
      V3 c[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) c[k] = to_cam(cam.view, verts + 3 * (int64_t)tris[3 * t + k]);
      int nin = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) nin += c[k].z >= zn;
      keep = nin > 0;
      if (nin == 3) {
        bool o1 = true, o2 = true, o3 = true, o4 = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          o1 = o1 && c[k].x > kr * c[k].z;
          o2 = o2 && c[k].x < kl * c[k].z;
          o3 = o3 && c[k].y > kb * c[k].z;
          o4 = o4 && c[k].y < kt * c[k].z;
        }
        keep = !(o1 || o2 || o3 || o4);
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    uint32_t off = 0;
    if (lane == 0 && m) off = atomicAdd(nvis, (uint32_t)__popc(m));
    off = __shfl_sync(0xffffffffu, off, 0);
    if (keep) vis[off + __popc(m & ((1u << lane) - 1u))] = (uint32_t)t;
  }
}

// Pass 2: clip, snap and rasterise the listed triangles (small ones here,
// larger ones queued).
__global__ void __launch_bounds__(256) raster_setup_kernel(const float *verts, const int32_t *tris,
                                                           const int32_t *face_page, const uint32_t *vis,
                                                           const uint32_t *nvis, vm3dgs_camera cam, int ds,
                                                           uint64_t *fb, Tri *queue, uint32_t *qcount, uint32_t qcap) {
  const int Wf = (cam.width + ds - 1) / ds, Hf = (cam.height + ds - 1) / ds;
  const float fds = (float)ds;
  const float fxf = cam.fx / fds, fyf = cam.fy / fds, cxf = cam.cx / fds, cyf = cam.cy / fds;
  const float zn = 0.2f;
  const int64_t n = *nvis;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int64_t t = vis[q];
    V3 c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = to_cam(cam.view, verts + 3 * (int64_t)tris[3 * t + k]);
    const uint32_t page1 = (uint32_t)(face_page[t] + 1);
    bool inside[3];
    int nin = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) { inside[k] = c[k].z >= zn; nin += inside[k]; }
    if (nin == 3) {
      setup_tri(c, page1, fxf, fyf, cxf, cyf, Wf, Hf, fb, queue, qcount, qcap);
      continue;
    }
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
      V3 tri[3] = {poly[0], poly[k], poly[k + 1]};
      setup_tri(tri, page1, fxf, fyf, cxf, cyf, Wf, Hf, fb, queue, qcount, qcap);
    }
  }
}

// medium triangles: one warp each, lanes over the pixel box
__global__ void __launch_bounds__(256) raster_medium_kernel(const Tri *queue, const uint32_t *qcount, uint32_t qcap,
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
    const int64_t bw = t.i1 - t.i0 + 1, npx = bw * (t.j1 - t.j0 + 1);
    for (int64_t p = lane; p < npx; p += 32) shade(t, dxe, dye, own, farea, t.i0 + p % bw, t.j0 + p / bw, Wf, fb);
  }
}

// huge triangles: one CTA each, threads over the pixel box
__global__ void __launch_bounds__(256) raster_huge_kernel(const Tri *queue, const uint32_t *qcount, uint32_t qcap,
                                                          int Wf, uint64_t *fb) {
  const uint32_t n = min(qcount[1], qcap / 2);
  for (uint32_t q = blockIdx.x; q < n; q += gridDim.x) {
    const Tri t = queue[qcap - 1 - q];
    int64_t dxe[3], dye[3];
    bool own[3];
    float farea;
    edges(t, dxe, dye, own, &farea);
    const int64_t bw = t.i1 - t.i0 + 1, npx = bw * (t.j1 - t.j0 + 1);
    for (int64_t p = threadIdx.x; p < npx; p += blockDim.x) shade(t, dxe, dye, own, farea, t.i0 + p % bw, t.j0 + p / bw, Wf, fb);
  }
}

__global__ void clear_kernel(uint64_t *fb, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) fb[i] = ~0ull;
}

__global__ void __launch_bounds__(256) reduce_kernel(const uint64_t *fb, int64_t npix, const int64_t *link_ptr,
                                                     const int32_t *link_col, int links, uint32_t *req, uint8_t *direct) {
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
    atomicMax(req + page, mx);
    direct[page] = 1;
    if (links)
      for (int64_t k = link_ptr[page]; k < link_ptr[page + 1]; ++k) atomicMax(req + link_col[k], mx);
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

void launch_feedback_clear(uint64_t *fb, int64_t n, cudaStream_t st) {
  int64_t b = (n + 255) / 256;
  if (b > 148 * 8) b = 148 * 8;
  clear_kernel<<<(unsigned)(b > 0 ? b : 1), 256, 0, st>>>(fb, n);
}

void launch_feedback_raster(const float *verts, const int32_t *tris, const int32_t *face_page, int64_t ntri,
                            const vm3dgs_camera &cam, int ds, uint64_t *fb, void *queue, uint32_t *qcount,
                            uint32_t qcap, uint32_t *vis, cudaStream_t st) {
  if (ntri <= 0) return;
  // qcount[0..1]: queued medium / huge triangles, qcount[2]: listed triangles
  cudaMemsetAsync(qcount, 0, 3 * sizeof(uint32_t), st);
  int64_t blocks = (ntri + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  raster_cull_kernel<<<(unsigned)blocks, 256, 0, st>>>(verts, tris, ntri, cam, ds, vis, qcount + 2);
  raster_setup_kernel<<<148 * 4, 256, 0, st>>>(verts, tris, face_page, vis, qcount + 2, cam, ds, fb,
                                               reinterpret_cast<Tri *>(queue), qcount, qcap);
  const int Wf = (cam.width + ds - 1) / ds;
  raster_medium_kernel<<<148 * 4, 256, 0, st>>>(reinterpret_cast<const Tri *>(queue), qcount, qcap, Wf, fb);
  raster_huge_kernel<<<148 * 2, 256, 0, st>>>(reinterpret_cast<const Tri *>(queue), qcount, qcap, Wf, fb);
}

void launch_feedback_reduce(const uint64_t *fb, int64_t npix, const int64_t *link_ptr, const int32_t *link_col,
                            int links, uint32_t *req, uint8_t *direct, cudaStream_t st) {
  int64_t b = (npix + 255) / 256;
  if (b > 148 * 8) b = 148 * 8;
  reduce_kernel<<<(unsigned)(b > 0 ? b : 1), 256, 0, st>>>(fb, npix, link_ptr, link_col, links, req, direct);
}

void launch_request_all(uint32_t *req, uint8_t *direct, int64_t NP, cudaStream_t st) {
  int64_t b = (NP + 255) / 256;
  if (b > 148 * 4) b = 148 * 4;
  request_all_kernel<<<(unsigned)(b > 0 ? b : 1), 256, 0, st>>>(req, direct, NP);
}

}  // namespace vm
