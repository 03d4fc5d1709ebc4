/*
 * ORACLE (test infrastructure only): the page-determination pass of the
 * per-frame path (Sec. 4.1 "Page Determination" and the evaluation's
 * "Page determination details"): the proxy mesh is rendered with per-face
 * page IDs into a low-resolution visibility buffer, which is reduced to one
 * "required + nearest depth" word per page with atomic-max semantics, linked
 * pages receiving the same value, and compacted into the ordered request
 * list.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code with the CUDA library.
 *
 * The paper rasterises with graphics hardware and states none of the
 * raster conventions, so the following readings define the result exactly
 * (all FP32 operations correctly rounded, compiled with -ffp-contract=off):
 *  - vertices go to camera space with the same row dot products as the
 *    splat projection; triangles crossing z = 0.2 are clipped against that
 *    plane (Sutherland-Hodgman), the polygon fanned from its first vertex;
 *  - feedback intrinsics are fx/ds, fy/ds, cx/ds, cy/ds; the buffer is
 *    ceil(W/ds) x ceil(H/ds);
 *  - screen positions are clamped to +-4e6 px and snapped to 1/256 px with
 *    round-half-even; coverage uses 64-bit integer edge functions at pixel
 *    centres (i+1/2, j+1/2) with a top-left style ownership rule so that an
 *    edge shared by two triangles covers each pixel once; both windings draw;
 *  - depth at a covered pixel is the perspective-correct z: 1/z is affine
 *    in screen space, so with w_k = 1/z_k per vertex,
 *    z = float(E_sum) / ((float(E_0) w_0 + float(E_1) w_1) + float(E_2) w_2),
 *    E_sum = E_0 + E_1 + E_2 being twice the snapped area;
 *  - the buffer keeps, per pixel, the minimum of (bits(z) << 32) | (page+1),
 *    faces without a page writing 0 in the low word (they occlude but
 *    request nothing); an untouched pixel holds all ones;
 *  - the request word is 0xFFFFFFFF - bits(z): it decreases with depth and
 *    is non-zero for every finite z > 0, zero meaning "not required".
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ZNEAR 0.2f
#define GUARD 4.0e6f

typedef struct {
  float view[12];
  float campos[3];
  float fx, fy, cx, cy;
  int32_t width, height, tile_w, tile_h;
} vo_camera;

static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

static int64_t floordiv(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}

typedef struct { float x, y, z; } v3;

static v3 to_cam(const float *V, const float *p) {
  v3 r;
  r.x = ((V[0] * p[0] + V[1] * p[1]) + V[2] * p[2]) + V[3];
  r.y = ((V[4] * p[0] + V[5] * p[1]) + V[6] * p[2]) + V[7];
  r.z = ((V[8] * p[0] + V[9] * p[1]) + V[10] * p[2]) + V[11];
  return r;
}

/* *dst = min(*dst, key), atomically: triangles may be rasterised by several
 * threads at once, and a minimum does not depend on their order */
static void min_store(uint64_t *dst, uint64_t key) {
  uint64_t cur = __atomic_load_n(dst, __ATOMIC_RELAXED);
  while (key < cur && !__atomic_compare_exchange_n(dst, &cur, key, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
  }
}

/* edge a->b owns pixels exactly on it when it points up, or right when flat */
static int owns(int64_t dx, int64_t dy) { return dy < 0 || (dy == 0 && dx > 0); }

static void raster_tri(const v3 *c, uint32_t page1, float fxf, float fyf, float cxf, float cyf, int Wf, int Hf,
                       uint64_t *buf) {
  int64_t X[3], Y[3];
  float Z[3];
  for (int k = 0; k < 3; ++k) {
    float xs = fxf * (c[k].x / c[k].z) + cxf;
    float ys = fyf * (c[k].y / c[k].z) + cyf;
    xs = fminf(fmaxf(xs, -GUARD), GUARD);
    ys = fminf(fmaxf(ys, -GUARD), GUARD);
    X[k] = (int64_t)nearbyintf(xs * 256.0f);
    Y[k] = (int64_t)nearbyintf(ys * 256.0f);
    Z[k] = c[k].z;
  }
  int64_t area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
  if (area == 0) return;
  if (area < 0) {
    int64_t t; float tf;
    t = X[1]; X[1] = X[2]; X[2] = t;
    t = Y[1]; Y[1] = Y[2]; Y[2] = t;
    tf = Z[1]; Z[1] = Z[2]; Z[2] = tf;
    area = -area;
  }
  int64_t xmin = X[0], xmax = X[0], ymin = Y[0], ymax = Y[0];
  for (int k = 1; k < 3; ++k) {
    if (X[k] < xmin) xmin = X[k];
    if (X[k] > xmax) xmax = X[k];
    if (Y[k] < ymin) ymin = Y[k];
    if (Y[k] > ymax) ymax = Y[k];
  }
  int64_t i0 = floordiv(xmin - 128 + 255, 256), i1 = floordiv(xmax - 128, 256);
  int64_t j0 = floordiv(ymin - 128 + 255, 256), j1 = floordiv(ymax - 128, 256);
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 > Wf - 1) i1 = Wf - 1;
  if (j1 > Hf - 1) j1 = Hf - 1;
  /* edge k is opposite vertex k: edge0 = v1->v2, edge1 = v2->v0, edge2 = v0->v1 */
  const int ea[3] = {1, 2, 0}, eb[3] = {2, 0, 1};
  int own[3];
  for (int k = 0; k < 3; ++k) own[k] = owns(X[eb[k]] - X[ea[k]], Y[eb[k]] - Y[ea[k]]);
  const float farea = (float)area;
  const float w0 = 1.0f / Z[0], w1 = 1.0f / Z[1], w2 = 1.0f / Z[2];
  for (int64_t j = j0; j <= j1; ++j)
    for (int64_t i = i0; i <= i1; ++i) {
      int64_t px = i * 256 + 128, py = j * 256 + 128;
      int64_t E[3];
      int in = 1;
      for (int k = 0; k < 3; ++k) {
        int64_t a = ea[k], b = eb[k];
        E[k] = (X[b] - X[a]) * (py - Y[a]) - (Y[b] - Y[a]) * (px - X[a]);
        if (!(E[k] > 0 || (E[k] == 0 && own[k]))) { in = 0; break; }
      }
      if (!in) continue;
      float s = ((float)E[0] * w0 + (float)E[1] * w1) + (float)E[2] * w2;
      float zp = farea / s;
      uint64_t key = ((uint64_t)fbits(zp) << 32) | page1;
      min_store(buf + j * Wf + i, key);
    }
}

/*
 * Rasterises n_tris proxy triangles (vertex indices tris[3t..3t+2] into
 * verts[3v..3v+2], page face_page[t], -1 = none) into buf[Hf][Wf], which the
 * caller fills with all ones beforehand.  Triangles are independent (the
 * per-pixel minimum is order-free), so they may run on several OpenMP threads
 * (vo_set_threads); one thread by default.
 */
void vo_feedback_raster(int64_t n_tris, const float *verts, const int32_t *tris, const int32_t *face_page,
                        const vo_camera *cam, int ds, uint64_t *buf) {
  const int Wf = (cam->width + ds - 1) / ds, Hf = (cam->height + ds - 1) / ds;
  const float fds = (float)ds;
  const float fxf = cam->fx / fds, fyf = cam->fy / fds, cxf = cam->cx / fds, cyf = cam->cy / fds;
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t t = 0; t < n_tris; ++t) {
    v3 c[3];
    for (int k = 0; k < 3; ++k) c[k] = to_cam(cam->view, verts + 3 * (int64_t)tris[3 * t + k]);
    uint32_t page1 = (uint32_t)(face_page[t] + 1);
    int inside[3], nin = 0;
    for (int k = 0; k < 3; ++k) { inside[k] = c[k].z >= ZNEAR; nin += inside[k]; }
    if (nin == 0) continue;
    if (nin == 3) { raster_tri(c, page1, fxf, fyf, cxf, cyf, Wf, Hf, buf); continue; }
    v3 poly[4];
    int m = 0;
    for (int k = 0; k < 3; ++k) {
      v3 a = c[k], b = c[(k + 1) % 3];
      int ia = inside[k], ib = inside[(k + 1) % 3];
      if (ia) poly[m++] = a;
      if (ia != ib) {
        float t = (ZNEAR - a.z) / (b.z - a.z);
        v3 p;
        p.x = a.x + t * (b.x - a.x);
        p.y = a.y + t * (b.y - a.y);
        p.z = ZNEAR;
        poly[m++] = p;
      }
    }
    for (int k = 1; k + 1 < m; ++k) {
      v3 tri[3] = {poly[0], poly[k], poly[k + 1]};
      raster_tri(tri, page1, fxf, fyf, cxf, cyf, Wf, Hf, buf);
    }
  }
}

/*
 * Reduction: req[p] = max over pixels showing page p, and over pixels showing
 * any page q with a link q -> p (row q of the CSR link_ptr/link_col), of the
 * request word; direct[p] = 1 when a pixel shows p itself.  n_pixels words of
 * buf; req and direct are cleared here.
 */
void vo_feedback_reduce(int64_t n_pixels, const uint64_t *buf, int n_vp, const int64_t *link_ptr,
                        const int32_t *link_col, int use_links, uint32_t *req, uint8_t *direct) {
  memset(req, 0, sizeof(uint32_t) * (size_t)n_vp);
  memset(direct, 0, (size_t)n_vp);
  for (int64_t i = 0; i < n_pixels; ++i) {
    uint64_t key = buf[i];
    if (key == ~0ull) continue;
    uint32_t page1 = (uint32_t)(key & 0xFFFFFFFFu);
    if (page1 == 0) continue;
    uint32_t p = page1 - 1;
    uint32_t enc = 0xFFFFFFFFu - (uint32_t)(key >> 32);
    if (enc > req[p]) req[p] = enc;
    direct[p] = 1;
    if (use_links)
      for (int64_t k = link_ptr[p]; k < link_ptr[p + 1]; ++k) {
        uint32_t q = (uint32_t)link_col[k];
        if (enc > req[q]) req[q] = enc;
      }
  }
}

/* ordered request list: ascending page id of every p with req[p] != 0 */
int vo_compact(int n_vp, const uint32_t *req, const uint8_t *direct, int32_t *out_page, uint32_t *out_enc,
               uint8_t *out_direct) {
  int m = 0;
  for (int p = 0; p < n_vp; ++p)
    if (req[p] != 0) {
      out_page[m] = p;
      out_enc[m] = req[p];
      out_direct[m] = direct[p];
      ++m;
    }
  return m;
}

/* float bits helper for tests */
uint32_t vo_float_bits(float f) { return fbits(f); }
