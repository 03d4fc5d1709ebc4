/*
 * ORACLE (test infrastructure only): plain, slow, single-threaded reference of
 * the splatting half of the per-frame path.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code with
 * the CUDA library.
 *
 * The paper renders with the 3DGS math of Kerbl et al. and does not restate
 * it (Sec. 4.2 "Rendering"; it defers to Kerbl for the per-Gaussian vertex
 * math, the per-fragment Gaussian and alpha blending).  This file therefore
 * writes out that math with the constants of the 3DGS reference renderer,
 * each one a stated reading:
 *   near plane 0.2, guard band 1.3, low-pass dilation 0.3, 3-sigma radius,
 *   eigenvalue floor 0.1, alpha cap 0.99, alpha skip 1/255, transmittance
 *   stop 1e-4, colour offset 0.5 clamped at 0, pixel centres at (i+.5, j+.5).
 *
 * Precision contract.  Every DISCRETE result (cull flag, radius, tile
 * rectangle, depth key) is defined by an FP32 formula of correctly rounded
 * operations in the exact order written below; this file must be compiled
 * with -ffp-contract=off so no multiply-add is fused.  CONTINUOUS results
 * (centre, conic, colour, alpha, transmittance, image) are computed in FP64.
 *
 * Tie order of the sort: (tile, depth bits, virtual Gaussian id), the id
 * being page * page_size + slot of the level the page is drawn at.
 *
 * Tiles of a splat (binning is left to the 3DGS renderer; this is a reading).
 * A splat is binned to the tiles of its rectangle whose box of pixel centres
 * meets its 3-sigma ellipse E = {d : ia dx^2 + 2 ib dx dy + ic dy^2 <= 9}
 * (d = pixel - centre, the FP32 conic), for rectangles of any size.  The test
 * is taken one tile row at a time, since a convex region cut by the row's
 * band of pixel-centre y values is an x-interval:
 *   D   = ia ic - ib^2 (the conic's determinant; if it is not positive the
 *         splat keeps every tile of its rectangle)
 *   ey  = sqrt(9 ia / D)           half the y-extent of E
 *   dys = -3 ib / sqrt(ic D)       dy of E's rightmost point (-dys: leftmost)
 *   band [l, h] = [yl - pv, yh - pv] clipped to [-ey, ey]; empty: no tile
 *   X1 = x_hi(clamp(dys, l, h)),  X0 = x_lo(clamp(-dys, l, h)), where
 *   x_hi/lo(t) = (-ib t +/- sqrt(max(0, 9 ia - D t^2))) / ia
 *         are E's right and left boundary at height t (x_hi is concave and
 *         peaks at dys, x_lo convex with its minimum at -dys, so X0 and X1
 *         bound E within the band)
 *   a tile column is kept when xl - pu <= X1 and xh - pu >= X0
 * ([xl, xh] x [yl, yh] is the tile's box of pixel centres).  Every operation
 * is one FP32 operation in the order written in tile_kept().  The kept tiles
 * of a row are contiguous.  With rect_binning the splat keeps every tile of
 * its rectangle instead (the 3DGS reference renderer's binning), for
 * measuring what the ellipse test changes.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ZNEAR 0.2f

typedef struct {
  float view[12]; /* rows of [R|t], world -> camera, OpenCV axes */
  float campos[3];
  float fx, fy, cx, cy;
  int32_t width, height, tile_w, tile_h;
} vo_camera;

static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* Is tile (tx, ty) one of the splat's?  The row rule stated above, FP32
 * spec; (pu, pv) is the FP32 centre and (ia, ib, ic) the FP32 conic. */
static int tile_kept(float pu, float pv, float ia, float ib, float ic, const vo_camera *cam, int tx, int ty) {
  const float D = ia * ic - ib * ib;
  if (!(D > 0.0f)) return 1;
  const float ey = sqrtf((9.0f * ia) / D);
  const float dys = -(3.0f * ib) / sqrtf(ic * D);
  const int py1 = (ty + 1) * cam->tile_h < cam->height ? (ty + 1) * cam->tile_h : cam->height;
  const int px1 = (tx + 1) * cam->tile_w < cam->width ? (tx + 1) * cam->tile_w : cam->width;
  const float yl = (float)(ty * cam->tile_h) + 0.5f, yh = (float)py1 - 0.5f;
  const float xl = (float)(tx * cam->tile_w) + 0.5f, xh = (float)px1 - 0.5f;
  const float l = fmaxf(yl - pv, -ey), h = fminf(yh - pv, ey);
  if (l > h) return 0;
  const float t1 = fminf(fmaxf(dys, l), h), t0 = fminf(fmaxf(-dys, l), h);
  const float s1 = sqrtf(fmaxf(0.0f, 9.0f * ia - D * (t1 * t1)));
  const float s0 = sqrtf(fmaxf(0.0f, 9.0f * ia - D * (t0 * t0)));
  const float X1 = (-(ib * t1) + s1) / ia;
  const float X0 = (-(ib * t0) - s0) / ia;
  return (xl - pu) <= X1 && (xh - pu) >= X0;
}

/* Threads of the OpenMP loops of the oracle (projection per Gaussian, blend
 * per tile, feedback raster per triangle: independent iterations, so the
 * results do not depend on the count).  One thread unless set. */
void vo_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int vo_max_threads(void) { return omp_get_max_threads(); }

int vo_tile_kept(float pu, float pv, float ia, float ib, float ic, const vo_camera *cam, int tx, int ty) {
  return tile_kept(pu, pv, ia, ib, ic, cam, tx, ty);
}

/* real spherical harmonics up to degree 3, constants from their definition
 * N_lm = sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) with the sqrt(2) of the real
 * basis, Condon-Shortley phase included; evaluated on the unit direction d.
 * Order of the 16 functions: l = 0..3, m = -l..l. */
static void sh_basis(const double d[3], double *Y) {
  const double pi = 3.14159265358979323846;
  double x = d[0], y = d[1], z = d[2];
  double xx = x * x, yy = y * y, zz = z * z;
  double c0 = sqrt(1.0 / (4 * pi));
  double c1 = sqrt(3.0 / (4 * pi));
  double c2a = sqrt(15.0 / (4 * pi));     /* xy, yz, xz */
  double c2b = sqrt(5.0 / (16 * pi));     /* 3z^2-1 = 2zz-xx-yy */
  double c2c = sqrt(15.0 / (16 * pi));    /* xx-yy */
  double c3a = sqrt(35.0 / (32 * pi));    /* y(3xx-yy), x(xx-3yy) */
  double c3b = sqrt(105.0 / (4 * pi));    /* xyz */
  double c3c = sqrt(21.0 / (32 * pi));    /* y(4zz-xx-yy), x(...) */
  double c3d = sqrt(7.0 / (16 * pi));     /* z(2zz-3xx-3yy) */
  double c3e = sqrt(105.0 / (16 * pi));   /* z(xx-yy) */
  Y[0] = c0;
  Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
  Y[4] = c2a * x * y; Y[5] = -c2a * y * z; Y[6] = c2b * (2 * zz - xx - yy);
  Y[7] = -c2a * x * z; Y[8] = c2c * (xx - yy);
  Y[9] = -c3a * y * (3 * xx - yy); Y[10] = c3b * x * y * z;
  Y[11] = -c3c * y * (4 * zz - xx - yy); Y[12] = c3d * z * (2 * zz - 3 * xx - 3 * yy);
  Y[13] = -c3c * x * (4 * zz - xx - yy); Y[14] = c3e * z * (xx - yy);
  Y[15] = -c3a * x * (xx - 3 * yy);
}

void vo_sh_basis(int64_t n, const double *dirs, double *out) {
  for (int64_t i = 0; i < n; ++i) sh_basis(dirs + 3 * i, out + 16 * i);
}

/*
 * Per-Gaussian projection.
 * Inputs: decoded Gaussians (pos, scale, unit quaternion (w,x,y,z), opacity,
 * sh [n][K][3]), camera.  Outputs, fp32-spec: vis, radius, rect (x0,y0,x1,y1
 * half-open tile range), depth (view z), touched.  Outputs, fp64: centre (u,v),
 * conic (A,B,C) with power = -1/2 (A dx^2 + C dy^2) - B dx dy, rgb.
 */
void vo_project(int64_t n, const float *pos, const float *scale, const float *rot, const float *opac,
                const float *sh, int K, const vo_camera *cam, uint8_t *vis, float *radius, int32_t *rect,
                float *depth, int32_t *touched, float *ctr32, float *con32, int rect_binning, double *centre,
                double *conic, double *rgb) {
  const float *V = cam->view;
  const int gx = (cam->width + cam->tile_w - 1) / cam->tile_w;
  const int gy = (cam->height + cam->tile_h - 1) / cam->tile_h;
  const float TW = (float)cam->tile_w, TH = (float)cam->tile_h;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    vis[i] = 0; radius[i] = 0; touched[i] = 0; depth[i] = 0;
    ctr32[2 * i] = ctr32[2 * i + 1] = 0; con32[3 * i] = con32[3 * i + 1] = con32[3 * i + 2] = 0;
    rect[4 * i + 0] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
    const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    const float o = opac[i];
    /* ---- fp32 spec: view transform and cull */
    float tx = ((V[0] * x + V[1] * y) + V[2] * z) + V[3];
    float ty = ((V[4] * x + V[5] * y) + V[6] * z) + V[7];
    float tz = ((V[8] * x + V[9] * y) + V[10] * z) + V[11];
    if (!(o > 0.0f) || !(tz > ZNEAR)) continue;
    /* ---- fp32 spec: 3D covariance Sigma = (R S)(R S)^T */
    const float qw = rot[4 * i], qx = rot[4 * i + 1], qy = rot[4 * i + 2], qz = rot[4 * i + 3];
    float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    float xy = qx * qy, xz = qx * qz, yz = qy * qz;
    float wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz); R[0][1] = 2.0f * (xy - wz); R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz); R[1][1] = 1.0f - 2.0f * (xx + zz); R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy); R[2][1] = 2.0f * (yz + wx); R[2][2] = 1.0f - 2.0f * (xx + yy);
    float M[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[r][c] = R[r][c] * scale[3 * i + c];
    float S[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) S[r][c] = (M[r][0] * M[c][0] + M[r][1] * M[c][1]) + M[r][2] * M[c][2];
    /* ---- fp32 spec: EWA Jacobian with guard-band clamp */
    float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
    float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
    float txtz = tx / tz, tytz = ty / tz;
    float clx = fminf(limx, fmaxf(-limx, txtz)) * tz;
    float cly = fminf(limy, fmaxf(-limy, tytz)) * tz;
    float tz2 = tz * tz;
    float J00 = cam->fx / tz, J02 = -(cam->fx * clx) / tz2;
    float J11 = cam->fy / tz, J12 = -(cam->fy * cly) / tz2;
    float T0[3], T1[3];
    for (int c = 0; c < 3; ++c) {
      T0[c] = J00 * V[c] + J02 * V[8 + c];
      T1[c] = J11 * V[4 + c] + J12 * V[8 + c];
    }
    float u[3], w[3];
    for (int r = 0; r < 3; ++r) {
      u[r] = (S[r][0] * T0[0] + S[r][1] * T0[1]) + S[r][2] * T0[2];
      w[r] = (S[r][0] * T1[0] + S[r][1] * T1[1]) + S[r][2] * T1[2];
    }
    float a = (T0[0] * u[0] + T0[1] * u[1]) + T0[2] * u[2];
    float b = (T1[0] * u[0] + T1[1] * u[1]) + T1[2] * u[2];
    float c = (T1[0] * w[0] + T1[1] * w[1]) + T1[2] * w[2];
    a = a + 0.3f;
    c = c + 0.3f;
    float det = fmaxf(a * c - b * b, 1e-12f);
    /* ---- fp32 spec: radius, centre, tile rectangle */
    float mid = 0.5f * (a + c);
    float disc = fmaxf(0.1f, mid * mid - det);
    float lam = mid + sqrtf(disc);
    float r = ceilf(3.0f * sqrtf(lam));
    float pu = cam->fx * txtz + cam->cx;
    float pv = cam->fy * tytz + cam->cy;
    float fx0 = floorf((pu - r) / TW), fx1 = floorf((pu + r) / TW) + 1.0f;
    float fy0 = floorf((pv - r) / TH), fy1 = floorf((pv + r) / TH) + 1.0f;
    fx0 = fminf(fmaxf(fx0, 0.0f), (float)gx); fx1 = fminf(fmaxf(fx1, 0.0f), (float)gx);
    fy0 = fminf(fmaxf(fy0, 0.0f), (float)gy); fy1 = fminf(fmaxf(fy1, 0.0f), (float)gy);
    int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
    if (x0 >= x1 || y0 >= y1) continue;
    vis[i] = 1;
    radius[i] = r;
    rect[4 * i + 0] = x0; rect[4 * i + 1] = y0; rect[4 * i + 2] = x1; rect[4 * i + 3] = y1;
    depth[i] = tz;
    /* ---- fp32 spec: conic and the tiles the 3-sigma ellipse meets */
    {
      const float ia = c / det, ib = -b / det, ic = a / det;
      ctr32[2 * i] = pu; ctr32[2 * i + 1] = pv;
      con32[3 * i] = ia; con32[3 * i + 1] = ib; con32[3 * i + 2] = ic;
      int cnt = 0;
      for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) cnt += rect_binning || tile_kept(pu, pv, ia, ib, ic, cam, tx, ty);
      touched[i] = cnt;
    }

    /* ---- fp64: continuous outputs */
    double X = x, Y = y, Z = z;
    double dtx = ((double)V[0] * X + (double)V[1] * Y) + (double)V[2] * Z + (double)V[3];
    double dty = ((double)V[4] * X + (double)V[5] * Y) + (double)V[6] * Z + (double)V[7];
    double dtz = ((double)V[8] * X + (double)V[9] * Y) + (double)V[10] * Z + (double)V[11];
    double dqw = qw, dqx = qx, dqy = qy, dqz = qz;
    double Rd[3][3];
    Rd[0][0] = 1 - 2 * (dqy * dqy + dqz * dqz); Rd[0][1] = 2 * (dqx * dqy - dqw * dqz); Rd[0][2] = 2 * (dqx * dqz + dqw * dqy);
    Rd[1][0] = 2 * (dqx * dqy + dqw * dqz); Rd[1][1] = 1 - 2 * (dqx * dqx + dqz * dqz); Rd[1][2] = 2 * (dqy * dqz - dqw * dqx);
    Rd[2][0] = 2 * (dqx * dqz - dqw * dqy); Rd[2][1] = 2 * (dqy * dqz + dqw * dqx); Rd[2][2] = 1 - 2 * (dqx * dqx + dqy * dqy);
    double Sd[3][3];
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += Rd[p][k] * Rd[q][k] * (double)scale[3 * i + k] * (double)scale[3 * i + k];
        Sd[p][q] = s;
      }
    double dlimx = 1.3 * (0.5 * cam->width / (double)cam->fx), dlimy = 1.3 * (0.5 * cam->height / (double)cam->fy);
    double dcx = fmin(dlimx, fmax(-dlimx, dtx / dtz)) * dtz, dcy = fmin(dlimy, fmax(-dlimy, dty / dtz)) * dtz;
    double Jd[2][3] = {{cam->fx / dtz, 0, -cam->fx * dcx / (dtz * dtz)}, {0, cam->fy / dtz, -cam->fy * dcy / (dtz * dtz)}};
    double Td[2][3];
    for (int p = 0; p < 2; ++p)
      for (int q = 0; q < 3; ++q) Td[p][q] = Jd[p][0] * V[q] + Jd[p][1] * V[4 + q] + Jd[p][2] * V[8 + q];
    double C2[2][2];
    for (int p = 0; p < 2; ++p)
      for (int q = 0; q < 2; ++q) {
        double s = 0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) s += Td[p][k] * Sd[k][l] * Td[q][l];
        C2[p][q] = s;
      }
    double A = C2[0][0] + 0.3, B = C2[0][1], Cc = C2[1][1] + 0.3;
    double dd = fmax(A * Cc - B * B, 1e-12);
    conic[3 * i + 0] = Cc / dd;
    conic[3 * i + 1] = -B / dd;
    conic[3 * i + 2] = A / dd;
    centre[2 * i + 0] = cam->fx * (dtx / dtz) + cam->cx;
    centre[2 * i + 1] = cam->fy * (dty / dtz) + cam->cy;
    double dir[3] = {X - cam->campos[0], Y - cam->campos[1], Z - cam->campos[2]};
    double nn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    dir[0] /= nn; dir[1] /= nn; dir[2] /= nn;
    double Yb[16];
    sh_basis(dir, Yb);
    for (int ch = 0; ch < 3; ++ch) {
      double s = 0;
      for (int k = 0; k < K; ++k) s += (double)sh[((int64_t)i * K + k) * 3 + ch] * Yb[k];
      s += 0.5;
      rgb[3 * i + ch] = s > 0 ? s : 0;
    }
  }
}

/* ---------------------------------------------------------------- bin + sort */
typedef struct { uint64_t key; int64_t vid; int64_t idx; } vo_pair;

static int cmp_pair(const void *pa, const void *pb) {
  const vo_pair *a = pa, *b = pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->vid != b->vid) return a->vid < b->vid ? -1 : 1;
  return 0;
}

/* Emits one (tile << 32 | depth bits) key per (visible splat, kept tile of
 * its rectangle, row-major) and sorts by (key, virtual id).  Returns the number
 * of pairs, or -needed when cap is too small. */
int64_t vo_bin_sort(int64_t n, const uint8_t *vis, const int32_t *rect, const int32_t *touched, const float *ctr32,
                    const float *con32, int rect_binning, const float *depth, const int64_t *vid,
                    const vo_camera *cam, uint64_t *keys_out, int64_t *idx_out, int64_t cap) {
  const int gx = (cam->width + cam->tile_w - 1) / cam->tile_w;
  int64_t M = 0;
  for (int64_t i = 0; i < n; ++i)
    if (vis[i]) M += touched[i];
  if (M > cap) return -M;
  vo_pair *p = (vo_pair *)malloc(sizeof(vo_pair) * (M > 0 ? M : 1));
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!vis[i]) continue;
    for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
      for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
        if (!rect_binning && !tile_kept(ctr32[2 * i], ctr32[2 * i + 1], con32[3 * i], con32[3 * i + 1],
                                        con32[3 * i + 2], cam, tx, ty))
          continue;
        if (k == M) { free(p); return -(M + 1); } /* touched disagrees with the rule */
        uint64_t tile = (uint64_t)ty * gx + tx;
        p[k].key = (tile << 32) | fbits(depth[i]);
        p[k].vid = vid[i];
        p[k].idx = i;
        ++k;
      }
  }
  qsort(p, M, sizeof(vo_pair), cmp_pair);
  for (int64_t j = 0; j < M; ++j) { keys_out[j] = p[j].key; idx_out[j] = p[j].idx; }
  free(p);
  return k == M ? M : -(M + 1);
}

/* [start, end) of every tile in the sorted key list */
void vo_ranges(int64_t M, const uint64_t *keys, int n_tiles, int64_t *ranges) {
  for (int t = 0; t < n_tiles; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
  for (int64_t j = 0; j < M; ++j) {
    uint64_t t = keys[j] >> 32;
    if (j == 0 || (keys[j - 1] >> 32) != t) ranges[2 * t] = j;
    if (j == M - 1 || (keys[j + 1] >> 32) != t) ranges[2 * t + 1] = j + 1;
  }
}

/*
 * Front-to-back blending per pixel in FP64.  img is [3][H][W]; flag[p] = 1
 * marks pixels where an alpha came within 2e-6 of the 1/255 skip threshold or
 * the transmittance test came within 2e-7 of 1e-4, i.e. where an FP32
 * evaluation may legitimately take the other branch (an FP32 alpha near the
 * threshold carries an error of about 2e-7 from the centre and exponent;
 * transmittance accumulates about 1e-3 relative error over a pixel).  bg is the background
 * colour added with the final transmittance.
 */
void vo_blend(const vo_camera *cam, const int64_t *ranges, const int64_t *idx, const double *centre,
              const double *conic, const float *opac, const double *rgb, const double *bg, double *img,
              uint8_t *flag, int32_t *n_contrib) {
  const int W = cam->width, H = cam->height, TW = cam->tile_w, TH = cam->tile_h;
  const int gx = (W + TW - 1) / TW, gy = (H + TH - 1) / TH;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int ty = 0; ty < gy; ++ty)
    for (int tx = 0; tx < gx; ++tx) {
      const int64_t s = ranges[2 * (ty * gx + tx)], e = ranges[2 * (ty * gx + tx) + 1];
      for (int py = ty * TH; py < (ty + 1) * TH && py < H; ++py)
        for (int px = tx * TW; px < (tx + 1) * TW && px < W; ++px) {
          double T = 1.0, C[3] = {0, 0, 0};
          int fl = 0, nc = 0;
          for (int64_t j = s; j < e; ++j) {
            const int64_t g = idx[j];
            double dx = centre[2 * g] - (px + 0.5), dy = centre[2 * g + 1] - (py + 0.5);
            double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
            if (power > 0) continue;
            double alpha = fmin(0.99, (double)opac[g] * exp(power));
            if (fabs(alpha - 1.0 / 255.0) < 2e-6) fl = 1;
            if (alpha < 1.0 / 255.0) continue;
            double tT = T * (1.0 - alpha);
            if (fabs(tT - 1e-4) < 2e-7) fl = 1;
            if (tT < 1e-4) break;
            for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
            T = tT;
            ++nc;
          }
          for (int ch = 0; ch < 3; ++ch) img[((int64_t)ch * H + py) * W + px] = C[ch] + T * bg[ch];
          flag[(int64_t)py * W + px] = (uint8_t)fl;
          if (n_contrib) n_contrib[(int64_t)py * W + px] = nc;
        }
    }
}
