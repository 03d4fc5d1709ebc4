// Tiles of a splat.  A splat is binned to the tiles of its rectangle whose
// box of pixel centres meets its 3-sigma ellipse
//   E = {d : A dx^2 + 2 B dx dy + C dy^2 <= 9}   (d = pixel - centre,
//                                                 (A, B, C) the FP32 conic)
// for rectangles of every size.  The test runs one tile row at a time: E cut
// by the row's band of pixel-centre y values is an x-interval [X0, X1]
// (E is convex), bounded by E's boundary at the heights nearest to its
// rightmost and leftmost points, and the row keeps the contiguous run of
// columns whose pixel-centre intervals meet [X0, X1]:
//   D = A C - B^2 (not positive: every tile of the rectangle),
//   ey = sqrt(9 A / D), dys = -3 B / sqrt(C D)
//   [l, h] = [yl - pv, yh - pv] clipped to [-ey, ey] (empty: no tile)
//   X1 = (-B t1 + sqrt(max(0, 9 A - D t1^2))) / A,  t1 = clamp(dys, l, h)
//   X0 = (-B t0 - sqrt(max(0, 9 A - D t0^2))) / A,  t0 = clamp(-dys, l, h)
//   column kept  <=>  xl - pu <= X1  and  xh - pu >= X0.
// (Binning is left by the paper to the 3DGS renderer, Sec. 4.2 Rendering;
// this rule is a reading.)  Each step is one correctly rounded FP32
// operation in a fixed order, written with _rn intrinsics so that no
// compiler flag can contract or reorder it: the projection that counts a
// splat's tiles and the emission that lists them see the same set.
#pragma once

#include <cuda_runtime.h>

namespace vm {

// image and tile size of a view, in pixels
struct TileGeom {
  int W, H, TW, TH;
};

// the per-splat constants of the row rule
struct SplatEllipse {
  float pu, pv, A, B, D, ey, dys;
  bool all;  // determinant not positive: every tile of the rectangle
};

__device__ __forceinline__ SplatEllipse splat_ellipse(float pu, float pv, float A, float B, float C) {
  SplatEllipse e;
  e.pu = pu;
  e.pv = pv;
  e.A = A;
  e.B = B;
  e.D = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
  e.all = !(e.D > 0.0f);
  e.ey = __fsqrt_rn(__fdiv_rn(__fmul_rn(9.0f, A), e.D));
  e.dys = __fdiv_rn(-__fmul_rn(3.0f, B), __fsqrt_rn(__fmul_rn(C, e.D)));
  return e;
}

// Kept columns [x, y) of tile row ty, within the rectangle's [x0, x1);
// y <= x means none.
__device__ __forceinline__ int2 row_span(const SplatEllipse &e, int ty, int x0, int x1, const TileGeom &g) {
  if (e.all) return make_int2(x0, x1);
  const float yl = __fadd_rn((float)(ty * g.TH), 0.5f);
  const float yh = __fsub_rn((float)min((ty + 1) * g.TH, g.H), 0.5f);
  const float l = fmaxf(__fsub_rn(yl, e.pv), -e.ey), h = fminf(__fsub_rn(yh, e.pv), e.ey);
  if (l > h) return make_int2(x0, x0);
  const float t1 = fminf(fmaxf(e.dys, l), h), t0 = fminf(fmaxf(-e.dys, l), h);
  const float a9 = __fmul_rn(9.0f, e.A);
  const float s1 = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(a9, __fmul_rn(e.D, __fmul_rn(t1, t1)))));
  const float s0 = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(a9, __fmul_rn(e.D, __fmul_rn(t0, t0)))));
  const float X1 = __fdiv_rn(__fadd_rn(-__fmul_rn(e.B, t1), s1), e.A);
  const float X0 = __fdiv_rn(__fsub_rn(-__fmul_rn(e.B, t0), s0), e.A);
  // first column whose right pixel centre reaches X0, and first whose left
  // one lies beyond X1: both predicates are monotone in the column, so a
  // guess corrected by single steps finds them exactly
  auto right_ok = [&](int tx) {
    return __fsub_rn(__fsub_rn((float)min((tx + 1) * g.TW, g.W), 0.5f), e.pu) >= X0;
  };
  auto left_past = [&](int tx) { return __fsub_rn(__fadd_rn((float)(tx * g.TW), 0.5f), e.pu) > X1; };
  const float inv_tw = 1.0f / (float)g.TW;
  int c0 = min(max(__float2int_rd((e.pu + X0) * inv_tw), x0), x1);
  while (c0 > x0 && right_ok(c0 - 1)) --c0;
  while (c0 < x1 && !right_ok(c0)) ++c0;
  int c1 = min(max(__float2int_rd((e.pu + X1) * inv_tw) + 1, c0), x1);
  while (c1 > c0 && left_past(c1 - 1)) --c1;
  while (c1 < x1 && !left_past(c1)) ++c1;
  return make_int2(c0, c1);
}

}  // namespace vm
