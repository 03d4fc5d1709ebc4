// Projection of the drawn Gaussians (the per-Gaussian 3DGS math of Kerbl et
// al., which the paper's renderer runs per Gaussian before rasterisation,
// Sec. 4.2 "Rendering"): gathers each Gaussian of the draw list from its pool
// slot, culls, builds the 3D covariance, the EWA 2D covariance, conic,
// radius, tile rectangle, the rectangle's tiles met by the 3-sigma ellipse,
// view-dependent SH colour and view depth.
//
// This file is compiled with -fmad=false: every discrete result (cull,
// radius, rectangle, depth key) is a chain of single, correctly rounded
// float32 operations in the order written, so it is reproducible bit for bit
// by any IEEE implementation of the same formula.  Constants follow the 3DGS
// reference renderer: near plane 0.2, guard band 1.3, dilation 0.3, 3 sigma,
// eigenvalue floor 0.1, colour offset 0.5 clamped at 0.
//
// Data layout: a pool slot holds fanout^l sub-slots at level l; sub-slot s
// of a slot is a contiguous block of m_l Gaussians in structure-of-arrays
// form (attribute a of Gaussian g at a * m_l + g), so consecutive threads
// read consecutive words of every attribute.  fp16 pools keep position and
// opacity in float and scale, rotation and SH in half; VQ pools (compressed
// pages) keep SH band 0 in half and the index of a codeword of the SH
// codebook (in device memory) for bands 1..3.
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "coverage.cuh"
#include "renderer.cuh"
#include "tma.cuh"

namespace vm {
namespace {

// FMT: kFmt32 (all attributes float rows), kFmt16 (position and opacity
// float rows, the rest half rows) or kFmtVQ (as kFmt16 for SH band 0, the
// codebook index of bands 1..3 in 16-bit row 10).
template <int K, int FMT>
struct Rec {
  // attribute loaders for one Gaussian of a block of m
  __device__ static float pos(const uint8_t *b, int m, int g, int a) {
    return reinterpret_cast<const float *>(b)[(int64_t)a * m + g];
  }
  __device__ static float opac(const uint8_t *b, int m, int g) {
    return reinterpret_cast<const float *>(b)[(int64_t)(FMT != kFmt32 ? 3 : 10) * m + g];
  }
  __device__ static const uint16_t *row16(const uint8_t *b, int m, int h) {
    return reinterpret_cast<const uint16_t *>(b + (int64_t)16 * m) + (int64_t)h * m;
  }
  __device__ static float half_at(const uint8_t *b, int m, int g, int h) {
    return __half2float(__ushort_as_half(row16(b, m, h)[g]));
  }
  __device__ static float scale(const uint8_t *b, int m, int g, int a) {
    if (FMT != kFmt32) return half_at(b, m, g, a);
    return reinterpret_cast<const float *>(b)[(int64_t)(3 + a) * m + g];
  }
  __device__ static float rot(const uint8_t *b, int m, int g, int a) {
    if (FMT != kFmt32) return half_at(b, m, g, 3 + a);
    return reinterpret_cast<const float *>(b)[(int64_t)(6 + a) * m + g];
  }
  // (VQ: band 0 only; bands 1..3 come from the codeword)
  __device__ static float sh(const uint8_t *b, int m, int g, int k, int c) {
    if (FMT != kFmt32) return half_at(b, m, g, 7 + 3 * k + c);
    return reinterpret_cast<const float *>(b)[(int64_t)(11 + 3 * k + c) * m + g];
  }
  __device__ static uint32_t code(const uint8_t *b, int m, int g) { return row16(b, m, 10)[g]; }
  static constexpr int kRec = FMT == kFmtVQ ? rec_bytes_vq() : FMT == kFmt16 ? rec_bytes16(K) : rec_bytes32(K);
};

// real SH basis (l <= 3, m = -l..l), Condon-Shortley phase; the constants are
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) with the sqrt(2) of the real basis
#define SHC0 0.28209479177387814f
#define SHC1 0.4886025119029199f
#define SHC2A 1.0925484305920792f
#define SHC2B 0.31539156525252005f
#define SHC2C 0.5462742152960396f
#define SHC3A 0.5900435899266435f
#define SHC3B 2.890611442640554f
#define SHC3C 0.4570457994644658f
#define SHC3D 0.3731763325901154f
#define SHC3E 1.445305721320277f

// Attributes of Gaussian g of a level block of m Gaussians in the pool; for
// VQ pools cw is its codeword (bands 1..3 of the SH).
template <int K, int FMT>
struct GlobalSrc {
  using R = Rec<K, FMT>;
  const uint8_t *blk;
  int m, g;
  const float *cw;
  __device__ GlobalSrc(const uint8_t *b, int m_, int g_, const float *codebook) : blk(b), m(m_), g(g_), cw(nullptr) {
    if (FMT == kFmtVQ) cw = codebook + (int64_t)R::code(b, m_, g_) * kCodeRow;
  }
  __device__ float pos(int a) const { return R::pos(blk, m, g, a); }
  __device__ float opac() const { return R::opac(blk, m, g); }
  __device__ float scale(int a) const { return R::scale(blk, m, g, a); }
  __device__ float rot(int a) const { return R::rot(blk, m, g, a); }
  __device__ float sh(int k, int c) const {
    if (FMT == kFmtVQ && k > 0) return __ldg(cw + 16 * c + (k - 1));
    return R::sh(blk, m, g, k, c);
  }
  // VQ: channel c's coefficients of bands 1..3, four at a time
  __device__ float4 cw4(int c, int v) const { return __ldg(reinterpret_cast<const float4 *>(cw + 16 * c) + v); }
};

// The same attributes staged in shared memory: the record's float rows (A)
// and 16-bit rows (B) of a chunk of CH Gaussians, row after row.
template <int K, int FMT, int CH>
struct SharedSrc {
  const float *A;
  const __half *B;
  int g;
  const float *cw;
  __device__ SharedSrc(const float *a, const __half *b, int g_, const float *codebook) : A(a), B(b), g(g_), cw(nullptr) {
    if (FMT == kFmtVQ)
      cw = codebook + (int64_t)__half_as_ushort(B[10 * CH + g_]) * kCodeRow;
  }
  __device__ float half_at(int h) const { return __half2float(B[h * CH + g]); }
  __device__ float pos(int a) const { return A[a * CH + g]; }
  __device__ float opac() const { return A[(FMT != kFmt32 ? 3 : 10) * CH + g]; }
  __device__ float scale(int a) const { return FMT != kFmt32 ? half_at(a) : A[(3 + a) * CH + g]; }
  __device__ float rot(int a) const { return FMT != kFmt32 ? half_at(3 + a) : A[(6 + a) * CH + g]; }
  __device__ float sh(int k, int c) const {
    if (FMT == kFmtVQ && k > 0) return __ldg(cw + 16 * c + (k - 1));
    return FMT != kFmt32 ? half_at(7 + 3 * k + c) : A[(11 + 3 * k + c) * CH + g];
  }
  __device__ float4 cw4(int c, int v) const { return __ldg(reinterpret_cast<const float4 *>(cw + 16 * c) + v); }
};

// Projects one Gaussian for one camera and writes splat record out.
// wt: the draw item's opacity weight (1, or a cross-fade weight in (0, 1))
template <int K, int FMT, class Src>
__device__ __forceinline__ void project_one(const Splats &sp, const vm3dgs_camera &cam, const Src &src, int64_t out,
                                            float wt) {
  const float *V = cam.view;
  const int gx = (cam.width + cam.tile_w - 1) / cam.tile_w;
  const int gy = (cam.height + cam.tile_h - 1) / cam.tile_h;
  const float TW = (float)cam.tile_w, TH = (float)cam.tile_h;
  float x = src.pos(0), y = src.pos(1), z = src.pos(2);
  float o = src.opac() * wt;
  // a culled splat: no tiles, zero rectangle, depth and radius
  auto culled = [&]() {
    sp.touched[out] = 0;
    sp.tmask[out] = 0;
    sp.rect[2 * out] = 0;
    sp.rect[2 * out + 1] = 0;
    sp.depth[out] = 0;
    sp.radius[out] = 0.0f;
  };
  float tx = ((V[0] * x + V[1] * y) + V[2] * z) + V[3];
  float ty = ((V[4] * x + V[5] * y) + V[6] * z) + V[7];
  float tz = ((V[8] * x + V[9] * y) + V[10] * z) + V[11];
  if (!(o > 0.0f) || !(tz > 0.2f)) {
    culled();
    return;
  }
  float qw = src.rot(0), qx = src.rot(1), qy = src.rot(2), qz = src.rot(3);
  float sc[3] = {src.scale(0), src.scale(1), src.scale(2)};
  float xx = qx * qx, yy = qy * qy, zz = qz * qz;
  float xy = qx * qy, xz = qx * qz, yz = qy * qz;
  float wx = qw * qx, wy = qw * qy, wz = qw * qz;
  float Rm[3][3];
  Rm[0][0] = 1.0f - 2.0f * (yy + zz); Rm[0][1] = 2.0f * (xy - wz); Rm[0][2] = 2.0f * (xz + wy);
  Rm[1][0] = 2.0f * (xy + wz); Rm[1][1] = 1.0f - 2.0f * (xx + zz); Rm[1][2] = 2.0f * (yz - wx);
  Rm[2][0] = 2.0f * (xz - wy); Rm[2][1] = 2.0f * (yz + wx); Rm[2][2] = 1.0f - 2.0f * (xx + yy);
  float M[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[r][c] = Rm[r][c] * sc[c];
  float S[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) S[r][c] = (M[r][0] * M[c][0] + M[r][1] * M[c][1]) + M[r][2] * M[c][2];
  float limx = 1.3f * ((0.5f * (float)cam.width) / cam.fx);
  float limy = 1.3f * ((0.5f * (float)cam.height) / cam.fy);
  float txtz = tx / tz, tytz = ty / tz;
  float clx = fminf(limx, fmaxf(-limx, txtz)) * tz;
  float cly = fminf(limy, fmaxf(-limy, tytz)) * tz;
  float tz2 = tz * tz;
  float J00 = cam.fx / tz, J02 = -(cam.fx * clx) / tz2;
  float J11 = cam.fy / tz, J12 = -(cam.fy * cly) / tz2;
  float T0[3], T1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T0[c] = J00 * V[c] + J02 * V[8 + c];
    T1[c] = J11 * V[4 + c] + J12 * V[8 + c];
  }
  float u[3], w[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    u[r] = (S[r][0] * T0[0] + S[r][1] * T0[1]) + S[r][2] * T0[2];
    w[r] = (S[r][0] * T1[0] + S[r][1] * T1[1]) + S[r][2] * T1[2];
  }
  float ca = (T0[0] * u[0] + T0[1] * u[1]) + T0[2] * u[2];
  float cb = (T1[0] * u[0] + T1[1] * u[1]) + T1[2] * u[2];
  float cc = (T1[0] * w[0] + T1[1] * w[1]) + T1[2] * w[2];
  ca = ca + 0.3f;
  cc = cc + 0.3f;
  float det = fmaxf(ca * cc - cb * cb, 1e-12f);
  float mid = 0.5f * (ca + cc);
  float disc = fmaxf(0.1f, mid * mid - det);
  float lam = mid + sqrtf(disc);
  float r = ceilf(3.0f * sqrtf(lam));
  float pu = cam.fx * txtz + cam.cx;
  float pv = cam.fy * tytz + cam.cy;
  float fx0 = floorf((pu - r) / TW), fx1 = floorf((pu + r) / TW) + 1.0f;
  float fy0 = floorf((pv - r) / TH), fy1 = floorf((pv + r) / TH) + 1.0f;
  fx0 = fminf(fmaxf(fx0, 0.0f), (float)gx); fx1 = fminf(fmaxf(fx1, 0.0f), (float)gx);
  fy0 = fminf(fmaxf(fy0, 0.0f), (float)gy); fy1 = fminf(fmaxf(fy1, 0.0f), (float)gy);
  const int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
  if (x0 >= x1 || y0 >= y1) {
    culled();
    return;
  }
  float ia = cc / det, ib = -cb / det, ic = ca / det;
  // tiles of the rectangle met by the 3-sigma ellipse, counted row by row;
  // a rectangle of at most 64 tiles also keeps them as a row-major mask
  const SplatEllipse el = splat_ellipse(pu, pv, ia, ib, ic);
  const TileGeom tg{cam.width, cam.height, cam.tile_w, cam.tile_h};
  const int rw = x1 - x0;
  const bool small_rect = rw * (y1 - y0) <= 64;
  uint64_t tmask = 0;
  int covered = 0;
  for (int ty = y0; ty < y1; ++ty) {
    const int2 sp2 = row_span(el, ty, x0, x1, tg);
    const int n = sp2.y - sp2.x;
    if (n <= 0) continue;
    covered += n;
    if (small_rect) tmask |= (n >= 64 ? ~0ull : ((1ull << n) - 1ull)) << ((ty - y0) * rw + (sp2.x - x0));
  }
  // continuous outputs
  float dx = x - cam.campos[0], dy = y - cam.campos[1], dz = z - cam.campos[2];
  float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
  dx *= inv; dy *= inv; dz *= inv;
  float Y[16];
  Y[0] = SHC0;
  if (K > 1) {
    Y[1] = -SHC1 * dy; Y[2] = SHC1 * dz; Y[3] = -SHC1 * dx;
  }
  if (K > 4) {
    float x2 = dx * dx, y2 = dy * dy, z2 = dz * dz;
    Y[4] = SHC2A * dx * dy; Y[5] = -SHC2A * dy * dz; Y[6] = SHC2B * (2.0f * z2 - x2 - y2);
    Y[7] = -SHC2A * dx * dz; Y[8] = SHC2C * (x2 - y2);
    if (K > 9) {
      Y[9] = -SHC3A * dy * (3.0f * x2 - y2); Y[10] = SHC3B * dx * dy * dz;
      Y[11] = -SHC3C * dy * (4.0f * z2 - x2 - y2); Y[12] = SHC3D * dz * (2.0f * z2 - 3.0f * x2 - 3.0f * y2);
      Y[13] = -SHC3C * dx * (4.0f * z2 - x2 - y2); Y[14] = SHC3E * dz * (x2 - y2);
      Y[15] = -SHC3A * dx * (x2 - 3.0f * y2);
    }
  }
  // (colour is a continuous output: fused multiply-adds are fine here)
  float rgb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float s = 0.0f;
    if constexpr (FMT == kFmtVQ) {
      // bands 1..3 from the codeword by 16-byte loads, summed in k order
      s = __fmaf_rn(src.sh(0, c), Y[0], s);
#pragma unroll
      for (int v = 0; v < (K + 2) / 4; ++v) {
        const float4 t = src.cw4(c, v);
        const float q[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (1 + 4 * v + i < K) s = __fmaf_rn(q[i], Y[1 + 4 * v + i], s);
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) s = __fmaf_rn(src.sh(k, c), Y[k], s);
    }
    s += 0.5f;
    rgb[c] = s > 0.0f ? s : 0.0f;
  }
  sp.rec[3 * out] = make_float4(pu, pv, ia, ib);
  sp.rec[3 * out + 1] = make_float4(ic, o, rgb[0], rgb[1]);
  sp.rec[3 * out + 2] = make_float4(rgb[2], 0.0f, 0.0f, 0.0f);
  sp.depth[out] = __float_as_uint(tz);
  sp.radius[out] = r;
  sp.rect[2 * out] = (uint32_t)x0 | ((uint32_t)x1 << 16);
  sp.rect[2 * out + 1] = (uint32_t)y0 | ((uint32_t)y1 << 16);
  sp.touched[out] = (uint32_t)covered;
  sp.tmask[out] = tmask;
}

template <int K, int FMT>
__global__ void __launch_bounds__(256) project_kernel(ProjectArgs a, vm3dgs_camera cam) {
  using R = Rec<K, FMT>;
  const int64_t N = a.ctl->draw_gauss < a.ncap ? a.ctl->draw_gauss : a.ncap;
  if (blockIdx.x == 0 && threadIdx.x == 0) a.rctl->r_drawn = a.ctl->draw_gauss;
  const int nd = a.ctl->n_draw;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < N; base += stride) {
    // lane 0 finds the draw item holding the warp's first Gaussian
    int j = 0;
    if (lane == 0) {
      int lo = 0, hi = nd - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.draw_off[mid] <= base) lo = mid; else hi = mid - 1;
      }
      j = lo;
    }
    j = __shfl_sync(0xffffffffu, j, 0);
    const int64_t i = base + lane;
    if (i >= N) continue;
    while (j + 1 < nd && a.draw_off[j + 1] <= i) ++j;
    const int4 it = a.draw[j];
    int m = a.page_size;
    for (int l = 0; l < it.y; ++l) m /= a.fanout;
    const int g = (int)(i - a.draw_off[j]);
    const uint8_t *blk = a.pool + (int64_t)it.z * a.slot_bytes + (int64_t)it.w * m * R::kRec;
    project_one<K, FMT>(a.sp, cam, GlobalSrc<K, FMT>(blk, m, g, a.codebook), i, a.draw_w ? a.draw_w[j] : 1.0f);
  }
}

// All views at once: blockIdx.y is the view; splat record v * N + i.
template <int K, int FMT>
__global__ void __launch_bounds__(256) project_batched_kernel(ProjectArgs a, const ViewTable *views) {
  using R = Rec<K, FMT>;
  const int v = blockIdx.y;
  if (v >= views->n) return;
  const vm3dgs_camera cam = views->cam[v];
  const int64_t N = a.ctl->draw_gauss < a.ncap ? a.ctl->draw_gauss : a.ncap;
  if (blockIdx.x == 0 && v == 0 && threadIdx.x == 0) a.rctl->r_drawn = a.ctl->draw_gauss;
  const int nd = a.ctl->n_draw;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < N; base += stride) {
    int j = 0;
    if (lane == 0) {
      int lo = 0, hi = nd - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.draw_off[mid] <= base) lo = mid; else hi = mid - 1;
      }
      j = lo;
    }
    j = __shfl_sync(0xffffffffu, j, 0);
    const int64_t i = base + lane;
    if (i >= N) continue;
    while (j + 1 < nd && a.draw_off[j + 1] <= i) ++j;
    const int4 it = a.draw[j];
    int m = a.page_size;
    for (int l = 0; l < it.y; ++l) m /= a.fanout;
    const int g = (int)(i - a.draw_off[j]);
    const uint8_t *blk = a.pool + (int64_t)it.z * a.slot_bytes + (int64_t)it.w * m * R::kRec;
    project_one<K, FMT>(a.sp, cam, GlobalSrc<K, FMT>(blk, m, g, a.codebook), (int64_t)v * N + i,
                        a.draw_w ? a.draw_w[j] : 1.0f);
  }
}

// Projection with the records staged by tile loads of the tensor memory
// accelerator: a CTA of 128 threads takes items of two 64-Gaussian chunks
// (every level block is a multiple of 64); warp 0 finds their draw entries
// and issues the tile loads (float rows, and 16-bit rows for fp16 and VQ pools) of the
// next item while the CTA projects the current one from shared memory (two
// stages).  The stages are handed over by mbarriers alone, with no CTA-wide
// barrier per item: a stage's `full` barrier completes when its loads have
// landed, its `empty` barrier when all four warps have projected from it, and
// warp 0 refills a stage only after its `empty` phase, so a warp that is done
// with an item goes on to the next one without waiting for the others.  A
// wait that expires records VM3DGS_E_TIMEOUT and ends the warp's loop; warp
// 0's copies still in flight land before the CTA ends.
constexpr int kMbarPolls = 1 << 20;

// CH Gaussians per chunk (64 or 32), 128 / CH chunks per CTA of 128 threads
template <int K, int FMT, int CH>
struct TmaShape {
  static constexpr int NA = FMT != kFmt32 ? 4 : n_attr32(K);                              // float rows
  static constexpr int NH = FMT == kFmtVQ ? kHalfVQ : FMT == kFmt16 ? n_half16(K) : 0;   // 16-bit rows
  static constexpr int ABYTES = NA * CH * 4, BBYTES = NH * CH * 2;
  static constexpr int CHUNK = ABYTES + BBYTES;
  static constexpr int PER = 128 / CH;                            // chunks per CTA item
  static constexpr int STAGE = PER * CHUNK;
  static constexpr int SMEM = 2 * STAGE + 64;                     // + barriers (full[2], empty[2])
};

template <int K, int FMT, int CH>
__global__ void __launch_bounds__(128) project_tma_kernel(ProjectArgs a, vm3dgs_camera cam,
                                                          const __grid_constant__ ProjMaps maps) {
  using S = TmaShape<K, FMT, CH>;
  constexpr int kChunk = CH, kChunksPerCta = S::PER;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * S::STAGE);  // full[0..1]
  uint64_t *empty = bar + 2;                                             // empty[0..1]
  constexpr int kWarps = 128 / 32;
  __shared__ float s_w[2][kChunksPerCta];  // opacity weight of each chunk's draw item, per stage
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t N = a.ctl->draw_gauss < a.ncap ? a.ctl->draw_gauss : a.ncap;
  if (blockIdx.x == 0 && tid == 0) a.rctl->r_drawn = a.ctl->draw_gauss;
  const int64_t nchunks = N / kChunk;
  const int64_t nitems = (nchunks + kChunksPerCta - 1) / kChunksPerCta;
  const int nd = a.ctl->n_draw;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&empty[0], kWarps);
    mbar_init(&empty[1], kWarps);
    mbar_init_fence();
  }
  __syncthreads();
  // warp 0: loads of item `it` into stage `stg`
  auto issue = [&](int64_t it, int stg) {
    int64_t e[kChunksPerCta];
    int valid = 0;
#pragma unroll
    for (int j = 0; j < kChunksPerCta; ++j) {
      const int64_t c = it * kChunksPerCta + j;
      e[j] = -1;
      if (c < nchunks) {
        // last draw entry whose first Gaussian is <= c * kChunk (warp-wide search)
        const int64_t gi = c * kChunk;
        int64_t lo = 0, hi = nd;
        while (hi - lo > 32) {
          const int64_t step = (hi - lo + 31) / 32;
          const int64_t p = lo + lane * step;
          const uint32_t m = __ballot_sync(0xffffffffu, p < hi && a.draw_off[p] <= gi);
          lo += (31 - __clz(m)) * step;
          hi = min(hi, lo + step);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, lo + lane < hi && a.draw_off[lo + lane] <= gi);
        e[j] = lo + (31 - __clz(m));
        ++valid;
      }
    }
    if (lane == 0) {
      uint8_t *buf = smem + stg * S::STAGE;
      proxy_fence_shared();
      mbar_arrive_expect(&bar[stg], (uint32_t)(valid * S::CHUNK));
#pragma unroll
      for (int j = 0; j < kChunksPerCta; ++j) {
        if (e[j] < 0) continue;
        const int4 d = a.draw[e[j]];
        s_w[stg][j] = a.draw_w ? a.draw_w[e[j]] : 1.0f;
        int sub = 1;
        for (int l = 0; l < d.y; ++l) sub *= a.fanout;
        const int u = d.z * sub + d.w;  // level block of the whole pool
        const int g0 = (int)((it * kChunksPerCta + j) * kChunk - a.draw_off[e[j]]);
        tma_load_3d(buf + j * S::CHUNK, &maps.a[d.y], g0, 0, u, &bar[stg]);
        if (FMT != kFmt32) tma_load_3d(buf + j * S::CHUNK + S::ABYTES, &maps.b[d.y], g0, 0, u, &bar[stg]);
      }
    }
    __syncwarp();
  };
  int64_t item = blockIdx.x;
  int pending = 0;  // (warp 0) bit s: stage s holds loads it issued and has not yet waited for
  if (item < nitems && warp == 0) {
    issue(item, 0);
    pending = 1;
  }
  uint32_t parity = 0u;   // bit s: phase parity of full[s] this warp waits for next
  uint32_t eparity = 0u;  // (warp 0) bit s: phase parity of empty[s] it waits for next
  bool timed_out = false;
  for (int k = 0; item < nitems; ++k, item += gridDim.x) {
    const int stg = k & 1;
    const int64_t next = item + gridDim.x;
    if (warp == 0 && next < nitems) {
      // stage stg ^ 1 last held item k - 1: all warps must have released it
      if (k >= 1) {
        const bool ok = mbar_wait(&empty[stg ^ 1], (eparity >> (stg ^ 1)) & 1u, kMbarPolls);
        if (__any_sync(0xffffffffu, !ok)) {
          timed_out = true;
          break;
        }
        eparity ^= 1u << (stg ^ 1);
      }
      issue(next, stg ^ 1);
      pending |= 1 << (stg ^ 1);
    }
    const bool ok = mbar_wait(&bar[stg], (parity >> stg) & 1u, kMbarPolls);
    if (__any_sync(0xffffffffu, !ok)) {
      timed_out = true;
      break;
    }
    parity ^= 1u << stg;
    pending &= ~(1 << stg);
    const int ch = tid / kChunk, g = tid % kChunk;
    const int64_t c = item * kChunksPerCta + ch;
    if (c < nchunks) {
      const uint8_t *buf = smem + stg * S::STAGE + ch * S::CHUNK;
      const SharedSrc<K, FMT, CH> src(reinterpret_cast<const float *>(buf),
                                      reinterpret_cast<const __half *>(buf + S::ABYTES), g, a.codebook);
      project_one<K, FMT>(a.sp, cam, src, c * kChunk + g, s_w[stg][ch]);
    }
    // this warp is done with the stage (and with its chunk weights)
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[stg]);
  }
  if (timed_out && lane == 0) atomicCAS(const_cast<int32_t *>(&a.ctl->status), 0, VM3DGS_E_TIMEOUT);
  // the CTA's memory stays until warp 0's copies still in flight have landed
  // (none unless a wait expired)
  if (warp == 0 && lane == 0)
    for (int s2 = 0; s2 < 2; ++s2)
      if (pending & (1 << s2)) mbar_wait(&bar[s2], (parity >> s2) & 1u, kMbarPolls);
}

template <int K>
void launch_kb(const ProjectArgs &a, const ViewTable *views, int n_views, cudaStream_t st) {
  int64_t blocks = (a.ncap + 255) / 256;
  int64_t cap = (148 * 16 + n_views - 1) / n_views;
  if (cap < 8) cap = 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  dim3 grid((unsigned)blocks, (unsigned)n_views);
  if (a.fmt == kFmtVQ)
    project_batched_kernel<K, kFmtVQ><<<grid, 256, 0, st>>>(a, views);
  else if (a.fmt == kFmt16)
    project_batched_kernel<K, kFmt16><<<grid, 256, 0, st>>>(a, views);
  else
    project_batched_kernel<K, kFmt32><<<grid, 256, 0, st>>>(a, views);
}

template <int K, int FMT, int CH>
void launch_tma(const ProjectArgs &a, const vm3dgs_camera &cam, cudaStream_t st) {
  using S = TmaShape<K, FMT, CH>;
  max_dynamic_smem((const void *)project_tma_kernel<K, FMT, CH>, S::SMEM);
  prefer_shared((const void *)project_tma_kernel<K, FMT, CH>);
  project_tma_kernel<K, FMT, CH>
      <<<full_wave((const void *)project_tma_kernel<K, FMT, CH>, 128, S::SMEM), 128, S::SMEM, st>>>(a, cam, *a.maps);
}

template <int K>
void launch_k(const ProjectArgs &a, const vm3dgs_camera &cam, cudaStream_t st) {
  if (a.maps) {
    if (a.maps->chunk == 64)
      a.fmt == kFmtVQ ? launch_tma<K, kFmtVQ, 64>(a, cam, st)
      : a.fmt == kFmt16 ? launch_tma<K, kFmt16, 64>(a, cam, st) : launch_tma<K, kFmt32, 64>(a, cam, st);
    else
      a.fmt == kFmtVQ ? launch_tma<K, kFmtVQ, 32>(a, cam, st)
      : a.fmt == kFmt16 ? launch_tma<K, kFmt16, 32>(a, cam, st) : launch_tma<K, kFmt32, 32>(a, cam, st);
    return;
  }
  int64_t blocks = (a.ncap + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  if (a.fmt == kFmtVQ)
    project_kernel<K, kFmtVQ><<<(unsigned)blocks, 256, 0, st>>>(a, cam);
  else if (a.fmt == kFmt16)
    project_kernel<K, kFmt16><<<(unsigned)blocks, 256, 0, st>>>(a, cam);
  else
    project_kernel<K, kFmt32><<<(unsigned)blocks, 256, 0, st>>>(a, cam);
}

}  // namespace

void launch_project_batched(const ProjectArgs &a, const ViewTable *views, int n_views, cudaStream_t st) {
  switch (a.K) {
    case 1: launch_kb<1>(a, views, n_views, st); break;
    case 4: launch_kb<4>(a, views, n_views, st); break;
    case 9: launch_kb<9>(a, views, n_views, st); break;
    default: launch_kb<16>(a, views, n_views, st); break;
  }
}

void launch_project(const ProjectArgs &a, const vm3dgs_camera &cam, cudaStream_t st) {
  switch (a.K) {
    case 1: launch_k<1>(a, cam, st); break;
    case 4: launch_k<4>(a, cam, st); break;
    case 9: launch_k<9>(a, cam, st); break;
    default: launch_k<16>(a, cam, st); break;
  }
}

bool encode_proj_maps(const vm3dgs_scene *s, const uint8_t *pool, int64_t P, int fmt, ProjMaps *out) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if (s->levels > kMaxLevels) return false;
  // the widest chunk that divides every level block
  int chunk = 64;
  {
    int64_t sub = 1;
    for (int l = 0; l < s->levels; ++l, sub *= s->fanout)
      if ((s->page_size / sub) % 64 != 0) chunk = 32;
  }
  const int kChunk = chunk;
  out->chunk = chunk;
  const int K = s->K;
  const cuuint32_t NA = fmt != kFmt32 ? 4u : (cuuint32_t)n_attr32(K);
  const cuuint32_t NH = fmt == kFmtVQ ? (cuuint32_t)kHalfVQ : fmt == kFmt16 ? (cuuint32_t)n_half16(K) : 0u;
  const int64_t rec = s->fmt_rec(fmt);
  int64_t sub = 1;
  for (int l = 0; l < s->levels; ++l) {
    const int64_t m = s->page_size / sub;
    if (m % kChunk != 0 || m * sub != s->page_size) return false;
    const cuuint64_t nsub = (cuuint64_t)(P * sub);
    const cuuint32_t box[3] = {(cuuint32_t)kChunk, NA, 1}, estr[3] = {1, 1, 1};
    const cuuint64_t dimA[3] = {(cuuint64_t)m, NA, nsub};
    const cuuint64_t strA[2] = {(cuuint64_t)(m * 4), (cuuint64_t)(m * rec)};
    if (enc(&out->a[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<uint8_t *>(pool), dimA, strA, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    if (fmt != kFmt32) {
      const cuuint32_t boxB[3] = {(cuuint32_t)kChunk, NH, 1};
      const cuuint64_t dimB[3] = {(cuuint64_t)m, NH, nsub};
      const cuuint64_t strB[2] = {(cuuint64_t)(m * 2), (cuuint64_t)(m * rec)};
      if (enc(&out->b[l], CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint8_t *>(pool + 16 * m), dimB, strB, boxB,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    }
    sub *= s->fanout;
  }
  return true;
}

}  // namespace vm
