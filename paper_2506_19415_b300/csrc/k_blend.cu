// Front-to-back alpha blending per image tile (Sec. 4.2: the paper blends
// quads in hardware; the per-pixel Gaussian and the compositing rule are
// those of Kerbl et al.).  One CTA per tile.  The tile's splats are staged
// in shared memory in batches; a pixel stops when its transmittance would
// fall below 1e-4, the CTA stops when every pixel has.  alpha = min(0.99, o exp(power)); splats
// with alpha < 1/255 are skipped; the image is C + T * background, CHW.
#include <cudaTypedefs.h>

#include <cstring>

#include "renderer.cuh"
#include "tma.cuh"

namespace vm {
namespace {

// Per staged splat the conic and opacity are rewritten once for the log2
// domain: q = log2(e) * power = dx (a dx + b dy) + c dy^2 with a = -A/2 log2 e,
// b = -B log2 e, c = -C/2 log2 e, and l = log2(opacity), so that
// alpha = min(0.99, 2^(q + l)) and the skip test alpha < 1/255 becomes
// q + l < log2(1/255), taken before the exponential.
#define LOG2E 1.4426950408889634f
#define LOG2_SKIP (-7.99435343685886f)  /* log2(1/255) */

__device__ __forceinline__ void stage(const Splats &sp, uint32_t g, float4 &a, float4 &b, float &c) {
  const float4 s0 = sp.rec[3 * g], s1 = sp.rec[3 * g + 1];
  a = make_float4(s0.x, s0.y, -0.5f * LOG2E * s0.z, -LOG2E * s0.w);
  b = make_float4(-0.5f * LOG2E * s1.x, __log2f(s1.y), s1.z, s1.w);
  c = sp.rec[3 * g + 2].x;
}

// Box (x0, x1, y0, y1) outside which a splat has alpha < 1/255 with a margin
// wider than the rounding of the per-pixel test, so that skipping the pixels
// outside changes nothing.  With conic M = [[A, B], [B, C]] the test is
// d^T M d <= tau = 2 ln(255 o); the box of that ellipse is
// |dx| <= sqrt(tau C / det M), |dy| <= sqrt(tau A / det M), taken here for
// 1.01 tau + 0.05 and widened by 1% + 0.1 px.  Splats whose conic is too
// ill-conditioned for that margin (eigenvalue ratio above 1e4) get an
// unbounded box; those with o < 0.999 / 255 an empty one.  s0, s1: the
// first two float4 of the splat's record.
__device__ __forceinline__ float4 alpha_box(const float4 &s0, const float4 &s1) {
  const float A = s0.z, B = s0.w, C = s1.x, o = s1.y;
  if (!(o * 255.0f >= 0.999f)) return make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
  const float det = A * C - B * B, m = 0.5f * (A + C);
  const float lmax = m + sqrtf(fmaxf(m * m - det, 0.0f));
  const float unbounded = INFINITY;
  if (!(det > 0.0f) || !(lmax > 0.0f) || !(lmax * lmax <= 1e4f * det))
    return make_float4(-unbounded, unbounded, -unbounded, unbounded);
  const float tau = 2.0f * logf(255.0f * o) * 1.01f + 0.05f;
  const float xr = sqrtf(tau * C / det) * 1.01f + 0.1f, yr = sqrtf(tau * A / det) * 1.01f + 0.1f;
  return make_float4(s0.x - xr, s0.x + xr, s0.y - yr, s0.y + yr);
}

// 2^t for a log2-alpha that passed the skip test (t >= log2(1/255), so the
// argument and the result are normal numbers and flushing subnormals changes
// nothing): the hardware base-2 exponential, PTX ex2.approx.ftz
__device__ __forceinline__ float exp2_alpha(float t) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  return r;
}

// one pixel whose log2-alpha t passed the skip test
__device__ __forceinline__ void accumulate(float t, const float4 &b, float c, float &T, float &C0, float &C1, float &C2,
                                           bool &done) {
  const float alpha = fminf(0.99f, exp2_alpha(t));
  const float tT = T * (1.0f - alpha);
  if (tT < 1e-4f) {
    done = true;
    return;
  }
  const float w = alpha * T;
  C0 += b.z * w;
  C1 += b.w * w;
  C2 += c * w;
  T = tT;
}

// one pixel against one staged splat
__device__ __forceinline__ void blend_one(const float4 &a, const float4 &b, float c, float fx, float fy, float &T,
                                          float &C0, float &C1, float &C2, bool &done) {
  const float dx = a.x - fx, dy = a.y - fy;
  const float q = dx * (a.z * dx + a.w * dy) + b.x * dy * dy;
  if (q > 0.0f) return;
  const float t = q + b.y;
  if (t < LOG2_SKIP) return;
  const float alpha = fminf(0.99f, exp2_alpha(t));
  const float tT = T * (1.0f - alpha);
  if (tT < 1e-4f) { done = true; return; }
  const float w = alpha * T;
  C0 += b.z * w;
  C1 += b.w * w;
  C2 += c * w;
  T = tT;
}

// Persistent CTAs of TW*TH/2 threads take tiles in the given order from a
// work counter, one tile at a time.  Warp w owns the 8x8 pixel block
// (w mod TW/8, w div TW/8) of the tile, lane l its pixels (l mod 8, l div 8)
// and (l mod 8, l div 8 + 4); a warp passes over the staged splats whose
// alpha box misses its block.
// Processing order of the tiles for the persistent kernels (segment sort,
// blend): by descending pair count in power-of-two classes, empty tiles last,
// so that the longest tiles start first and none is left for the end of the
// launch.  Also resets the work counters work[0..2].
__global__ void __launch_bounds__(1024) tile_order_kernel(const uint2 *ranges, int ntiles, uint32_t *order,
                                                          uint32_t *work) {
  __shared__ uint32_t cnt[33], off[33];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
  __syncthreads();
  // per warp, lanes of one class add once (match + leader)
  for (int b = threadIdx.x & ~31; b < ntiles; b += blockDim.x) {
    const int t = b + lane;
    int cls = -1;
    if (t < ntiles) {
      const uint2 rg = ranges[t];
      const uint32_t c = rg.y - rg.x;
      cls = c ? 32 - __clz(c) : 0;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, cls);
    if (cls >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[cls], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t o = 0;
    for (int k = 32; k >= 0; --k) {
      off[k] = o;
      o += cnt[k];
    }
    work[0] = 0;
    work[1] = 0;
    work[2] = 0;
  }
  __syncthreads();
  for (int b = threadIdx.x & ~31; b < ntiles; b += blockDim.x) {
    const int t = b + lane;
    int cls = -1;
    if (t < ntiles) {
      const uint2 rg = ranges[t];
      const uint32_t c = rg.y - rg.x;
      cls = c ? 32 - __clz(c) : 0;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, cls);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (cls >= 0 && lane == leader) base = atomicAdd(&off[cls], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (cls >= 0) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
  }
}

constexpr int kBlendPolls = 1 << 20;  // bound of each staging wait (try_wait polls)

// Staged splat j of a batch: float4 index of its record in the staging
// area, where records come in groups of four, 256 bytes apart (the 128-byte
// aligned destinations of the gather loads), 48 bytes each within a group.
__device__ __forceinline__ int rec_slot(int j) { return (j >> 2) * 16 + (j & 3) * 3; }

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH / 2, 8) blend_kernel(const uint2 *ranges, const uint32_t *vals,
                                                          const uint64_t *packed, uint32_t idx_mask, Splats sp,
                                                          uint32_t ncap, vm3dgs_camera cam, float bg0, float bg1,
                                                          float bg2, float *img, const uint32_t *order,
                                                          uint32_t ntiles, uint32_t *work,
                                                          const __grid_constant__ CUtensorMap rec_map, int use_tma,
                                                          Ctl *ctl) {
  static_assert(TW % 8 == 0 && TH % 8 == 0, "tiles are made of 8x8 blocks");
  constexpr int NT = TW * TH / 2, BS = 2 * NT, NW = NT / 32;
  // the batch's records: raw as loaded, then rewritten in place for the
  // blend (log2-domain conic and opacity)
  __shared__ __align__(128) float4 s_rec[BS / 4 * 16];
  __shared__ __align__(16) uint64_t s_key[BS + 2];  // the batch's sorted keys (or values), bulk-copied
  __shared__ __align__(8) uint64_t s_bar[2];        // [0] keys, [1] records
  __shared__ uint8_t s_blocks[BS];      // bit w: the alpha box meets warp w's block
  __shared__ uint16_t s_list[NW][BS];   // per warp, the record slots of the staged splats meeting its block, in order
  __shared__ uint32_t s_tile;
  const int W = cam.width, H = cam.height;
  const int gx = (W + TW - 1) / TW;
  if (use_tma && threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t ph = 0;    // parity of the staging barriers' current phase (each completes once per batch)
  bool first = true;  // a CTA's first tile is its index in the order; later ones come from the counter
  for (;;) {
  if (threadIdx.x == 0) {
    const uint32_t w = first ? blockIdx.x : gridDim.x + atomicAdd(work, 1u);
    s_tile = w < ntiles ? order[w] : 0xFFFFFFFFu;
  }
  first = false;
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile == 0xFFFFFFFFu) break;
  const int tx = (int)tile % gx, ty = (int)tile / gx;
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int bx = tx * TW + (warp % (TW / 8)) * 8, by = ty * TH + (warp / (TW / 8)) * 8;
  const int px = bx + (lane & 7), py0 = by + (lane >> 3), py1 = py0 + 4;
  const bool in0 = px < W && py0 < H, in1 = px < W && py1 < H;
  const float fx = (float)px + 0.5f, fy0 = (float)py0 + 0.5f, fy1 = (float)py1 + 0.5f;
  const uint2 rg = ranges[tile];
  const int n = (int)(rg.y - rg.x);
  bool done0 = !in0, done1 = !in1;
  float T0 = 1.0f, A0 = 0.0f, B0 = 0.0f, D0 = 0.0f;
  float T1 = 1.0f, A1 = 0.0f, B1 = 0.0f, D1 = 0.0f;
  for (int r0 = 0; r0 < n; r0 += BS) {
    if (__syncthreads_count(done0 && done1) == NT) break;
    const int cnt = min(BS, n - r0);
    const int64_t first_pair = (int64_t)rg.x + r0;
    if (use_tma) {
      // the batch's keys: one bulk copy of the 16-byte-aligned span around them
      const int esz = packed ? 8 : 4, per16 = 16 / esz;
      const int64_t a0 = first_pair & ~(int64_t)(per16 - 1);
      const int lead = (int)(first_pair - a0);
      const uint32_t bytes = (uint32_t)(((lead + cnt) * esz + 15) & ~15);
      if (threadIdx.x == 0) {
        proxy_fence_shared();
        mbar_arrive_expect(&s_bar[0], bytes);
        bulk_load(s_key, packed ? (const void *)(packed + a0) : (const void *)(vals + a0), bytes, &s_bar[0]);
      }
      bool ok = mbar_wait(&s_bar[0], ph, kBlendPolls);
      // the records: thread t gathers those of staged splats 4t .. 4t+3
      const int ng = (cnt + 3) / 4;
      if (threadIdx.x == 0) mbar_arrive_expect(&s_bar[1], (uint32_t)(ng * 4 * 48));
      const uint32_t *k32 = reinterpret_cast<const uint32_t *>(s_key);
      for (int t = threadIdx.x; t < ng; t += NT) {
        int rows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = lead + min(4 * t + q, cnt - 1);
          uint32_t g = packed ? (uint32_t)s_key[j] & idx_mask : k32[j];
          rows[q] = (int)(g < ncap ? g : 0u);  // (only after a timed-out sort or wait)
        }
        proxy_fence_shared();
        tma_gather4(&s_rec[t * 16], &rec_map, 0, rows[0], rows[1], rows[2], rows[3], &s_bar[1]);
      }
      ok = mbar_wait(&s_bar[1], ph, kBlendPolls) && ok;
      if (!ok) {
        atomicCAS(&ctl->status, 0, VM3DGS_E_TIMEOUT);
        mbar_wait(&s_bar[1], ph, kBlendPolls);  // the gathers still in flight land before the area is reused
      }
      ph ^= 1u;
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = (int)threadIdx.x + h * NT;
        if (k < cnt) {
          uint32_t g = packed ? (uint32_t)packed[first_pair + k] & idx_mask : vals[first_pair + k];
          if (g >= ncap) g = 0;  // only after a timed-out sort
          const int o = rec_slot(k);
          s_rec[o] = sp.rec[3 * g];
          s_rec[o + 1] = sp.rec[3 * g + 1];
          s_rec[o + 2] = sp.rec[3 * g + 2];
        }
      }
      __syncthreads();
    }
    // rewrite each staged record for the blend, and mark the 8x8 blocks
    // (pixel centres) of the tile that its alpha box meets
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = (int)threadIdx.x + h * NT;
      if (k < cnt) {
        const int o = rec_slot(k);
        const float4 r0v = s_rec[o], r1v = s_rec[o + 1];
        const float4 bb = alpha_box(r0v, r1v);
        s_rec[o] = make_float4(r0v.x, r0v.y, -0.5f * LOG2E * r0v.z, -LOG2E * r0v.w);
        s_rec[o + 1] = make_float4(-0.5f * LOG2E * r1v.x, __log2f(r1v.y), r1v.z, r1v.w);
        uint32_t m = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const float x0 = (float)(tx * TW + (w % (TW / 8)) * 8), y0 = (float)(ty * TH + (w / (TW / 8)) * 8);
          const bool miss = bb.y < x0 + 0.5f || bb.x > x0 + 7.5f || bb.w < y0 + 0.5f || bb.z > y0 + 7.5f;
          m |= miss ? 0u : 1u << w;
        }
        s_blocks[k] = (uint8_t)m;
      }
    }
    __syncthreads();
    // this warp's list: the staged splats whose alpha box meets its block
    int nl = 0;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const int j = c0 + lane;
      const bool meets = j < cnt && ((s_blocks[j] >> warp) & 1u);
      const uint32_t bal = __ballot_sync(0xffffffffu, meets);
      if (meets) s_list[warp][nl + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)rec_slot(j);
      nl += __popc(bal);
    }
    __syncwarp();
    // both pixels share x: the exponents of the two in packed FP32 pairs
    auto expo = [&](const float4 &a, const float4 &b, float2 &q, float2 &t) {
      const float dx = a.x - fx;
      const float2 dy = __fadd2_rn(make_float2(a.y, a.y), make_float2(-fy0, -fy1));
      const float ad = a.z * dx;
      const float2 inner = __ffma2_rn(make_float2(a.w, a.w), dy, make_float2(ad, ad));
      const float2 cdy = __fmul2_rn(make_float2(b.x, b.x), dy);
      q = __ffma2_rn(make_float2(dx, dx), inner, __fmul2_rn(cdy, dy));
      t = __fadd2_rn(q, make_float2(b.y, b.y));
    };
    auto composite = [&](int o, const float4 &b, const float2 &q, const float2 &t) {
      const bool go0 = !done0 && q.x <= 0.0f && t.x >= LOG2_SKIP;
      const bool go1 = !done1 && q.y <= 0.0f && t.y >= LOG2_SKIP;
      if (!(go0 || go1)) return;
      const float c = s_rec[o + 2].x;
      if (go0) accumulate(t.x, b, c, T0, A0, B0, D0, done0);
      if (go1) accumulate(t.y, b, c, T1, A1, B1, D1, done1);
    };
    // two splats a round: their loads and exponents are independent and go
    // together; they are composited in list order (the second sees the
    // first's transmittance and stop flags), so every pixel takes the same
    // operations in the same order as one splat a round
    int i = 0;
    for (; i + 1 < nl && !(done0 && done1); i += 2) {
      const int o1 = s_list[warp][i], o2 = s_list[warp][i + 1];
      const float4 a1 = s_rec[o1], b1 = s_rec[o1 + 1], a2 = s_rec[o2], b2 = s_rec[o2 + 1];
      float2 q1, t1, q2, t2;
      expo(a1, b1, q1, t1);
      expo(a2, b2, q2, t2);
      composite(o1, b1, q1, t1);
      composite(o2, b2, q2, t2);
    }
    if (i < nl && !(done0 && done1)) {
      const int o = s_list[warp][i];
      const float4 a = s_rec[o], b = s_rec[o + 1];
      float2 q, t;
      expo(a, b, q, t);
      composite(o, b, q, t);
    }
  }
  const int64_t HW = (int64_t)W * H;
  if (in0) {
    const int64_t o = (int64_t)py0 * W + px;
    img[o] = A0 + T0 * bg0;
    img[HW + o] = B0 + T0 * bg1;
    img[2 * HW + o] = D0 + T0 * bg2;
  }
  if (in1) {
    const int64_t o = (int64_t)py1 * W + px;
    img[o] = A1 + T1 * bg0;
    img[HW + o] = B1 + T1 * bg1;
    img[2 * HW + o] = D1 + T1 * bg2;
  }
  __syncthreads();  // the next tile reuses the staging arrays and s_tile
  }
}

// All tiles of all views of a batch: a persistent grid takes (view, tile)
// items from a counter; each view has its own tile shape (16x16, 32x8 or
// 8x8; for 8x8 only 64 of the 256 threads own pixels) and image.
__global__ void __launch_bounds__(256) blend_batched_kernel(const uint2 *ranges, const uint32_t *vals, Splats sp,
                                                           uint32_t ncap, const ViewTable *vt, float bg0, float bg1,
                                                           float bg2, const uint32_t *order, uint32_t *work) {
  constexpr int BS = 256;
  __shared__ float4 s0[BS];
  __shared__ float4 s1[BS];
  __shared__ float s2[BS];
  __shared__ int s_item;
  const int nv = vt->n;
  const int total = vt->tile_off[nv];
  for (;;) {
    if (threadIdx.x == 0) {
      const int w = (int)atomicAdd(work, 1u);
      s_item = w < total ? (int)order[w] : -1;
    }
    __syncthreads();
    const int gt = s_item;
    if (gt < 0) break;
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (vt->tile_off[mid] <= gt) lo = mid; else hi = mid - 1;
    }
    const int v = lo;
    const int W = vt->cam[v].width, H = vt->cam[v].height, TW = vt->cam[v].tile_w, TH = vt->cam[v].tile_h;
    const int gx = vt->gx[v], local = gt - vt->tile_off[v];
    const int tx = local % gx, ty = local / gx;
    const bool owner = (int)threadIdx.x < TW * TH;
    const int px = tx * TW + (int)threadIdx.x % TW, py = ty * TH + (int)threadIdx.x / TW;
    const bool inside = owner && px < W && py < H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 rg = ranges[gt];
    const int n = (int)(rg.y - rg.x);
    bool done = !inside;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    for (int r0 = 0; r0 < n; r0 += BS) {
      if (__syncthreads_count(done) == BS) break;
      const int idx = r0 + (int)threadIdx.x;
      if (idx < n) {
        uint32_t g = vals[rg.x + idx];
        if (g >= ncap) g = 0;  // only after a timed-out sort
        float4 a, b;
        float c;
        stage(sp, g, a, b, c);
        s0[threadIdx.x] = a;
        s1[threadIdx.x] = b;
        s2[threadIdx.x] = c;
      }
      __syncthreads();
      const int cnt = min(BS, n - r0);
      for (int j = 0; !done && j < cnt; ++j) blend_one(s0[j], s1[j], s2[j], fx, fy, T, C0, C1, C2, done);
    }
    if (inside) {
      float *img = vt->img[v];
      const int64_t HW = (int64_t)W * H, o = (int64_t)py * W + px;
      img[o] = C0 + T * bg0;
      img[HW + o] = C1 + T * bg1;
      img[2 * HW + o] = C2 + T * bg2;
    }
    __syncthreads();
  }
}

}  // namespace

void launch_tile_order(const uint2 *ranges, int ntiles, uint32_t *order, uint32_t *work, cudaStream_t st) {
  tile_order_kernel<<<1, 1024, 0, st>>>(ranges, ntiles, order, work);
}

void launch_blend_batched(const uint2 *ranges, const uint32_t *vals, const Splats &sp, int64_t ncap_total,
                          const ViewTable *vt, int ntiles, const float bg[3], uint32_t *order, uint32_t *work,
                          cudaStream_t st) {
  tile_order_kernel<<<1, 1024, 0, st>>>(ranges, ntiles, order, work);
  prefer_shared((const void *)blend_batched_kernel);
  blend_batched_kernel<<<full_wave((const void *)blend_batched_kernel, 256, 0), 256, 0, st>>>(
      ranges, vals, sp, (uint32_t)ncap_total, vt, bg[0], bg[1], bg[2], order, work);
}

bool encode_rec_map(const float4 *rec, int64_t n, CUtensorMap *out) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // rows of 12 floats (the 48-byte record), one row per box (gather loads)
  const cuuint64_t dim[2] = {12, (cuuint64_t)(n > 0 ? n : 1)};
  const cuuint64_t str[1] = {48};
  const cuuint32_t box[2] = {12, 1}, estr[2] = {1, 1};
  return enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float4 *>(rec), dim, str, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_blend(const uint2 *ranges, const uint32_t *vals, const uint64_t *packed, uint32_t idx_mask,
                  const Splats &sp, int64_t ncap, const vm3dgs_camera &cam, const float bg[3], float *image,
                  uint32_t *order, uint32_t *work, const CUtensorMap *rec_map, Ctl *ctl, cudaStream_t st) {
  const int gx = (cam.width + cam.tile_w - 1) / cam.tile_w, gy = (cam.height + cam.tile_h - 1) / cam.tile_h;
  const int nt = gx * gy;
  const uint32_t nc = (uint32_t)ncap;
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  const CUtensorMap &map = rec_map ? *rec_map : none;
  const int tma = rec_map ? 1 : 0;
  prefer_shared((const void *)blend_kernel<16, 16>);
  prefer_shared((const void *)blend_kernel<8, 8>);
  prefer_shared((const void *)blend_kernel<32, 8>);
  if (cam.tile_w == 16 && cam.tile_h == 16)
    blend_kernel<16, 16><<<wave_grid((const void *)blend_kernel<16, 16>, 128, 0, nt, 1), 128, 0, st>>>(
        ranges, vals, packed, idx_mask, sp, nc, cam, bg[0], bg[1], bg[2], image, order, (uint32_t)nt, work, map, tma,
        ctl);
  else if (cam.tile_w == 8 && cam.tile_h == 8)
    blend_kernel<8, 8><<<wave_grid((const void *)blend_kernel<8, 8>, 32, 0, nt, 1), 32, 0, st>>>(
        ranges, vals, packed, idx_mask, sp, nc, cam, bg[0], bg[1], bg[2], image, order, (uint32_t)nt, work, map, tma,
        ctl);
  else
    blend_kernel<32, 8><<<wave_grid((const void *)blend_kernel<32, 8>, 128, 0, nt, 1), 128, 0, st>>>(
        ranges, vals, packed, idx_mask, sp, nc, cam, bg[0], bg[1], bg[2], image, order, (uint32_t)nt, work, map, tma,
        ctl);
}

}  // namespace vm
