// Front-to-back alpha blending per image tile (Sec. 4.2: the paper blends
// quads in hardware; the per-pixel Gaussian and the compositing rule are
// those of Kerbl et al.).  One CTA per tile, one thread per pixel.  The
// tile's splats are staged in shared memory in batches of one splat per
// thread; a pixel stops when its transmittance would fall below 1e-4, the
// CTA stops when every pixel has.  alpha = min(0.99, o exp(power)); splats
// with alpha < 1/255 are skipped; the image is C + T * background, CHW.
#include "renderer.cuh"

namespace vm {
namespace {

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) blend_kernel(const uint2 *ranges, const uint32_t *vals, Splats sp,
                                                      uint32_t ncap, vm3dgs_camera cam, float bg0, float bg1,
                                                      float bg2, float *img) {
  constexpr int BS = TW * TH;
  __shared__ float4 s0[BS];
  __shared__ float4 s1[BS];
  __shared__ float s2[BS];
  const int W = cam.width, H = cam.height;
  const int gx = (W + TW - 1) / TW;
  const int tile = blockIdx.x;
  const int tx = tile % gx, ty = tile / gx;
  const int px = tx * TW + (int)(threadIdx.x % TW), py = ty * TH + (int)(threadIdx.x / TW);
  const bool inside = px < W && py < H;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 rg = ranges[tile];
  const int n = (int)(rg.y - rg.x);
  bool done = !inside;
  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  for (int r0 = 0; r0 < n; r0 += BS) {
    if (__syncthreads_count(done) == BS) break;
    const int idx = r0 + (int)threadIdx.x;
    if (idx < n) {
      uint32_t g = vals[rg.x + idx];
      if (g >= ncap) g = 0;  // only after a timed-out sort
      s0[threadIdx.x] = sp.s0[g];
      s1[threadIdx.x] = sp.s1[g];
      s2[threadIdx.x] = sp.s2[g];
    }
    __syncthreads();
    const int cnt = min(BS, n - r0);
    for (int j = 0; !done && j < cnt; ++j) {
      const float4 a = s0[j];
      const float4 b = s1[j];
      const float dx = a.x - fx, dy = a.y - fy;
      const float power = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
      if (power > 0.0f) continue;
      const float alpha = fminf(0.99f, b.y * __expf(power));
      if (alpha < (1.0f / 255.0f)) continue;
      const float tT = T * (1.0f - alpha);
      if (tT < 1e-4f) { done = true; break; }
      const float w = alpha * T;
      C0 += b.z * w;
      C1 += b.w * w;
      C2 += s2[j] * w;
      T = tT;
    }
  }
  if (inside) {
    const int64_t HW = (int64_t)W * H, o = (int64_t)py * W + px;
    img[o] = C0 + T * bg0;
    img[HW + o] = C1 + T * bg1;
    img[2 * HW + o] = C2 + T * bg2;
  }
}

// All tiles of all views of a batch: a persistent grid takes (view, tile)
// items from a counter; each view has its own tile shape (16x16, 32x8 or
// 8x8; for 8x8 only 64 of the 256 threads own pixels) and image.
__global__ void __launch_bounds__(256) blend_batched_kernel(const uint2 *ranges, const uint32_t *vals, Splats sp,
                                                           uint32_t ncap, const ViewTable *vt, float bg0, float bg1,
                                                           float bg2, uint32_t *work) {
  constexpr int BS = 256;
  __shared__ float4 s0[BS];
  __shared__ float4 s1[BS];
  __shared__ float s2[BS];
  __shared__ int s_item;
  const int nv = vt->n;
  const int total = vt->tile_off[nv];
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(work, 1u);
    __syncthreads();
    const int gt = s_item;
    if (gt >= total) break;
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
        s0[threadIdx.x] = sp.s0[g];
        s1[threadIdx.x] = sp.s1[g];
        s2[threadIdx.x] = sp.s2[g];
      }
      __syncthreads();
      const int cnt = min(BS, n - r0);
      for (int j = 0; !done && j < cnt; ++j) {
        const float4 a = s0[j];
        const float4 b = s1[j];
        const float dx = a.x - fx, dy = a.y - fy;
        const float power = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
        if (power > 0.0f) continue;
        const float alpha = fminf(0.99f, b.y * __expf(power));
        if (alpha < (1.0f / 255.0f)) continue;
        const float tT = T * (1.0f - alpha);
        if (tT < 1e-4f) { done = true; break; }
        const float w = alpha * T;
        C0 += b.z * w;
        C1 += b.w * w;
        C2 += s2[j] * w;
        T = tT;
      }
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

void launch_blend_batched(const uint2 *ranges, const uint32_t *vals, const Splats &sp, int64_t ncap_total,
                          const ViewTable *vt, const float bg[3], uint32_t *work, cudaStream_t st) {
  cudaMemsetAsync(work, 0, sizeof(uint32_t), st);
  blend_batched_kernel<<<148 * 6, 256, 0, st>>>(ranges, vals, sp, (uint32_t)ncap_total, vt, bg[0], bg[1], bg[2], work);
}

void launch_blend(const uint2 *ranges, const uint32_t *vals, const Splats &sp, int64_t ncap, const vm3dgs_camera &cam,
                  const float bg[3], float *image, cudaStream_t st) {
  const int gx = (cam.width + cam.tile_w - 1) / cam.tile_w, gy = (cam.height + cam.tile_h - 1) / cam.tile_h;
  const unsigned nt = (unsigned)(gx * gy);
  if (cam.tile_w == 16 && cam.tile_h == 16)
    blend_kernel<16, 16><<<nt, 256, 0, st>>>(ranges, vals, sp, (uint32_t)ncap, cam, bg[0], bg[1], bg[2], image);
  else if (cam.tile_w == 8 && cam.tile_h == 8)
    blend_kernel<8, 8><<<nt, 64, 0, st>>>(ranges, vals, sp, (uint32_t)ncap, cam, bg[0], bg[1], bg[2], image);
  else
    blend_kernel<32, 8><<<nt, 256, 0, st>>>(ranges, vals, sp, (uint32_t)ncap, cam, bg[0], bg[1], bg[2], image);
}

}  // namespace vm
