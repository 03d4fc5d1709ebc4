// Prefetching for the next frame with the learned network (see
// vm3dgs_prefetch in include/vm3dgs.h): network input built on the device
// from the camera and this frame's request words, training targets from the
// request words, and placement of predicted pages into entries this frame did
// not use, within the staging budget the frame left unused.  One CTA runs
// each of the small steps so that they are deterministic.
#include <cstring>
#include <string>

#include "mlp.cuh"
#include "prefetcher.cuh"
#include "block_sel.cuh"
#include "renderer.cuh"

namespace vm {
namespace {


struct FeatArgs {
  vm3dgs_camera cam, prev;
  const float4 *centroid;  // [NP] (x, y, z, radius)
  const uint32_t *req;
  int32_t NP, n_out;
  float cx, cy, cz, half;  // scene centre and half-extent
  float *x;                // [12 + n_out / 16]
  int32_t *base;
};

__global__ void __launch_bounds__(RT) features_kernel(FeatArgs a) {
  __shared__ unsigned long long best;
  if (threadIdx.x == 0) best = ~0ull;
  __syncthreads();
  const float px = a.cam.campos[0], py = a.cam.campos[1], pz = a.cam.campos[2];
  unsigned long long mine = ~0ull;
  for (int p = threadIdx.x; p < a.NP; p += RT) {
    const float4 c = a.centroid[p];
    const float dx = c.x - px, dy = c.y - py, dz = c.z - pz;
    const float d2 = dx * dx + dy * dy + dz * dz;
    const unsigned long long k = ((unsigned long long)__float_as_uint(d2) << 32) | (uint32_t)p;
    mine = k < mine ? k : mine;
  }
  atomicMin(&best, mine);
  __syncthreads();
  const int pstar = (int)(best & 0xFFFFFFFFull);
  int base = pstar - a.n_out / 2;
  const int hi = a.NP - a.n_out > 0 ? a.NP - a.n_out : 0;
  base = base < 0 ? 0 : (base > hi ? hi : base);
  if (threadIdx.x == 0) {
    if (a.base) *a.base = base;
    const float *f = a.cam.view + 8, *g = a.prev.view + 8;
    const float inv = 1.0f / a.half, vinv = 1.0f / (0.01f * a.half);
    a.x[0] = (px - a.cx) * inv;
    a.x[1] = (py - a.cy) * inv;
    a.x[2] = (pz - a.cz) * inv;
    a.x[3] = f[0]; a.x[4] = f[1]; a.x[5] = f[2];
    a.x[6] = (px - a.prev.campos[0]) * vinv;
    a.x[7] = (py - a.prev.campos[1]) * vinv;
    a.x[8] = (pz - a.prev.campos[2]) * vinv;
    a.x[9] = (f[0] - g[0]) * 10.0f;
    a.x[10] = (f[1] - g[1]) * 10.0f;
    a.x[11] = (f[2] - g[2]) * 10.0f;
  }
  const int nb = a.n_out / 16;
  for (int b = threadIdx.x; b < nb; b += RT) {
    int cnt = 0;
    for (int k = 0; k < 16; ++k) {
      const int p = base + 16 * b + k;
      if (p < a.NP && a.req[p] != 0u) ++cnt;
    }
    a.x[12 + b] = (float)cnt / 16.0f;
  }
}

// labels of the window's pages; with accumulate, OR-ed into what y holds
// (the pages requested in any frame of a horizon)
__global__ void labels_kernel(const uint32_t *req, int32_t NP, int32_t n_out, const int32_t *base_p, float *y,
                              float *mask, int accumulate) {
  const int base = *base_p;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_out; j += gridDim.x * blockDim.x) {
    const int p = base + j;
    const bool in = p < NP;
    const float l = (in && req[p] != 0u) ? 1.0f : 0.0f;
    y[j] = accumulate ? fmaxf(y[j], l) : l;
    mask[j] = in ? 1.0f : 0.0f;
  }
}

struct PlaceArgs {
  Ctl *ctl;
  const float *logits;     // [n_out]
  const int32_t *base_p;
  const uint32_t *req;
  const float4 *centroid;
  const float *err;
  int32_t *pt_lod, *pt_last, *pt_slot;
  uint8_t *pf_flag, *mask;
  uint64_t *cand, *free_keys;
  int4 *copies;
  int64_t *copy_seg;
  int32_t *count;
  int32_t NP, P, Smax, levels, fanout, page_size, n_out, lod_on, rec, cand_cap, free_cap;
  int64_t budget;
  float threshold, f_px;
  float campos[3];
};

// order-preserving map of a float to uint32 (larger float -> larger key)
__device__ __forceinline__ uint32_t ordered(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(RT) place_kernel(PlaceArgs a) {
  extern __shared__ uint64_t s_keys[];
  __shared__ ScanSmem sm;
  __shared__ int m_l[kMaxLevels], S_l[kMaxLevels], fresh_start[kMaxLevels + 1], n_lvl[kMaxLevels];
  Ctl *ctl = a.ctl;
  const int tid = threadIdx.x;
  const int frame_now = ctl->frame - 1;
  const int L = a.levels, Smax = a.Smax;
  const int base = *a.base_p;
  const float tau = ctl->tau;
  if (tid < kMaxLevels) {
    int m = a.page_size, S = 1;
    for (int l = 0; l < tid; ++l) { m /= a.fanout; S *= a.fanout; }
    m_l[tid] = m;
    S_l[tid] = S;
  }
  // levels resident per page
  for (int p = tid; p < a.NP; p += RT) a.mask[p] = 0;
  __syncthreads();
  for (int e = tid; e < a.P; e += RT) {
    const int l = a.pt_lod[e];
    if (l < 0) continue;
    for (int s = 0; s < S_l[l]; ++s) {
      const int p = a.pt_slot[(int64_t)e * Smax + s];
      if (p >= 0) atomicOr(reinterpret_cast<unsigned int *>(a.mask + (p & ~3)), (1u << l) << (8 * (p & 3)));
    }
  }
  __syncthreads();
  // candidates: above threshold, not requested, not resident at their level
  int64_t nc = 0, tot;
  for (int c = 0; c < a.n_out; c += RT) {
    const int j = c + tid, p = base + j;
    int f = 0, lev = 0;
    float lg = 0.0f;
    if (j < a.n_out && p < a.NP) {
      lg = a.logits[j];
      if (a.lod_on && L > 1) {
        const float4 cc = a.centroid[p];
        const float dx = cc.x - a.campos[0], dy = cc.y - a.campos[1], dz = cc.z - a.campos[2];
        const float d = fmaxf(sqrtf(dx * dx + dy * dy + dz * dz) - cc.w, 0.2f);
        for (int l = L - 1; l >= 1; --l)
          if ((a.f_px * a.err[(int64_t)p * L + l]) / d <= tau) { lev = l; break; }
      }
      f = lg > a.threshold && a.req[p] == 0u && !((a.mask[p] >> lev) & 1);
    }
    const int64_t pos = bscan(f, &tot, sm);
    if (f && nc + pos < a.cand_cap)
      a.cand[nc + pos] = ((uint64_t)(~ordered(lg)) << 32) | ((uint64_t)lev << 28) | (uint32_t)p;
    nc += tot;
  }
  if (nc > a.cand_cap) nc = a.cand_cap;
  if (nc == 0) {
    if (tid == 0) { a.copy_seg[0] = 0; *a.count = 0; }
    return;
  }
  // budget left by this frame; no prefix of more than kmax candidates fits it
  // (each costs at least a page of the coarsest level), so only the kmax
  // smallest keys need ordering
  const int64_t remaining = a.budget - ctl->streamed_bytes;
  const int64_t min_cost = (int64_t)m_l[L - 1] * a.rec;
  const int64_t kfit = remaining >= 0 ? remaining / min_cost + 1 : 1;
  if (kfit < nc && kfit <= kSmemKeys) {
    select_smallest(a.cand, (int)nc, (int)kfit, s_keys, sm);
    nc = kfit;
  } else {
    const int np2 = pow2_at_least((int)nc);
    for (int i = (int)nc + tid; i < np2; i += RT) a.cand[i] = ~0ull;
    __syncthreads();
    bitonic(a.cand, np2, s_keys);
  }
  int64_t nadm = 0, cum = 0;
  for (int c = 0; c < nc; c += RT) {
    const int i = c + tid;
    int64_t cost = 0;
    if (i < nc) cost = (int64_t)m_l[(int)((a.cand[i] >> 28) & 7ull)] * a.rec;
    const int64_t pre = bscan(cost, &tot, sm);
    int64_t t2;
    bscan((i < nc && cum + pre + cost <= remaining) ? 1 : 0, &t2, sm);
    nadm += t2;
    cum += tot;
  }
  if (nadm == 0) {
    if (tid == 0) { a.copy_seg[0] = 0; *a.count = 0; }
    return;
  }
  // per-level ranks (stored in the low bits' place: reuse cand's page field order)
  for (int l = 0; l < L; ++l) {
    int64_t b0 = 0;
    for (int c = 0; c < nadm; c += RT) {
      const int i = c + tid;
      const int f = (i < nadm && (int)((a.cand[i] >> 28) & 7ull) == l) ? 1 : 0;
      bscan(f, &tot, sm);
      b0 += tot;
    }
    if (tid == 0) n_lvl[l] = (int)b0;
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int l = 0; l < L; ++l) { fresh_start[l] = acc; acc += (n_lvl[l] + S_l[l] - 1) / S_l[l]; }
    fresh_start[L] = acc;
  }
  __syncthreads();
  // free entries: not used this frame, least recently used first (only the
  // fresh_start[L] least recently used are taken: select them)
  int64_t nfree = 0;
  for (int c = 0; c < a.P; c += RT) {
    const int e = c + tid;
    const int f = (e < a.P && a.pt_last[e] < frame_now) ? 1 : 0;
    const int64_t pos = bscan(f, &tot, sm);
    if (f) a.free_keys[nfree + pos] = ((uint64_t)(uint32_t)(a.pt_last[e] + 1) << 32) | (uint32_t)e;
    nfree += tot;
  }
  __syncthreads();
  if (fresh_start[L] > 0 && fresh_start[L] < nfree && fresh_start[L] <= kSmemKeys) {
    select_smallest(a.free_keys, (int)nfree, fresh_start[L], s_keys, sm);
  } else if (fresh_start[L] > 0) {
    const int fp2 = pow2_at_least((int)nfree);
    for (int i = (int)nfree + tid; i < fp2; i += RT) a.free_keys[i] = ~0ull;
    __syncthreads();
    bitonic(a.free_keys, fp2, s_keys);
  }
  const int nf = fresh_start[L] < nfree ? fresh_start[L] : (int)nfree;
  for (int64_t x = tid; x < (int64_t)nf * Smax; x += RT) {
    const int k = (int)(x / Smax), s = (int)(x % Smax);
    const int e = (int)(a.free_keys[k] & 0xFFFFFFFFull);
    a.pt_slot[(int64_t)e * Smax + s] = -1;
    a.pf_flag[(int64_t)e * Smax + s] = 0;
    if (s == 0) {
      int l = 0;
      while (l + 1 < L && fresh_start[l + 1] <= k) ++l;
      a.pt_lod[e] = l;
      a.pt_last[e] = frame_now;
    }
  }
  __syncthreads();
  // placement and copy list (priority order)
  int64_t ncopy = 0, nseg = 0, sbytes = 0;
  int64_t rank_base[kMaxLevels] = {0, 0, 0, 0, 0, 0};
  for (int c = 0; c < nadm; c += RT) {
    const int i = c + tid;
    int lev = 0, p = 0;
    if (i < nadm) { lev = (int)((a.cand[i] >> 28) & 7ull); p = (int)(a.cand[i] & 0x0FFFFFFFull); }
    // rank of this candidate within its level
    int64_t my_rank = 0;
    for (int l = 0; l < L; ++l) {
      const int f = (i < nadm && lev == l) ? 1 : 0;
      const int64_t pos = bscan(f, &tot, sm);
      if (f) my_rank = rank_base[l] + pos;
      rank_base[l] += tot;
    }
    int placed = 0;
    int64_t slot = -1;
    if (i < nadm) {
      const int k = fresh_start[lev] + (int)(my_rank / S_l[lev]);
      if (k < nfree) {
        const int e = (int)(a.free_keys[k] & 0xFFFFFFFFull);
        slot = (int64_t)e * Smax + my_rank % S_l[lev];
        a.pt_slot[slot] = p;
        a.pf_flag[slot] = 1;
        placed = 1;
      }
    }
    const int64_t bytes = placed ? (int64_t)m_l[lev] * a.rec : 0;
    const int64_t segs = (bytes + kCopySeg - 1) / kCopySeg;
    int64_t ts, tb;
    const int64_t pos = bscan(placed, &tot, sm);
    const int64_t spos = bscan(segs, &ts, sm);
    bscan(bytes, &tb, sm);
    if (placed) {
      a.copies[ncopy + pos] = make_int4(p, lev, (int)(slot / Smax), (int)(slot % Smax));
      a.copy_seg[ncopy + pos] = nseg + spos;
    }
    ncopy += tot;
    nseg += ts;
    sbytes += tb;
  }
  if (tid == 0) {
    a.copy_seg[ncopy] = nseg;
    *a.count = (int)ncopy;
    ctl->acc_prefetched_pages += ncopy;
    ctl->acc_prefetched_bytes += sbytes;
  }
}

}  // namespace

void launch_prefetch_features(const vm3dgs_renderer *r, const uint32_t *req, int n_out, const vm3dgs_camera &cam,
                              const vm3dgs_camera &prev, float *x, int32_t *base, cudaStream_t st) {
  FeatArgs a{};
  a.cam = cam;
  a.prev = prev;
  a.centroid = r->at<float4>(r->lay.centroid);
  a.req = req;
  a.NP = (int32_t)r->dims.NP;
  a.n_out = n_out;
  a.cx = r->scene_center[0]; a.cy = r->scene_center[1]; a.cz = r->scene_center[2];
  a.half = r->scene_half;
  a.x = x;
  a.base = base;
  features_kernel<<<1, RT, 0, st>>>(a);
}

}  // namespace vm

using namespace vm;

extern "C" int vm3dgs_prefetch_features(vm3dgs_renderer *r, int32_t n_out, const vm3dgs_camera *cam,
                                        const vm3dgs_camera *prev, float *x_dev, int32_t *base_dev, void *stream) {
  if (!r || !cam || !prev || !x_dev) return fail(VM3DGS_E_INVAL, "null argument");
  if (n_out <= 0 || n_out % 16) return fail(VM3DGS_E_INVAL, "n_out must be a positive multiple of 16");
  if (r->state < 1) return fail(VM3DGS_E_STATE, "features before render_feedback");
  launch_prefetch_features(r, r->req_buf(r->fb_buf), n_out, *cam, *prev, x_dev, base_dev, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, cudaGetErrorString(e));
}

extern "C" int vm3dgs_prefetch_labels(vm3dgs_renderer *r, int32_t n_out, const int32_t *base_dev, float *y_dev,
                                      float *mask_dev, int32_t accumulate, void *stream) {
  if (!r || !base_dev || !y_dev || !mask_dev) return fail(VM3DGS_E_INVAL, "null argument");
  if (n_out <= 0) return fail(VM3DGS_E_INVAL, "n_out must be positive");
  labels_kernel<<<(n_out + 255) / 256, 256, 0, (cudaStream_t)stream>>>(r->req_buf(r->fb_buf),
                                                                      (int32_t)r->dims.NP, n_out, base_dev, y_dev,
                                                                      mask_dev, accumulate ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, cudaGetErrorString(e));
}

extern "C" int vm3dgs_prefetch(vm3dgs_renderer *r, vm3dgs_prefetcher *p, const vm3dgs_camera *cam,
                               const vm3dgs_camera *prev, float threshold, void *stream, void *copy_stream) {
  if (!r || !p || !cam || !prev) return fail(VM3DGS_E_INVAL, "null argument");
  if (r->state < 2) return fail(VM3DGS_E_STATE, "prefetch before update_residency");
  if (r->staged)
    return fail(VM3DGS_E_STATE, "prefetch streams from page-locked scene memory; a scene opened from a file has none");
  const int n_out = p->cfg.n_out;
  if (n_out % 16 || p->cfg.n_in != 12 + n_out / 16)
    return fail(VM3DGS_E_INVAL, "network must have n_in = 12 + n_out / 16 and n_out a multiple of 16");
  // The whole step runs on the copy stream after this frame's page-table
  // update, concurrently with the frame's render: it reads a copy of this
  // frame's requests (so the next page determination waits only for the
  // copy) and writes only entries the frame does not use.  The next update
  // waits for it.
  cudaStream_t cst = copy_stream ? (cudaStream_t)copy_stream : (cudaStream_t)stream;
  cudaStreamWaitEvent(cst, r->res_done, 0);
  cudaStream_t st = cst;
  const int span = r->span_begin(VM3DGS_STAGE_PREFETCH, st);
  uint32_t *req = r->at<uint32_t>(r->lay.pf_req);
  // the buffer the last update read (page determination of the next frame
  // writes the other one)
  cudaMemcpyAsync(req, r->req_buf(r->res_buf), 4 * r->dims.NP, cudaMemcpyDeviceToDevice, st);
  cudaEventRecord(r->pf_req_done, st);
  r->pf_req_pending = true;
  r->pf_req_buf = r->res_buf;
  const PfLayout &PL = p->lay;
  float *x = p->at<float>(PL.feat);
  int32_t *base = r->at<int32_t>(r->lay.pf_base);
  launch_prefetch_features(r, req, n_out, *cam, *prev, x, base, st);
  float *logits = p->at<float>(PL.logits);
  pf_forward(p, x, 1, logits, st);
  const vm3dgs_scene *s = r->scene;
  PlaceArgs a{};
  a.ctl = r->at<Ctl>(r->lay.ctl);
  a.logits = logits;
  a.base_p = base;
  a.req = req;
  a.centroid = r->at<float4>(r->lay.centroid);
  a.err = r->at<float>(r->lay.err);
  a.pt_lod = r->at<int32_t>(r->lay.pt_lod);
  a.pt_last = r->at<int32_t>(r->lay.pt_last);
  a.pt_slot = r->at<int32_t>(r->lay.pt_slot);
  a.pf_flag = r->at<uint8_t>(r->lay.pf_flag);
  a.mask = r->at<uint8_t>(r->lay.pf_mask);
  a.cand = r->at<uint64_t>(r->lay.pf_cand);
  a.free_keys = r->at<uint64_t>(r->lay.free_keys);
  a.copies = r->at<int4>(r->lay.pf_copies);
  a.copy_seg = r->at<int64_t>(r->lay.pf_copy_seg);
  a.count = r->at<int32_t>(r->lay.pf_count);
  a.NP = (int32_t)r->dims.NP;
  a.P = r->P;
  a.Smax = (int32_t)r->dims.Smax;
  a.levels = s->levels;
  a.fanout = s->fanout;
  a.page_size = s->page_size;
  a.n_out = n_out;
  a.lod_on = r->prm.lod;
  a.rec = r->rec;
  a.cand_cap = r->dims.ukey_cap;
  a.free_cap = r->dims.free_cap;
  a.budget = r->prm.staging_bytes;
  a.threshold = threshold;
  a.f_px = cam->fy;
  for (int k = 0; k < 3; ++k) a.campos[k] = cam->campos[k];
  const int smem = kSmemKeys * (int)sizeof(uint64_t);
  max_dynamic_smem((const void *)place_kernel, smem);
  place_kernel<<<1, RT, smem, st>>>(a);
  StreamArgs sa{};
  sa.count = a.count;
  sa.copies = a.copies;
  sa.copy_seg = a.copy_seg;
  sa.host = r->host_dev;
  for (int l = 0; l < s->levels; ++l) sa.level_off[l] = s->fmt_off(r->fmt)[l];
  sa.page_size = s->page_size;
  sa.fanout = s->fanout;
  sa.rec = r->rec;
  sa.pool = r->pool;
  sa.slot_bytes = r->slot_bytes;
  launch_stream(sa, cst);
  r->span_end(span, 7, cst);
  cudaEventRecord(r->pf_done, cst);
  cudaEventRecord(r->copy_done, cst);
  r->pf_pending = true;
  r->copy_pending = true;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, cudaGetErrorString(e));
}
