// C ABI of the per-frame path: renderer set-up over caller-owned device
// memory and the three frame calls (page determination, page-table update
// with streaming, rendering).  Every step runs in the kernels of this
// library; the host only validates arguments and enqueues work.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "renderer.cuh"

#include <mutex>
#include <unordered_map>

namespace vm {

int full_wave(const void *kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<uint64_t, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t key = (uint64_t)(uintptr_t)kernel ^ ((uint64_t)dev << 56) ^ ((uint64_t)threads << 40) ^ (uint64_t)smem;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int g = sms * per_sm;
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = g;
  return g;
}

void prefer_shared(const void *kernel) {
  static std::mutex mu;
  static std::unordered_map<uint64_t, bool> done;
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t key = (uint64_t)(uintptr_t)kernel ^ ((uint64_t)dev << 56);
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(key)) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  cudaGetLastError();
  done[key] = true;
}

void max_dynamic_smem(const void *kernel, int bytes) {
  static std::mutex mu;
  static std::unordered_map<uint64_t, int> done;
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t key = (uint64_t)(uintptr_t)kernel ^ ((uint64_t)dev << 56);
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  done[key] = bytes;
}

int wave_grid(const void *kernel, int threads, size_t smem, int64_t n, int64_t per_block) {
  const int64_t need = per_block > 0 ? (n + per_block - 1) / per_block : 1;
  const int64_t g = std::min<int64_t>(need, full_wave(kernel, threads, smem));
  return (int)std::max<int64_t>(g, 1);
}

namespace {
int64_t pow2_at_least(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}
int64_t al(int64_t x) { return (x + 255) & ~int64_t(255); }

bool cuda_ok(cudaError_t e, const char *what, int *rc) {
  if (e == cudaSuccess) return true;
  *rc = fail(VM3DGS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return false;
}

int check_cams(const vm3dgs_renderer *r, const vm3dgs_camera *cams, int n) {
  if (!cams || n <= 0) return fail(VM3DGS_E_INVAL, "no cameras");
  for (int v = 0; v < n; ++v) {
    const vm3dgs_camera &c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > r->prm.max_width || c.height > r->prm.max_height)
      return fail(VM3DGS_E_INVAL, "camera size outside the renderer's maximum");
    const bool tiles_ok = (c.tile_w == 16 && c.tile_h == 16) || (c.tile_w == 8 && c.tile_h == 8) ||
                          (c.tile_w == 32 && c.tile_h == 8);
    if (!tiles_ok) return fail(VM3DGS_E_INVAL, "tile shape must be 16x16, 8x8 or 32x8");
    const float *f = &c.view[0];
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(f[i])) return fail(VM3DGS_E_INVAL, "camera matrix is not finite");
    if (!(c.fx > 0) || !(c.fy > 0) || !std::isfinite(c.cx) || !std::isfinite(c.cy) || !std::isfinite(c.campos[0]) ||
        !std::isfinite(c.campos[1]) || !std::isfinite(c.campos[2]))
      return fail(VM3DGS_E_INVAL, "camera intrinsics are not finite");
  }
  return VM3DGS_OK;
}
}  // namespace

Dims make_dims(const vm3dgs_scene *s, const vm3dgs_params *p, int64_t P) {
  Dims d{};
  d.NP = s->n_pages;
  d.P = P;
  d.Smax = 1;
  for (int l = 1; l < s->levels; ++l) d.Smax *= s->fanout;
  const int ds = p->feedback_ds > 0 ? p->feedback_ds : 1;
  d.fb_pixels = (int64_t)((p->max_width + ds - 1) / ds) * ((p->max_height + ds - 1) / ds);
  d.ncap = P * s->page_size;
  d.nviews = p->max_views > 1 ? (p->max_views < kMaxViews ? p->max_views : kMaxViews) : 1;
  d.pair_cap = p->max_pairs > 0 ? p->max_pairs : 8 * d.ncap;
  if (p->max_pairs <= 0 && d.pair_cap < (int64_t(1) << 22)) d.pair_cap = int64_t(1) << 22;
  if (d.pair_cap > (int64_t(1) << 30) - 1) d.pair_cap = (int64_t(1) << 30) - 1;
  d.tile_cap = (int64_t)((p->max_width + 7) / 8) * ((p->max_height + 7) / 8);
  d.ntri = (int64_t)s->face_page.size();
  d.nvert = (int64_t)s->verts.size() / 3;
  d.nlink = (int64_t)s->link_col.size();
  d.scan_blocks = (d.ncap * d.nviews + kScanItems - 1) / kScanItems;
  d.lookback_words = (int64_t)kMaxPasses * ((d.pair_cap + kSortTile - 1) / kSortTile) * 256;
  d.ncl_cap = (d.ntri + 31) / 32 + d.NP + 1;
  d.piece_cap = d.pair_cap / 28 + 1;
  d.raster_cap = 2 * (d.ntri < (int64_t(1) << 20) ? (d.ntri > 0 ? d.ntri : 1) : (int64_t(1) << 20));
  d.ukey_cap = (int)pow2_at_least(d.NP > 0 ? d.NP : 1);
  d.free_cap = (int)pow2_at_least(P > 0 ? P : 1);
  d.cb_floats = p->fp16_pool == kFmtVQ ? (int64_t)s->n_codes * kCodeRow : 0;
  return d;
}

Layout make_layout(const Dims &d) {
  Layout L{};
  int64_t o = 0;
  auto take = [&](int64_t bytes) {
    int64_t r = o;
    o = al(o + (bytes > 0 ? bytes : 1));
    return r;
  };
  const int64_t NP = d.NP, P = d.P, N = d.ncap * d.nviews;
  L.ctl = take(sizeof(Ctl));
  L.fb = take(8 * d.fb_pixels);
  L.req = take(2 * 4 * NP);   // two buffers
  L.direct = take(2 * NP);
  L.reqlev = take(4 * NP);
  L.matched = take(NP);
  L.draw_info = take(4 * NP);
  L.requests = take(16 * NP);
  L.ukeys = take(8 * (int64_t)d.ukey_cap);
  L.free_keys = take(8 * (int64_t)d.free_cap);
  L.open_list = take(4 * (P + kMaxLevels));
  L.open_off = take(4 * (P + kMaxLevels));
  L.admitted_pos = take(4 * NP);
  L.copies = take(16 * NP);
  L.copy_seg = take(8 * (NP + 1));
  // (a page may be drawn at two levels during an LOD cross-fade)
  L.draw = take(16 * 2 * NP);
  L.draw_off = take(8 * (2 * NP + 1));
  L.draw_w = take(4 * 2 * NP);
  L.fade_state = take(4 * NP);
  L.fade_frame = take(4 * NP);
  L.fade_lev = take(4 * NP);
  L.fade_info = take(4 * NP);
  L.missing = take(4 * NP);
  L.pt_lod = take(4 * P);
  L.pt_last = take(4 * P);
  L.pt_slot = take(4 * P * d.Smax);
  L.required = take(P * d.Smax);
  L.any_req = take(P);
  L.tri_v = take(48 * d.ntri);
  L.clusters = take((int64_t)sizeof(Cluster) * d.ncl_cap);
  L.link_ptr = take(8 * (NP + 1));
  L.link_col = take(4 * d.nlink);
  L.err = take(4 * NP * kMaxLevels);
  L.raster_queue = take(kRasterRecord * d.raster_cap);
  L.raster_count = take(32);
  L.raster_vis = take(4 * d.ntri);
  L.raster_clip = take(4 * d.ntri);
  L.raster_bands = take(8 * d.raster_cap);
  L.raster_live = take(4 * d.ncl_cap);
  L.dreq = take(4 * NP);
  L.centroid = take(16 * NP);
  L.pf_flag = take(P * d.Smax);
  L.pf_mask = take((NP + 3) / 4 * 4);
  L.pf_cand = take(8 * (int64_t)d.ukey_cap);
  L.pf_copies = take(16 * NP);
  L.pf_copy_seg = take(8 * (NP + 1));
  L.pf_count = take(16);
  L.pf_base = take(16);
  L.pf_req = take(4 * NP);
  L.views = take(sizeof(ViewTable));
  L.codebook = take(4 * d.cb_floats);
  for (int k = 0; k < kContexts; ++k) {
    CtxLayout &C = L.cx[k];
    C.ctl = take(sizeof(Ctl));
    C.splat_rec = take(48 * N);
    C.splat_depth = take(4 * N);
    C.splat_rect = take(8 * N);
    C.splat_touched = take(4 * N);
    C.splat_radius = take(4 * N);
    C.splat_tmask = take(8 * N);
    C.block_sums = take(8 * d.scan_blocks);
    C.offsets = take(4 * N);
    C.keys0 = take(8 * d.pair_cap);
    C.keys1 = take(8 * d.pair_cap);
    C.vals0 = take(4 * d.pair_cap);
    C.vals1 = take(4 * d.pair_cap);
    C.ranges = take(8 * d.tile_cap * d.nviews);
    C.work = take(16);
    C.tile_order = take(4 * d.tile_cap * d.nviews);
    C.hist = take(4 * kMaxPasses * 256);
    C.lookback = take(4 * d.lookback_words);
    C.tile_ctr = take(4 * kMaxPasses);
    C.pieces = take(8 * d.piece_cap);
    C.piece_ctr = take(16);
  }
  L.total = o;
  return L;
}

Splats splats_of(const vm3dgs_renderer *r, int k) {
  const CtxLayout &C = r->lay.cx[k];
  Splats s;
  s.rec = r->at<float4>(C.splat_rec);
  s.depth = r->at<uint32_t>(C.splat_depth);
  s.rect = r->at<uint32_t>(C.splat_rect);
  s.touched = r->at<uint32_t>(C.splat_touched);
  s.radius = r->at<float>(C.splat_radius);
  s.tmask = r->at<uint64_t>(C.splat_tmask);
  return s;
}

}  // namespace vm

using namespace vm;

extern "C" int vm3dgs_pool_slot_bytes(const vm3dgs_scene *s, int32_t fp16_pool, int64_t *out) {
  if (!s || !out) return fail(VM3DGS_E_INVAL, "null argument");
  if (fp16_pool < kFmt32 || fp16_pool > kFmtVQ) return fail(VM3DGS_E_INVAL, "pool format must be 0, 1 or 2");
  if (fp16_pool == kFmt16 && !s->rec16) return fail(VM3DGS_E_STATE, "scene built without fp16 records");
  if (fp16_pool == kFmtVQ && !s->data_vq) return fail(VM3DGS_E_STATE, "scene has no VQ records (vm3dgs_scene_quantize_sh)");
  *out = (int64_t)s->page_size * s->fmt_rec(fp16_pool);
  return VM3DGS_OK;
}

extern "C" int vm3dgs_scratch_bytes(const vm3dgs_scene *s, const vm3dgs_params *p, int64_t pool_bytes, int64_t *out) {
  if (!s || !p || !out) return fail(VM3DGS_E_INVAL, "null argument");
  int64_t slot;
  int rc = vm3dgs_pool_slot_bytes(s, p->fp16_pool, &slot);
  if (rc) return rc;
  const int64_t P = pool_bytes / slot;
  Dims d = make_dims(s, p, P);
  *out = make_layout(d).total;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_renderer_create(const vm3dgs_scene *s, const vm3dgs_params *p, void *pool_dev,
                                      int64_t pool_bytes, void *scratch_dev, int64_t scratch_bytes, void *stream,
                                      vm3dgs_renderer **out) {
  if (!s || !p || !out || !pool_dev || !scratch_dev) return fail(VM3DGS_E_INVAL, "null argument");
  *out = nullptr;
  if (p->feedback_ds < 1 || p->max_width < 1 || p->max_height < 1 || p->staging_bytes < 0 ||
      !(p->usage_lo >= 0) || !(p->usage_hi >= p->usage_lo) || !(p->tau0 >= 0) || !(p->step0 > 0))
    return fail(VM3DGS_E_INVAL, "bad renderer parameters");
  if (p->lod_fade_frames < 0 || p->lod_fade_frames > 255)
    return fail(VM3DGS_E_INVAL, "lod_fade_frames must be 0..255");
  if ((p->max_height + p->feedback_ds - 1) / p->feedback_ds > 16000)
    return fail(VM3DGS_E_INVAL, "feedback buffer taller than 16000 rows (max_height / feedback_ds)");
  if (s->m(s->levels - 1) % 4 != 0) return fail(VM3DGS_E_INVAL, "smallest level page must hold a multiple of 4");
  int64_t slot;
  int rc = vm3dgs_pool_slot_bytes(s, p->fp16_pool, &slot);
  if (rc) return rc;
  const int64_t P = pool_bytes / slot;
  if (P < 1) return fail(VM3DGS_E_CAPACITY, "pool holds no page slot (" + std::to_string(slot) + " bytes each)");
  if (P * (int64_t)s->page_size >= (int64_t(1) << 31) / 1) return fail(VM3DGS_E_CAPACITY, "pool too large");
  Dims d = make_dims(s, p, P);
  Layout L = make_layout(d);
  if (scratch_bytes < L.total)
    return fail(VM3DGS_E_CAPACITY, "scratch needs " + std::to_string(L.total) + " bytes");
  auto *r = new (std::nothrow) vm3dgs_renderer();
  if (!r) return fail(VM3DGS_E_NOMEM, "renderer");
  r->scene = s;
  r->prm = *p;
  r->pool = (uint8_t *)pool_dev;
  r->pool_bytes = pool_bytes;
  r->slot_bytes = slot;
  r->P = (int32_t)P;
  r->fmt = p->fp16_pool;
  r->rec = s->fmt_rec(r->fmt);
  r->scratch = (uint8_t *)scratch_dev;
  r->dims = d;
  r->lay = L;
  cudaStream_t st = (cudaStream_t)stream;
  // page-lock the pages the GPU will pull, once per scene; a scene mapped
  // from a file is read by the host into a page-locked staging buffer instead
  auto *ms = const_cast<vm3dgs_scene *>(s);
  uint8_t *data = ms->fmt_data(r->fmt);
  const int64_t bytes = ms->fmt_bytes(r->fmt);
  bool &reg = ms->fmt_registered(r->fmt);
  if (ms->mapped && r->fmt != kFmtVQ) {
    r->staged = true;
    const size_t sbytes = (size_t)((p->staging_bytes + 4095) / 4096 * 4096);
    if (!cuda_ok(cudaHostAlloc((void **)&r->staging, sbytes > 0 ? sbytes : 4096, cudaHostAllocMapped), "cudaHostAlloc",
                 &rc) ||
        !cuda_ok(cudaHostAlloc((void **)&r->h_copies, 16 * (size_t)d.NP + 16, cudaHostAllocDefault), "cudaHostAlloc",
                 &rc) ||
        !cuda_ok(cudaHostAlloc((void **)&r->h_off, 8 * (size_t)(d.NP + 1), cudaHostAllocMapped), "cudaHostAlloc",
                 &rc) ||
        !cuda_ok(cudaHostGetDevicePointer((void **)&r->h_off_dev, r->h_off, 0), "cudaHostGetDevicePointer", &rc) ||
        !cuda_ok(cudaHostAlloc((void **)&r->h_count, 64, cudaHostAllocDefault), "cudaHostAlloc", &rc)) {
      vm3dgs_renderer_destroy(r);
      return rc;
    }
    data = r->staging;
  } else if (!reg) {
    if (!cuda_ok(cudaHostRegister(data, (size_t)((bytes + 4095) / 4096 * 4096),
                                  cudaHostRegisterMapped | cudaHostRegisterPortable),
                 "cudaHostRegister", &rc)) {
      delete r;
      return rc;
    }
    reg = true;
  }
  void *dp = nullptr;
  if (!cuda_ok(cudaHostGetDevicePointer(&dp, data, 0), "cudaHostGetDevicePointer", &rc)) { delete r; return rc; }
  r->host_dev = (const uint8_t *)dp;
  // static scene arrays
  bool ok = true;
  {
    // proxy triangles regrouped by page, de-indexed, in clusters for the frustum test
    std::vector<float> tv((size_t)(12 * d.ntri));
    std::vector<Cluster> cl((size_t)d.ncl_cap);
    r->ncl = build_clusters(s->verts.data(), s->tris.data(), s->face_page.data(), d.ntri, d.NP, tv.data(), cl.data());
    ok = ok && cuda_ok(cudaMemcpy(r->at<void>(L.tri_v), tv.data(), 4 * tv.size(), cudaMemcpyHostToDevice), "copy", &rc);
    ok = ok && cuda_ok(cudaMemcpy(r->at<void>(L.clusters), cl.data(), sizeof(Cluster) * (size_t)r->ncl,
                                  cudaMemcpyHostToDevice), "copy", &rc);
  }
  r->maps_ok = encode_proj_maps(s, r->pool, P, r->fmt, &r->maps);
  if (r->fmt == kFmtVQ) {
    // device rows of kCodeRow floats: channel c's bands-1..3 coefficients
    // at [16 c, 16 c + K - 1) (zero padded), for aligned 16-byte loads
    std::vector<float> rows((size_t)s->n_codes * kCodeRow, 0.0f);
    for (int j = 0; j < s->n_codes; ++j)
      for (int k = 1; k < s->K; ++k)
        for (int c = 0; c < 3; ++c)
          rows[(size_t)j * kCodeRow + 16 * c + (k - 1)] = s->codebook[(size_t)j * s->code_dim + 3 * (k - 1) + c];
    ok = ok && cuda_ok(cudaMemcpy(r->at<void>(L.codebook), rows.data(), 4 * rows.size(), cudaMemcpyHostToDevice),
                       "copy", &rc);
  }
  r->rec_maps_ok = true;
  for (int k = 0; k < kContexts; ++k)
    r->rec_maps_ok = r->rec_maps_ok && encode_rec_map(r->at<float4>(L.cx[k].splat_rec), d.ncap, &r->rec_map[k]);
  // a box around every page's sphere (centroid, radius), hence around every
  // Gaussian mean of every level: it bounds the depth of any splat
  for (int a = 0; a < 3; ++a) { r->gbox_lo[a] = 0.0; r->gbox_hi[a] = 0.0; }
  for (int64_t p2 = 0; p2 < d.NP; ++p2)
    for (int a = 0; a < 3; ++a) {
      const double c = s->centroid[4 * p2 + a], rad = s->centroid[4 * p2 + 3];
      if (p2 == 0 || c - rad < r->gbox_lo[a]) r->gbox_lo[a] = c - rad;
      if (p2 == 0 || c + rad > r->gbox_hi[a]) r->gbox_hi[a] = c + rad;
    }
  ok = ok && cuda_ok(cudaMemcpyAsync(r->at<void>(L.link_ptr), s->link_ptr.data(), 8 * s->link_ptr.size(), cudaMemcpyHostToDevice, st), "copy", &rc);
  if (!s->link_col.empty())
    ok = ok && cuda_ok(cudaMemcpyAsync(r->at<void>(L.link_col), s->link_col.data(), 4 * s->link_col.size(), cudaMemcpyHostToDevice, st), "copy", &rc);
  ok = ok && cuda_ok(cudaMemcpyAsync(r->at<void>(L.err), s->err.data(), 4 * s->err.size(), cudaMemcpyHostToDevice, st), "copy", &rc);
  ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.pt_lod), 0xFF, 4 * P, st), "memset", &rc);
  ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.pt_last), 0xFF, 4 * P, st), "memset", &rc);
  ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.pt_slot), 0xFF, 4 * P * d.Smax, st), "memset", &rc);
  ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.pf_flag), 0, P * d.Smax, st), "memset", &rc);
  ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.fade_state), 0, 4 * d.NP, st), "memset", &rc);
  // (a stamp no frame number - 1 can equal)
  ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.fade_frame), 0x80, 4 * d.NP, st), "memset", &rc);
  ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.pf_count), 0, 16, st), "memset", &rc);
  ok = ok && cuda_ok(cudaMemcpyAsync(r->at<void>(L.centroid), s->centroid.data(), 4 * s->centroid.size(),
                                     cudaMemcpyHostToDevice, st), "copy", &rc);
  for (int k = 0; k < 3; ++k) r->scene_center[k] = s->box_center[k];
  r->scene_half = s->box_half;
  Ctl c{};
  c.tau = p->tau0;
  c.step = p->step0;
  c.last_move = -1000;
  ok = ok && cuda_ok(cudaMemcpyAsync(r->at<void>(L.ctl), &c, sizeof(Ctl), cudaMemcpyHostToDevice, st), "copy", &rc);
  for (int k = 0; k < kContexts; ++k) {
    ok = ok && cuda_ok(cudaMemsetAsync(r->at<void>(L.cx[k].ctl), 0, sizeof(Ctl), st), "memset", &rc);
    ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->ctx_free[k], cudaEventDisableTiming), "event", &rc);
  }
  ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->copy_done, cudaEventDisableTiming), "event", &rc);
  ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->res_done, cudaEventDisableTiming), "event", &rc);
  ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->pf_done, cudaEventDisableTiming), "event", &rc);
  ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->pf_req_done, cudaEventDisableTiming), "event", &rc);
  for (auto &e : r->res_done_buf) ok = ok && cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event", &rc);
  ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->fb_done, cudaEventDisableTiming), "event", &rc);
  ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->upd_done, cudaEventDisableTiming), "event", &rc);
  ok = ok && cuda_ok(cudaEventCreateWithFlags(&r->proj_done, cudaEventDisableTiming), "event", &rc);
  ok = ok && cuda_ok(cudaStreamSynchronize(st), "sync", &rc);
  if (!ok) { delete r; return rc; }
  *out = r;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_timing_enable(vm3dgs_renderer *r, int32_t on) {
  if (!r) return fail(VM3DGS_E_INVAL, "null renderer");
  r->timing = on != 0;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_timing_read(vm3dgs_renderer *r, double *ms_total, int64_t *launches, int32_t n) {
  if (!r || !ms_total || !launches || n < 0) return fail(VM3DGS_E_INVAL, "null argument");
  int rc = 0;
  if (!cuda_ok(cudaDeviceSynchronize(), "timing sync", &rc)) return rc;
  for (auto &t : r->spans) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) ms = 0.0f;
    if (t.stage < n) {
      ms_total[t.stage] += ms;
      launches[t.stage] += t.launches;
    }
    r->spare_events.push_back(t.a);
    r->spare_events.push_back(t.b);
  }
  r->spans.clear();
  cudaGetLastError();
  return VM3DGS_OK;
}

extern "C" void vm3dgs_renderer_destroy(vm3dgs_renderer *r) {
  if (!r) return;
  cudaDeviceSynchronize();
  for (auto &t : r->spans) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  for (auto e : r->spare_events) cudaEventDestroy(e);
  if (r->copy_done) cudaEventDestroy(r->copy_done);
  if (r->res_done) cudaEventDestroy(r->res_done);
  if (r->graph_exec) cudaGraphExecDestroy(r->graph_exec);
  if (r->graph) cudaGraphDestroy(r->graph);
  if (r->pf_done) cudaEventDestroy(r->pf_done);
  if (r->pf_req_done) cudaEventDestroy(r->pf_req_done);
  for (auto e : r->res_done_buf)
    if (e) cudaEventDestroy(e);
  if (r->fb_done) cudaEventDestroy(r->fb_done);
  if (r->upd_done) cudaEventDestroy(r->upd_done);
  if (r->proj_done) cudaEventDestroy(r->proj_done);
  for (auto e : r->ctx_free)
    if (e) cudaEventDestroy(e);
  if (r->staging) cudaFreeHost(r->staging);
  if (r->h_copies) cudaFreeHost(r->h_copies);
  if (r->h_off) cudaFreeHost(r->h_off);
  if (r->h_count) cudaFreeHost(r->h_count);
  delete r;
}

extern "C" int vm3dgs_render_feedback(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams, void *stream) {
  if (!r) return fail(VM3DGS_E_INVAL, "null renderer");
  int rc = check_cams(r, cams, n_cams);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t NP = r->dims.NP;
  const int kb = r->fb_buf ^ 1;  // the request buffer this page determination writes
  if (r->pf_req_pending && r->pf_req_buf == kb) {  // a prefetch still copies these request words
    cudaStreamWaitEvent(st, r->pf_req_done, 0);
    r->pf_req_pending = false;
  }
  // the update that read this buffer (two page determinations ago) is done;
  // the visibility buffer and raster scratch are free
  if (r->res_recorded_buf[kb]) cudaStreamWaitEvent(st, r->res_done_buf[kb], 0);
  if (r->fb_recorded) cudaStreamWaitEvent(st, r->fb_done, 0);
  uint32_t *req = r->req_buf(kb);
  uint8_t *direct = r->direct_buf(kb);
  // with links the pixels' codes gather per page first, then spread
  uint32_t *dreq = r->prm.links ? r->at<uint32_t>(r->lay.dreq) : req;
  const int ds = r->prm.feedback_ds;
  float fpx = 0.0f;
  const int sp_fb = r->span_begin(VM3DGS_STAGE_FEEDBACK, st);
  for (int v = 0; v < n_cams; ++v) {
    const vm3dgs_camera &c = cams[v];
    const int64_t npix = (int64_t)((c.width + ds - 1) / ds) * ((c.height + ds - 1) / ds);
    uint64_t *fb = r->at<uint64_t>(r->lay.fb);
    launch_feedback_clear(fb, npix, r->at<uint32_t>(r->lay.raster_count), v == 0 ? req : nullptr, direct,
                          r->prm.links ? dreq : nullptr, NP, st);
    launch_feedback_raster(r->at<float4>(r->lay.tri_v), r->at<Cluster>(r->lay.clusters), r->ncl, r->dims.ntri, c, ds, fb,
                           r->at<void>(r->lay.raster_queue),
                           r->at<uint32_t>(r->lay.raster_count), (uint32_t)r->dims.raster_cap,
                           r->at<uint64_t>(r->lay.raster_bands), (uint32_t)r->dims.raster_cap,
                           r->at<uint32_t>(r->lay.raster_vis), r->at<uint32_t>(r->lay.raster_clip),
                           r->at<uint32_t>(r->lay.raster_live), st);
    launch_feedback_reduce(fb, npix, dreq, direct, st);
    r->last_fb_pixels = npix;
    if (c.fy > fpx) fpx = c.fy;
  }
  if (r->prm.links)
    launch_feedback_links(dreq, NP, r->at<int64_t>(r->lay.link_ptr), r->at<int32_t>(r->lay.link_col), req, st);
  r->span_end(sp_fb, 8 * n_cams + (r->prm.links ? 1 : 0), st);  // kernels: clear, cluster and triangle cull, setup, clip, medium, huge, reduce; links
  cudaEventRecord(r->fb_done, st);
  r->fb_recorded = true;
  r->fb_buf = kb;
  r->f_px = fpx;
  r->state = 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VM3DGS_E_CUDA, std::string("feedback: ") + cudaGetErrorString(e));
  return VM3DGS_OK;
}

extern "C" int vm3dgs_request_all(vm3dgs_renderer *r, void *stream) {
  if (!r) return fail(VM3DGS_E_INVAL, "null renderer");
  cudaStream_t st = (cudaStream_t)stream;
  const int kb = r->fb_buf ^ 1;
  if (r->pf_req_pending && r->pf_req_buf == kb) {
    cudaStreamWaitEvent(st, r->pf_req_done, 0);
    r->pf_req_pending = false;
  }
  if (r->res_recorded_buf[kb]) cudaStreamWaitEvent(st, r->res_done_buf[kb], 0);
  if (r->fb_recorded) cudaStreamWaitEvent(st, r->fb_done, 0);
  launch_request_all(r->req_buf(kb), r->direct_buf(kb), r->dims.NP, st);
  cudaEventRecord(r->fb_done, st);
  r->fb_recorded = true;
  r->fb_buf = kb;
  r->f_px = 1.0f;
  r->state = 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VM3DGS_E_CUDA, std::string("request_all: ") + cudaGetErrorString(e));
  return VM3DGS_OK;
}

namespace {
// Host function of a file-backed update: staging offsets of the copy list
// just read back, then the pages from the scene mapping into the staging
// buffer (host threads).  Makes no CUDA call.
void CUDART_CB gather_staged(void *user) {
  auto *r = static_cast<vm3dgs_renderer *>(user);
  const vm3dgs_scene *s = r->scene;
  const int n = std::min(std::max(*r->h_count, 0), (int)r->dims.NP);
  int64_t cum = 0;
  for (int i = 0; i < n; ++i) {
    r->h_off[i] = cum;
    cum += (int64_t)s->m(r->h_copies[i].y) * r->rec;
  }
  r->h_off[n] = cum;
  if (cum > r->prm.staging_bytes) {  // cannot happen: admission keeps the copies within the budget;
    r->staged_err = 1;               // every copy then reads the buffer's start (each page fits in it)
    for (int i = 0; i <= n; ++i) r->h_off[i] = 0;
    return;
  }
  const uint8_t *base = s->fmt_data(r->fmt);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) {
    const int4 c = r->h_copies[i];
    const int64_t pb = (int64_t)s->m(c.y) * r->rec;
    const int64_t lo = s->fmt_off(r->fmt)[c.y];
    std::memcpy(r->staging + r->h_off[i], base + lo + (int64_t)c.x * pb, (size_t)pb);
  }
}
}  // namespace

extern "C" int vm3dgs_update_residency(vm3dgs_renderer *r, void *stream, void *copy_stream) {
  if (!r) return fail(VM3DGS_E_INVAL, "null renderer");
  if (r->state < 1) return fail(VM3DGS_E_STATE, "update_residency before render_feedback");
  cudaStream_t st = (cudaStream_t)stream, cst = copy_stream ? (cudaStream_t)copy_stream : st;
  if (r->pf_pending) {
    cudaStreamWaitEvent(st, r->pf_done, 0);
    r->pf_pending = false;
  }
  if (r->copy_pending) {  // the copy list is rewritten below: earlier copies must be done reading it
    cudaStreamWaitEvent(st, r->copy_done, 0);
    r->copy_pending = false;
  }
  if (r->fb_recorded) cudaStreamWaitEvent(st, r->fb_done, 0);  // page determination on another stream
  // a file-backed update reuses the read-back and staging buffers of the last one
  if (r->staged && r->upd_recorded) cudaStreamWaitEvent(st, r->upd_done, 0);
  // the last render's projection has read the pool and the draw list
  if (r->proj_recorded) cudaStreamWaitEvent(st, r->proj_done, 0);
  const vm3dgs_scene *s = r->scene;
  ResidencyArgs a{};
  a.ctl = r->at<Ctl>(r->lay.ctl);
  a.req = r->req_buf(r->fb_buf);
  a.direct = r->direct_buf(r->fb_buf);
  a.reqlev = r->at<int32_t>(r->lay.reqlev);
  a.draw_info = r->at<int32_t>(r->lay.draw_info);
  a.matched = r->at<uint8_t>(r->lay.matched);
  a.requests = r->at<int4>(r->lay.requests);
  a.ukeys = r->at<uint64_t>(r->lay.ukeys);
  a.free_keys = r->at<uint64_t>(r->lay.free_keys);
  a.open_list = r->at<int32_t>(r->lay.open_list);
  a.open_off = r->at<int32_t>(r->lay.open_off);
  a.admitted_pos = r->at<int32_t>(r->lay.admitted_pos);
  a.copies = r->at<int4>(r->lay.copies);
  a.copy_seg = r->at<int64_t>(r->lay.copy_seg);
  a.draw = r->at<int4>(r->lay.draw);
  a.draw_off = r->at<int64_t>(r->lay.draw_off);
  a.draw_w = r->at<float>(r->lay.draw_w);
  a.fade_state = r->at<int32_t>(r->lay.fade_state);
  a.fade_frame = r->at<int32_t>(r->lay.fade_frame);
  a.fade_lev = r->at<int32_t>(r->lay.fade_lev);
  a.fade_info = r->at<int32_t>(r->lay.fade_info);
  a.fade_frames = r->prm.lod_fade_frames;
  a.missing = r->at<int32_t>(r->lay.missing);
  a.pt_lod = r->at<int32_t>(r->lay.pt_lod);
  a.pt_last = r->at<int32_t>(r->lay.pt_last);
  a.pt_slot = r->at<int32_t>(r->lay.pt_slot);
  a.required = r->at<uint8_t>(r->lay.required);
  a.any_req = r->at<uint8_t>(r->lay.any_req);
  a.pf_flag = r->at<uint8_t>(r->lay.pf_flag);
  a.err = r->at<float>(r->lay.err);
  a.NP = (int32_t)r->dims.NP;
  a.P = r->P;
  a.Smax = (int32_t)r->dims.Smax;
  a.levels = s->levels;
  a.fanout = s->fanout;
  a.page_size = s->page_size;
  a.lod_on = r->prm.lod;
  a.budget = r->prm.staging_bytes;
  a.rec = r->rec;
  a.f_px = r->f_px;
  a.usage_lo = r->prm.usage_lo;
  a.usage_hi = r->prm.usage_hi;
  a.ukey_cap = r->dims.ukey_cap;
  a.free_cap = r->dims.free_cap;
  const int sp_res = r->span_begin(VM3DGS_STAGE_RESIDENCY, st);
  launch_residency(a, st);
  r->span_end(sp_res, 1, st);
  cudaEventRecord(r->res_done, st);
  r->res_recorded = true;
  cudaEventRecord(r->res_done_buf[r->fb_buf], st);
  r->res_recorded_buf[r->fb_buf] = true;
  r->res_buf = r->fb_buf;
  StreamArgs sa{};
  sa.count = &a.ctl->n_copies;
  sa.copies = a.copies;
  sa.copy_seg = a.copy_seg;
  sa.host = r->host_dev;
  for (int l = 0; l < s->levels; ++l) sa.level_off[l] = s->fmt_off(r->fmt)[l];
  sa.page_size = s->page_size;
  sa.fanout = s->fanout;
  sa.rec = r->rec;
  sa.pool = r->pool;
  sa.slot_bytes = r->slot_bytes;
  if (r->staged) {
    // the paper's transfer: the copy list returns to the host, which copies
    // the pages from the file mapping (the OS reads what is not cached) into
    // the staging buffer, then the GPU streams them.  The host gather is a
    // host function in stream order (between the list's read-back and the
    // stream kernel), so the calling thread does not wait; the next update's
    // gather follows this update's copies on the same stream.
    if (r->staged_err) {
      r->staged_err = 0;
      return fail(VM3DGS_E_CAPACITY, "an earlier update's copies exceeded the staging buffer");
    }
    int rc = VM3DGS_OK;
    const int NPc = (int)r->dims.NP;
    const bool ok =
        cuda_ok(cudaMemcpyAsync(r->h_count, &a.ctl->n_copies, 4, cudaMemcpyDeviceToHost, st), "copy", &rc) &&
        cuda_ok(cudaMemcpyAsync(r->h_copies, a.copies, 16 * (size_t)NPc, cudaMemcpyDeviceToHost, st), "copy", &rc) &&
        cuda_ok(cudaLaunchHostFunc(st, gather_staged, r), "cudaLaunchHostFunc", &rc);
    if (!ok) return rc;
    sa.staged_off = r->h_off_dev;
    cst = st;
  }
  if (cst == st) {
    const int sp = r->span_begin(VM3DGS_STAGE_STREAM, st);
    launch_stream(sa, st);
    r->span_end(sp, 1, st);
    r->copy_pending = false;
  } else {
    cudaEventRecord(r->copy_done, st);
    cudaStreamWaitEvent(cst, r->copy_done, 0);
    const int sp = r->span_begin(VM3DGS_STAGE_STREAM, cst);
    launch_stream(sa, cst);
    r->span_end(sp, 1, cst);
    cudaEventRecord(r->copy_done, cst);
    r->copy_pending = true;
  }
  cudaEventRecord(r->upd_done, st);
  r->upd_recorded = true;
  r->state = 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VM3DGS_E_CUDA, std::string("update_residency: ") + cudaGetErrorString(e));
  return VM3DGS_OK;
}

namespace {
int bit_length(uint64_t x) {
  int b = 0;
  while (x) { ++b; x >>= 1; }
  return b;
}

// Key layout for one view: the depth field spans bits(0.2f) .. bits(far),
// far bounding the view depth of every Gaussian mean (box corners, plus a
// margin above the rounding of the device's depth); splat indices are packed
// below it when tile, depth and index bits fit in 64.
KeyFormat key_format(const vm3dgs_renderer *r, const vm3dgs_camera &c, int tbits) {
  const float *V = c.view;
  double far = -1e300, mag = std::fabs((double)V[11]);
  for (int k = 0; k < 8; ++k) {
    double z = V[11];
    for (int a = 0; a < 3; ++a) z += (double)V[8 + a] * ((k >> a) & 1 ? r->gbox_hi[a] : r->gbox_lo[a]);
    far = std::max(far, z);
  }
  for (int a = 0; a < 3; ++a)
    mag += std::fabs((double)V[8 + a]) * std::max(std::fabs(r->gbox_lo[a]), std::fabs(r->gbox_hi[a]));
  far += 1e-3 * (1.0 + mag);
  KeyFormat kf{};
  uint32_t base_bits, far_bits;
  const float near = 0.2f;
  std::memcpy(&base_bits, &near, 4);
  const float farf = far > 3.0e38 ? 3.0e38f : (float)far;
  std::memcpy(&far_bits, &farf, 4);
  kf.base = base_bits;
  kf.R = farf > near ? std::max(1, bit_length((uint64_t)(far_bits - base_bits))) : 1;
  const int ib = bit_length((uint64_t)(r->dims.ncap > 1 ? r->dims.ncap - 1 : 1));
  kf.packed = !r->prm.separate_values && tbits + kf.R + ib <= 64;
  kf.ib = kf.packed ? ib : 0;
  kf.tshift = kf.R + kf.ib;
  return kf;
}
}  // namespace

extern "C" int vm3dgs_render(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams, float *const *images,
                             void *stream) {
  if (!r || !images) return fail(VM3DGS_E_INVAL, "null argument");
  if (r->state < 2) return fail(VM3DGS_E_STATE, "render before update_residency");
  int rc = check_cams(r, cams, n_cams);
  if (rc) return rc;
  if (n_cams > (r->prm.max_views > 0 ? r->prm.max_views : 1)) return fail(VM3DGS_E_INVAL, "more views than max_views");
  cudaStream_t st = (cudaStream_t)stream;
  if (r->copy_pending) {
    cudaStreamWaitEvent(st, r->copy_done, 0);
    r->copy_pending = false;
  }
  if (r->upd_recorded) cudaStreamWaitEvent(st, r->upd_done, 0);  // page-table update on another stream
  // render contexts alternate: this one's last render must be done with it
  const int k = r->ctx;
  if (r->ctx_recorded[k]) cudaStreamWaitEvent(st, r->ctx_free[k], 0);
  const CtxLayout &C = r->lay.cx[k];
  const vm3dgs_scene *s = r->scene;
  Ctl *ctl = r->at<Ctl>(C.ctl);  // the scan, sort and ranges count with the context's control block
  Splats sp = splats_of(r, k);
  ProjectArgs pa{};
  pa.ctl = r->at<Ctl>(r->lay.ctl);
  pa.rctl = ctl;
  pa.draw = r->at<int4>(r->lay.draw);
  pa.draw_off = r->at<int64_t>(r->lay.draw_off);
  pa.draw_w = r->prm.lod_fade_frames > 0 ? r->at<float>(r->lay.draw_w) : nullptr;
  pa.pool = r->pool;
  pa.slot_bytes = r->slot_bytes;
  pa.page_size = s->page_size;
  pa.fanout = s->fanout;
  pa.K = s->K;
  pa.fmt = r->fmt;
  pa.codebook = r->fmt == kFmtVQ ? r->at<float>(r->lay.codebook) : nullptr;
  pa.ncap = r->dims.ncap;
  pa.sp = sp;
  pa.maps = r->maps_ok ? &r->maps : nullptr;
  uint64_t *keys[2] = {r->at<uint64_t>(C.keys0), r->at<uint64_t>(C.keys1)};
  uint32_t *vals[2] = {r->at<uint32_t>(C.vals0), r->at<uint32_t>(C.vals1)};
  for (int v = 0; v < n_cams; ++v) {
    const vm3dgs_camera &c = cams[v];
    if (!images[v]) return fail(VM3DGS_E_INVAL, "null image");
    const int gx = (c.width + c.tile_w - 1) / c.tile_w, gy = (c.height + c.tile_h - 1) / c.tile_h;
    const int ntiles = gx * gy;
    if (ntiles > r->dims.tile_cap) return fail(VM3DGS_E_CAPACITY, "too many tiles");
    int tbits = 0;
    while ((1 << tbits) < ntiles) ++tbits;
    int t = r->span_begin(VM3DGS_STAGE_PROJECT, st);
    launch_project(pa, c, st);
    r->span_end(t, 1, st);
    if (v == n_cams - 1) {  // the next page-table update may start
      cudaEventRecord(r->proj_done, st);
      r->proj_recorded = true;
    }
    t = r->span_begin(VM3DGS_STAGE_SCAN_EMIT, st);
    const KeyFormat kf = key_format(r, c, tbits);
    const int lo_bit = kf.ib, hi_bit = kf.tshift + tbits;
    const int passes = (hi_bit - lo_bit + 7) / 8;
    const int64_t max_tiles = (r->dims.pair_cap + kSortTile - 1) / kSortTile;
    if (passes < 1 || passes > kMaxPasses || (int64_t)passes * max_tiles * 256 > r->dims.lookback_words)
      return fail(VM3DGS_E_CAPACITY, "sort look-back area too small");
    // the cooperative sort needs no look-back words (the emission clears them otherwise)
    const bool coop = r->prm.sort_mode == 1 && coop_sort_grid() > 0;
    const SortHist sh{r->at<uint32_t>(C.hist), coop ? nullptr : r->at<uint32_t>(C.lookback), max_tiles,
                      r->at<uint32_t>(C.tile_ctr), lo_bit, passes};
    launch_scan_emit(ctl, ctl, sp, r->dims.ncap, r->at<uint32_t>(C.block_sums), r->at<uint32_t>(C.offsets),
                     keys[0], vals[0], r->dims.pair_cap, TileGeom{c.width, c.height, c.tile_w, c.tile_h}, gx, kf,
                     sh, r->at<uint64_t>(C.pieces),
                     r->at<uint32_t>(C.piece_ctr), r->dims.piece_cap, r->at<uint2>(C.ranges), ntiles, st);
    r->span_end(t, 5, st);  // scan reduce, scan blocks, scan offsets, emit, emit pieces
    uint32_t *no_vals[2] = {nullptr, nullptr};
    t = r->span_begin(VM3DGS_STAGE_SORT, st);
    const int cur = coop ? launch_sort_coop(ctl, keys, kf.packed ? no_vals : vals, r->dims.pair_cap, lo_bit, hi_bit,
                                            r->at<uint32_t>(C.hist), r->at<uint32_t>(C.lookback),
                                            r->dims.lookback_words, r->at<uint32_t>(C.tile_ctr), st)
                         : launch_sort_passes(ctl, keys, kf.packed ? no_vals : vals, r->dims.pair_cap, lo_bit, hi_bit,
                                              r->at<uint32_t>(C.hist), r->at<uint32_t>(C.lookback),
                                              r->at<uint32_t>(C.tile_ctr), st);
    r->span_end(t, coop ? 1 : passes, st);
    if (cur == -3) return fail(VM3DGS_E_CUDA, "cooperative sort launch refused");
    if (cur == -2) return fail(VM3DGS_E_CUDA, coop ? "cooperative sort scratch too small" : "sort shared-memory attribute refused");
    if (cur < 0) return fail(VM3DGS_E_CAPACITY, "sort look-back area too small");
    uint2 *ranges = r->at<uint2>(C.ranges);
    uint32_t *order = r->at<uint32_t>(C.tile_order), *work = r->at<uint32_t>(C.work);
    t = r->span_begin(VM3DGS_STAGE_RANGES, st);
    launch_ranges(ctl, keys[cur], r->dims.pair_cap, ranges, ntiles, kf.tshift, st, true);
    launch_tile_order(ranges, ntiles, order, work, st);
    r->span_end(t, 2, st);
    t = r->span_begin(VM3DGS_STAGE_BLEND, st);
    const uint32_t idx_mask = kf.ib >= 32 ? 0xFFFFFFFFu : (uint32_t)((1ull << kf.ib) - 1ull);
    launch_blend(ranges, vals[cur], kf.packed ? keys[cur] : nullptr, idx_mask, sp, r->dims.ncap, c, r->prm.bg,
                 images[v], order, work + 1, r->rec_maps_ok ? &r->rec_map[k] : nullptr, ctl, st);
    r->span_end(t, 1, st);
    r->kf = kf;
    r->sorted_buf = cur;
    r->last_ntiles = ntiles;
  }
  cudaEventRecord(r->ctx_free[k], st);
  r->ctx_recorded[k] = true;
  r->last_ctx = k;
  r->ctx = (k + 1) % kContexts;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VM3DGS_E_CUDA, std::string("render: ") + cudaGetErrorString(e));
  return VM3DGS_OK;
}

namespace {
// orders stream after every outstanding page determination, update and render
void wait_all(vm3dgs_renderer *r, cudaStream_t st) {
  if (r->fb_recorded) cudaStreamWaitEvent(st, r->fb_done, 0);
  if (r->upd_recorded) cudaStreamWaitEvent(st, r->upd_done, 0);
  for (int k = 0; k < kContexts; ++k)
    if (r->ctx_recorded[k]) cudaStreamWaitEvent(st, r->ctx_free[k], 0);
}
}  // namespace

extern "C" int vm3dgs_get_stats(vm3dgs_renderer *r, vm3dgs_stats *out, void *stream) {
  if (!r || !out) return fail(VM3DGS_E_INVAL, "null argument");
  Ctl c, cx[kContexts];
  int rc = 0;
  cudaStream_t st = (cudaStream_t)stream;
  wait_all(r, st);
  if (!cuda_ok(cudaMemcpyAsync(&c, r->at<void>(r->lay.ctl), sizeof(Ctl), cudaMemcpyDeviceToHost, st), "stats", &rc))
    return rc;
  for (int k = 0; k < kContexts; ++k)
    if (!cuda_ok(cudaMemcpyAsync(&cx[k], r->at<void>(r->lay.cx[k].ctl), sizeof(Ctl), cudaMemcpyDeviceToHost, st),
                 "stats", &rc))
      return rc;
  if (!cuda_ok(cudaStreamSynchronize(st), "stats sync", &rc)) return rc;
  // the render contexts hold the pair counts and their sums; statuses from any block
  const Ctl &last = cx[r->last_ctx];
  c.pairs = last.pairs;
  for (int k = 0; k < kContexts; ++k) {
    c.acc_pairs += cx[k].acc_pairs;
    c.acc_views += cx[k].acc_views;
    if (c.status == 0) c.status = cx[k].status;
  }
  std::memset(out, 0, sizeof(*out));
  out->frame = c.frame;
  out->requested = c.n_req;
  out->direct = c.n_direct;
  out->resident = c.n_resident;
  out->missing = c.n_missing;
  out->fading = c.n_fading;
  out->streamed_pages = c.n_copies;
  out->streamed_bytes = c.streamed_bytes;
  out->drawn_pages = c.n_draw;
  out->drawn_gaussians = c.draw_gauss;
  out->pairs = c.pairs;
  out->usage = c.usage;
  out->tau = c.tau;
  out->status = c.status;
  if (c.status == 0 && c.pairs > r->dims.pair_cap) out->status = VM3DGS_E_CAPACITY;
  out->acc_frames = c.acc_frames;
  out->acc_views = c.acc_views;
  out->acc_pairs = c.acc_pairs;
  out->acc_drawn_gaussians = c.acc_draw_gauss;
  out->acc_streamed_bytes = c.acc_streamed_bytes;
  out->acc_streamed_pages = c.acc_streamed_pages;
  out->acc_missing = c.acc_missing;
  out->acc_requested = c.acc_requested;
  out->acc_prefetched_pages = c.acc_prefetched_pages;
  out->acc_prefetched_bytes = c.acc_prefetched_bytes;
  out->acc_prefetch_hits = c.acc_prefetch_hits;
  out->staged_projection = r->maps_ok ? 1 : 0;
  int tbits = 0;
  while ((1 << tbits) < r->last_ntiles) ++tbits;
  out->key_tile_bits = tbits;
  out->key_depth_bits = r->kf.R;
  out->key_index_bits = r->kf.packed ? r->kf.ib : 0;
  out->key_packed = r->kf.packed ? 1 : 0;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_reset_sums(vm3dgs_renderer *r, void *stream) {
  if (!r) return fail(VM3DGS_E_INVAL, "null renderer");
  int rc = 0;
  const size_t off = offsetof(Ctl, acc_frames);
  cudaStream_t st = (cudaStream_t)stream;
  wait_all(r, st);
  if (!cuda_ok(cudaMemsetAsync(r->scratch + r->lay.ctl + off, 0, sizeof(Ctl) - off, st), "reset", &rc)) return rc;
  for (int k = 0; k < kContexts; ++k)
    if (!cuda_ok(cudaMemsetAsync(r->scratch + r->lay.cx[k].ctl + off, 0, sizeof(Ctl) - off, st), "reset", &rc))
      return rc;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_debug_read(vm3dgs_renderer *r, int32_t what, void *dst, int64_t bytes, int64_t *needed,
                                 void *stream) {
  if (!r) return fail(VM3DGS_E_INVAL, "null renderer");
  cudaStream_t st = (cudaStream_t)stream;
  wait_all(r, st);  // the buffers may be written on other streams
  Ctl c, cr;
  int rc = 0;
  const Layout &L = r->lay;
  const CtxLayout &C = L.cx[r->last_ctx];  // the last render's buffers
  if (!cuda_ok(cudaMemcpyAsync(&c, r->at<void>(L.ctl), sizeof(Ctl), cudaMemcpyDeviceToHost, st), "debug", &rc) ||
      !cuda_ok(cudaMemcpyAsync(&cr, r->at<void>(C.ctl), sizeof(Ctl), cudaMemcpyDeviceToHost, st), "debug", &rc))
    return rc;
  if (!cuda_ok(cudaStreamSynchronize(st), "debug sync", &rc)) return rc;
  const int64_t NP = r->dims.NP, P = r->P, N = cr.r_drawn < r->dims.ncap ? cr.r_drawn : r->dims.ncap;
  const int64_t M = cr.pairs < r->dims.pair_cap ? cr.pairs : r->dims.pair_cap;
  const void *src = nullptr;
  int64_t n = 0;
  switch (what) {
    case VM3DGS_DBG_FEEDBACK: src = r->at<void>(L.fb); n = 8 * r->last_fb_pixels; break;
    case VM3DGS_DBG_REQ: src = r->req_buf(r->fb_buf); n = 4 * NP; break;
    case VM3DGS_DBG_DIRECT: src = r->direct_buf(r->fb_buf); n = NP; break;
    case VM3DGS_DBG_REQUESTS: src = r->at<void>(L.requests); n = 16 * (int64_t)c.n_req; break;
    case VM3DGS_DBG_PT_LOD: src = r->at<void>(L.pt_lod); n = 4 * P; break;
    case VM3DGS_DBG_PT_LAST: src = r->at<void>(L.pt_last); n = 4 * P; break;
    case VM3DGS_DBG_PT_SLOT: src = r->at<void>(L.pt_slot); n = 4 * P * r->dims.Smax; break;
    case VM3DGS_DBG_COPIES: src = r->at<void>(L.copies); n = 16 * (int64_t)c.n_copies; break;
    case VM3DGS_DBG_DRAW: src = r->at<void>(L.draw); n = 16 * (int64_t)c.n_draw; break;
    case VM3DGS_DBG_MISSING: src = r->at<void>(L.missing); n = 4 * (int64_t)c.n_missing; break;
    case VM3DGS_DBG_SPLAT_RECT: {
      // unpack (x0 | x1 << 16, y0 | y1 << 16) into int32 x0, y0, x1, y1
      n = 16 * N;
      if (needed) *needed = n;
      if (!dst) return VM3DGS_OK;
      if (bytes < n) return fail(VM3DGS_E_CAPACITY, "destination too small");
      std::vector<uint32_t> packed(2 * N);
      if (N && !cuda_ok(cudaMemcpy(packed.data(), r->at<void>(C.splat_rect), 8 * N, cudaMemcpyDeviceToHost), "debug", &rc))
        return rc;
      int32_t *o = (int32_t *)dst;
      for (int64_t i = 0; i < N; ++i) {
        o[4 * i + 0] = (int32_t)(packed[2 * i] & 0xFFFFu);
        o[4 * i + 1] = (int32_t)(packed[2 * i + 1] & 0xFFFFu);
        o[4 * i + 2] = (int32_t)(packed[2 * i] >> 16);
        o[4 * i + 3] = (int32_t)(packed[2 * i + 1] >> 16);
      }
      return VM3DGS_OK;
    }
    case VM3DGS_DBG_SPLAT_DEPTH: src = r->at<void>(C.splat_depth); n = 4 * N; break;
    case VM3DGS_DBG_SPLAT_RADIUS: src = r->at<void>(C.splat_radius); n = 4 * N; break;
    case VM3DGS_DBG_SPLAT_TMASK: src = r->at<void>(C.splat_tmask); n = 8 * N; break;
    case VM3DGS_DBG_SPLAT_TOUCHED: src = r->at<void>(C.splat_touched); n = 4 * N; break;
    case VM3DGS_DBG_DRAW_W: src = r->at<void>(L.draw_w); n = 4 * (int64_t)c.n_draw; break;
    case VM3DGS_DBG_KEYS:
    case VM3DGS_DBG_VALUES: {
      // the sorted pairs as (tile << 32 | bits(depth), splat), whatever the
      // key layout of the last sort
      n = (what == VM3DGS_DBG_KEYS ? 8 : 4) * M;
      if (needed) *needed = n;
      if (!dst) return VM3DGS_OK;
      if (bytes < n) return fail(VM3DGS_E_CAPACITY, "destination too small");
      const KeyFormat kf = r->kf;
      std::vector<uint64_t> k(M);
      if (M && !cuda_ok(cudaMemcpy(k.data(), r->at<void>(r->sorted_buf ? C.keys1 : C.keys0), 8 * M,
                                   cudaMemcpyDeviceToHost), "debug", &rc))
        return rc;
      if (what == VM3DGS_DBG_VALUES && !kf.packed) {
        if (M && !cuda_ok(cudaMemcpy(dst, r->at<void>(r->sorted_buf ? C.vals1 : C.vals0), 4 * M,
                                     cudaMemcpyDeviceToHost), "debug", &rc))
          return rc;
        return VM3DGS_OK;
      }
      const uint64_t dmask = (1ull << kf.R) - 1ull, imask = (1ull << kf.ib) - 1ull;
      for (int64_t j = 0; j < M; ++j) {
        if (what == VM3DGS_DBG_VALUES) {
          ((uint32_t *)dst)[j] = (uint32_t)(k[j] & imask);
        } else {
          const uint64_t tile = k[j] >> kf.tshift;
          const uint32_t db = (uint32_t)(((k[j] >> kf.ib) & dmask) + kf.base);
          ((uint64_t *)dst)[j] = (tile << 32) | db;
        }
      }
      return VM3DGS_OK;
    }
    case VM3DGS_DBG_RANGES: src = r->at<void>(C.ranges); n = 8 * (int64_t)r->last_ntiles; break;
    case VM3DGS_DBG_SPLAT_XY:
    case VM3DGS_DBG_SPLAT_CONIC:
    case VM3DGS_DBG_SPLAT_RGB: {
      n = (what == VM3DGS_DBG_SPLAT_XY ? 8 : what == VM3DGS_DBG_SPLAT_CONIC ? 16 : 12) * N;
      if (needed) *needed = n;
      if (!dst) return VM3DGS_OK;
      if (bytes < n) return fail(VM3DGS_E_CAPACITY, "destination too small");
      std::vector<float4> rec(3 * N);
      if (N && !cuda_ok(cudaMemcpy(rec.data(), r->at<void>(C.splat_rec), 48 * N, cudaMemcpyDeviceToHost), "debug", &rc))
        return rc;
      float *o = (float *)dst;
      for (int64_t i = 0; i < N; ++i) {
        const float4 &a = rec[3 * i], &b = rec[3 * i + 1], &c3 = rec[3 * i + 2];
        if (what == VM3DGS_DBG_SPLAT_XY) { o[2 * i] = a.x; o[2 * i + 1] = a.y; }
        else if (what == VM3DGS_DBG_SPLAT_CONIC) { o[4 * i] = a.z; o[4 * i + 1] = a.w; o[4 * i + 2] = b.x; o[4 * i + 3] = b.y; }
        else { o[3 * i] = b.z; o[3 * i + 1] = b.w; o[3 * i + 2] = c3.x; }
      }
      return VM3DGS_OK;
    }
    case VM3DGS_DBG_POOL: src = r->pool; n = (int64_t)r->P * r->slot_bytes; break;
    case VM3DGS_DBG_RASTER: src = r->at<void>(L.raster_count); n = 20; break;
    default: return fail(VM3DGS_E_INVAL, "unknown debug item");
  }
  if (needed) *needed = n;
  if (!dst) return VM3DGS_OK;
  if (bytes < n) return fail(VM3DGS_E_CAPACITY, "destination too small");
  if (n && !cuda_ok(cudaMemcpy(dst, src, (size_t)n, cudaMemcpyDeviceToHost), "debug copy", &rc)) return rc;
  return VM3DGS_OK;
}
