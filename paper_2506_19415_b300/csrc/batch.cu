// Many views of uneven resolution rendered together over one shared pool:
// one projection launch over (view, Gaussian), one scan / pair emission and
// one radix sort over the pairs of all views (keys carry a global tile id:
// the view's first tile plus its local tile), one persistent blend over all
// (view, tile) items with per-view tile shapes.  The cameras live in a
// device table written by a kernel that takes the table by value, so a CUDA
// graph of the whole batch can be replayed with new poses by updating that
// one node.  A tile-shape autotuner picks 8x8 / 16x16 / 32x8 per resolution
// class by timing the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "renderer.cuh"

namespace vm {
namespace {

__global__ void load_views_kernel(ViewTable tbl, ViewTable *dst) {
  // word-parallel copy of the table into device memory
  const uint32_t *src = reinterpret_cast<const uint32_t *>(&tbl);
  uint32_t *d = reinterpret_cast<uint32_t *>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(ViewTable) / 4); i += blockDim.x) d[i] = src[i];
}

bool tile_ok(int w, int h) { return (w == 16 && h == 16) || (w == 8 && h == 8) || (w == 32 && h == 8); }

int make_table(const vm3dgs_renderer *r, const vm3dgs_camera *cams, int n, float *const *images, ViewTable *t) {
  if (!cams || n <= 0) return fail(VM3DGS_E_INVAL, "no cameras");
  if (n > kMaxViews || n > (r->prm.max_views > 0 ? r->prm.max_views : 1))
    return fail(VM3DGS_E_INVAL, "more views than max_views (at most " + std::to_string(kMaxViews) + ")");
  std::memset(t, 0, sizeof(*t));
  int64_t off = 0;
  for (int v = 0; v < n; ++v) {
    const vm3dgs_camera &c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > r->prm.max_width || c.height > r->prm.max_height)
      return fail(VM3DGS_E_INVAL, "camera size outside the renderer's maximum");
    if (!tile_ok(c.tile_w, c.tile_h)) return fail(VM3DGS_E_INVAL, "tile shape must be 16x16, 8x8 or 32x8");
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(c.view[i])) return fail(VM3DGS_E_INVAL, "camera matrix is not finite");
    if (!(c.fx > 0) || !(c.fy > 0)) return fail(VM3DGS_E_INVAL, "camera intrinsics are not positive");
    if (images && !images[v]) return fail(VM3DGS_E_INVAL, "null image");
    const int gx = (c.width + c.tile_w - 1) / c.tile_w, gy = (c.height + c.tile_h - 1) / c.tile_h;
    t->cam[v] = c;
    t->gx[v] = gx;
    t->tile_off[v] = (int32_t)off;
    t->img[v] = images ? images[v] : nullptr;
    off += (int64_t)gx * gy;
  }
  if (off > r->dims.tile_cap * (int64_t)(r->prm.max_views > 0 ? r->prm.max_views : 1))
    return fail(VM3DGS_E_CAPACITY, "too many tiles in the batch");
  t->tile_off[n] = (int32_t)off;
  t->n = n;
  return VM3DGS_OK;
}

// the batch's kernels, in stream order (also what a graph captures); batches
// always take render context 0
int enqueue_batch(vm3dgs_renderer *r, const ViewTable &t, cudaStream_t st, bool timed) {
  const vm3dgs_scene *s = r->scene;
  const CtxLayout &C = r->lay.cx[0];
  Ctl *ctl = r->at<Ctl>(C.ctl);
  ViewTable *dvt = r->at<ViewTable>(r->lay.views);
  load_views_kernel<<<1, 256, 0, st>>>(t, dvt);
  const Splats sp = splats_of(r, 0);
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
  const int n = t.n;
  int span = timed ? r->span_begin(VM3DGS_STAGE_PROJECT, st) : -1;
  launch_project_batched(pa, dvt, n, st);
  r->span_end(span, 2, st);
  uint64_t *keys[2] = {r->at<uint64_t>(C.keys0), r->at<uint64_t>(C.keys1)};
  uint32_t *vals[2] = {r->at<uint32_t>(C.vals0), r->at<uint32_t>(C.vals1)};
  span = timed ? r->span_begin(VM3DGS_STAGE_SCAN_EMIT, st) : -1;
  launch_scan_emit_batched(ctl, sp, r->dims.ncap, n, dvt, r->at<uint32_t>(C.block_sums),
                           r->at<uint32_t>(C.offsets), keys[0], vals[0], r->dims.pair_cap,
                           r->at<uint64_t>(C.pieces), r->at<uint32_t>(C.piece_ctr), r->dims.piece_cap, st);
  r->span_end(span, 4, st);
  const int ntiles = t.tile_off[n];
  int tbits = 0;
  while ((1 << tbits) < ntiles) ++tbits;
  span = timed ? r->span_begin(VM3DGS_STAGE_SORT, st) : -1;
  const int cur = launch_sort(ctl, keys, vals, r->dims.pair_cap, 0, 32 + tbits, r->at<uint32_t>(C.hist),
                              r->at<uint32_t>(C.lookback), r->dims.lookback_words,
                              r->at<uint32_t>(C.tile_ctr), st);
  r->span_end(span, 1 + (32 + tbits + 7) / 8, st);  // histograms, passes
  if (cur == -2) return fail(VM3DGS_E_CUDA, "sort shared-memory attribute refused");
  if (cur < 0) return fail(VM3DGS_E_CAPACITY, "sort look-back area too small");
  uint2 *ranges = r->at<uint2>(C.ranges);
  span = timed ? r->span_begin(VM3DGS_STAGE_RANGES, st) : -1;
  launch_ranges(ctl, keys[cur], r->dims.pair_cap, ranges, ntiles, 32, st);
  r->span_end(span, 1, st);
  span = timed ? r->span_begin(VM3DGS_STAGE_BLEND, st) : -1;
  launch_blend_batched(ranges, vals[cur], sp, r->dims.ncap * (int64_t)n, dvt, ntiles, r->prm.bg,
                       r->at<uint32_t>(C.tile_order), r->at<uint32_t>(C.work), st);
  r->span_end(span, 2, st);
  r->sorted_buf = cur;
  r->kf = KeyFormat{32, 0, 32, 0u, false};
  r->last_ntiles = ntiles;
  r->last_ctx = 0;
  return VM3DGS_OK;
}

}  // namespace
}  // namespace vm

using namespace vm;

extern "C" int vm3dgs_render_batched(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams,
                                     float *const *images, void *stream) {
  if (!r || !images) return fail(VM3DGS_E_INVAL, "null argument");
  if (r->state < 2) return fail(VM3DGS_E_STATE, "render before update_residency");
  ViewTable t;
  int rc = make_table(r, cams, n_cams, images, &t);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (r->copy_pending) {
    cudaStreamWaitEvent(st, r->copy_done, 0);
    r->copy_pending = false;
  }
  if (r->upd_recorded) cudaStreamWaitEvent(st, r->upd_done, 0);
  if (r->ctx_recorded[0]) cudaStreamWaitEvent(st, r->ctx_free[0], 0);
  rc = enqueue_batch(r, t, st, r->timing);
  if (rc) return rc;
  cudaEventRecord(r->proj_done, st);  // conservatively after the whole batch
  r->proj_recorded = true;
  cudaEventRecord(r->ctx_free[0], st);
  r->ctx_recorded[0] = true;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, std::string("render_batched: ") + cudaGetErrorString(e));
}

extern "C" int vm3dgs_batch_graph_capture(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams,
                                          float *const *images, void *stream) {
  if (!r || !images) return fail(VM3DGS_E_INVAL, "null argument");
  ViewTable t;
  int rc = make_table(r, cams, n_cams, images, &t);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return fail(VM3DGS_E_INVAL, "capture needs a non-default stream");
  if (r->graph_exec) {
    cudaGraphExecDestroy(r->graph_exec);
    r->graph_exec = nullptr;
  }
  if (r->graph) {
    cudaGraphDestroy(r->graph);
    r->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(VM3DGS_E_CUDA, "cudaStreamBeginCapture failed");
  rc = enqueue_batch(r, t, st, false);
  const cudaError_t ec = cudaStreamEndCapture(st, &g);
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (ec != cudaSuccess || !g) return fail(VM3DGS_E_CUDA, std::string("capture: ") + cudaGetErrorString(ec));
  // the node that loads the camera table
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  r->graph_views_node = nullptr;
  for (auto node : nodes) {
    cudaGraphNodeType ty;
    cudaGraphNodeGetType(node, &ty);
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(node, &kp) == cudaSuccess && kp.func == (void *)load_views_kernel) {
      r->graph_views_node = node;
      break;
    }
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  r->graph = g;
  if (ei != cudaSuccess || !r->graph_views_node) return fail(VM3DGS_E_CUDA, "graph instantiation failed");
  r->graph_exec = ex;
  r->graph_table = t;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_batch_graph_launch(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams,
                                         void *stream) {
  if (!r || !r->graph_exec) return fail(VM3DGS_E_STATE, "no captured batch");
  if (r->state < 2) return fail(VM3DGS_E_STATE, "render before update_residency");
  if (n_cams != r->graph_table.n) return fail(VM3DGS_E_INVAL, "view count differs from the captured batch");
  ViewTable t = r->graph_table;
  for (int v = 0; v < n_cams; ++v) {
    const vm3dgs_camera &c = cams[v], &o = r->graph_table.cam[v];
    if (c.width != o.width || c.height != o.height || c.tile_w != o.tile_w || c.tile_h != o.tile_h)
      return fail(VM3DGS_E_INVAL, "resolution or tile shape differs from the captured batch");
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(c.view[i])) return fail(VM3DGS_E_INVAL, "camera matrix is not finite");
    t.cam[v] = c;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (r->copy_pending) {
    cudaStreamWaitEvent(st, r->copy_done, 0);
    r->copy_pending = false;
  }
  if (r->upd_recorded) cudaStreamWaitEvent(st, r->upd_done, 0);
  if (r->ctx_recorded[0]) cudaStreamWaitEvent(st, r->ctx_free[0], 0);
  ViewTable *dvt = r->at<ViewTable>(r->lay.views);
  void *args[2] = {&t, &dvt};
  cudaKernelNodeParams kp{};
  kp.func = (void *)load_views_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(256);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  if (cudaGraphExecKernelNodeSetParams(r->graph_exec, r->graph_views_node, &kp) != cudaSuccess)
    return fail(VM3DGS_E_CUDA, "graph node update failed");
  const cudaError_t e = cudaGraphLaunch(r->graph_exec, st);
  cudaEventRecord(r->proj_done, st);
  r->proj_recorded = true;
  cudaEventRecord(r->ctx_free[0], st);
  r->ctx_recorded[0] = true;
  r->last_ctx = 0;
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
}

extern "C" int vm3dgs_autotune_tiles(vm3dgs_renderer *r, vm3dgs_camera *cams, int32_t n_cams, float *const *images,
                                     int32_t repeats, void *stream) {
  if (!r || !cams || !images || n_cams <= 0) return fail(VM3DGS_E_INVAL, "null argument");
  if (r->state < 2) return fail(VM3DGS_E_STATE, "autotune before update_residency");
  cudaStream_t st = (cudaStream_t)stream;
  const int shapes[3][2] = {{16, 16}, {8, 8}, {32, 8}};
  // resolution classes by pixel count: < 0.5, < 1, < 1.5, >= 1.5 megapixels
  auto cls = [](const vm3dgs_camera &c) {
    const double mp = (double)c.width * c.height / 1.0e6;
    return mp < 0.5 ? 0 : mp < 1.0 ? 1 : mp < 1.5 ? 2 : 3;
  };
  std::vector<vm3dgs_camera> cur(cams, cams + n_cams);
  for (auto &c : cur) { c.tile_w = 16; c.tile_h = 16; }
  if (r->copy_pending) {
    cudaStreamWaitEvent(st, r->copy_done, 0);
    r->copy_pending = false;
  }
  if (r->upd_recorded) cudaStreamWaitEvent(st, r->upd_done, 0);
  if (r->ctx_recorded[0]) cudaStreamWaitEvent(st, r->ctx_free[0], 0);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const bool was_timing = r->timing;
  r->timing = false;
  auto time_batch = [&](const std::vector<vm3dgs_camera> &cs, float *ms) -> int {
    ViewTable t;
    int rc = make_table(r, cs.data(), n_cams, images, &t);
    if (rc) return rc;
    rc = enqueue_batch(r, t, st, false);  // warm
    if (rc) return rc;
    std::vector<float> v;
    for (int k = 0; k < (repeats > 0 ? repeats : 3); ++k) {
      cudaEventRecord(a, st);
      enqueue_batch(r, t, st, false);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float x = 0;
      cudaEventElapsedTime(&x, a, b);
      v.push_back(x);
    }
    std::sort(v.begin(), v.end());
    *ms = v[v.size() / 2];
    return VM3DGS_OK;
  };
  int rc = VM3DGS_OK;
  for (int c = 0; c < 4 && rc == VM3DGS_OK; ++c) {
    bool any = false;
    for (auto &cam : cur) any = any || cls(cam) == c;
    if (!any) continue;
    float best_ms = 1e30f;
    int best = 0;
    for (int k = 0; k < 3; ++k) {
      for (auto &cam : cur)
        if (cls(cam) == c) { cam.tile_w = shapes[k][0]; cam.tile_h = shapes[k][1]; }
      float ms = 0;
      rc = time_batch(cur, &ms);
      if (rc) break;
      if (ms < best_ms) { best_ms = ms; best = k; }
    }
    for (auto &cam : cur)
      if (cls(cam) == c) { cam.tile_w = shapes[best][0]; cam.tile_h = shapes[best][1]; }
    r->tuned_shape[c] = best;
  }
  r->timing = was_timing;
  cudaEventRecord(r->proj_done, st);
  r->proj_recorded = true;
  cudaEventRecord(r->ctx_free[0], st);
  r->ctx_recorded[0] = true;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  for (int v = 0; v < n_cams; ++v) { cams[v].tile_w = cur[v].tile_w; cams[v].tile_h = cur[v].tile_h; }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
}
