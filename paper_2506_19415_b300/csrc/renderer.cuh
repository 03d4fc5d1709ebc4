// Internal renderer state, scratch layout and kernel launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "coverage.cuh"
#include "scene.h"

struct vm3dgs_renderer;

namespace vm {

// Device control block: per-frame counters, controller state, error word.
struct Ctl {
  int32_t n_req, n_direct, n_unmatched, n_admitted, n_copies, n_draw, n_missing, n_resident;
  int32_t n_free, n_fading;  // n_fading: pages drawn at two levels (LOD cross-fade)
  int64_t draw_gauss;      // Gaussians of the draw list
  int64_t pairs;           // pairs of the last rendered view
  int64_t r_drawn;         // draw_gauss as the last projection read it: the scan and emission
                           // read this copy while the next page-table update may rewrite draw_gauss
  int64_t streamed_bytes;
  int64_t copy_segments;   // 64 KiB copy segments of this frame
  float usage, tau, step;
  int32_t last_dir, last_move, frame;
  int32_t status;          // 0 or a VM3DGS_E_* code written by a kernel
  int32_t depth_lo;        // unused
  int32_t pad1;
  int32_t n_hits;          // requested pages found resident thanks to a prefetch, this frame
  int32_t pad2;
  // running sums since the last reset (read without per-frame syncs)
  int64_t acc_frames, acc_views, acc_pairs, acc_draw_gauss, acc_streamed_bytes, acc_streamed_pages, acc_missing,
      acc_requested, acc_prefetched_pages, acc_prefetched_bytes, acc_prefetch_hits;
};

struct Splats {
  float4 *rec;       // [3] per splat, one 48-byte record: (x, y, A, B), (C, opacity, r, g), (b, 0, 0, 0)
  uint32_t *depth;   // float bits of view z
  uint32_t *rect;    // [2] per splat: x0 | x1 << 16, y0 | y1 << 16
  uint32_t *touched; // tiles covered (0 = culled)
  float *radius;     // pixels
  uint64_t *tmask;   // kept tiles of a rectangle of <= 64 tiles, row-major bits (0 for larger ones)
};

// One render context: the buffers a render writes after its projection
// (splats, pairs, tile ranges, sort scratch) and its own control block (the
// drawn count it projected, its pair count, its running pair sums and
// status).  Two contexts let the projection of frame t+1 run while frame t
// is still sorted and blended.
struct CtxLayout {
  int64_t ctl, splat_rec, splat_depth, splat_rect, splat_touched, splat_radius, splat_tmask,
      block_sums, offsets, keys0, keys1, vals0, vals1, ranges, work, tile_order, hist, lookback, tile_ctr, pieces,
      piece_ctr;
};
constexpr int kContexts = 2;

// Layout of the scratch area; offsets in bytes.
struct Layout {
  int64_t ctl, fb, req, direct, reqlev, matched, draw_info, requests, ukeys, free_keys, open_list, open_off,
      admitted_pos, copies, copy_seg, draw, draw_off, missing, pt_lod, pt_last, pt_slot, required, any_req, tri_v,
      clusters, link_ptr, link_col, err, raster_queue, raster_count, raster_vis, raster_clip, raster_bands, raster_live, dreq, centroid,
      pf_flag, pf_mask, pf_cand, pf_copies, pf_copy_seg, pf_count, pf_base, pf_req, views, codebook, fade_state,
      fade_frame, fade_lev, fade_info, draw_w, total;
  CtxLayout cx[kContexts];
};

struct Dims {
  int64_t NP, P, Smax, fb_pixels, ncap, pair_cap, tile_cap, ntri, nvert, nlink, scan_blocks, lookback_words;
  int ukey_cap, free_cap;
  int64_t raster_cap;
  int64_t ncl_cap;  // proxy clusters (at most 32 triangles of one page each)
  int64_t piece_cap;  // pieces of 256 pairs of the splats with more than 32 pairs (at most pairs / 28)
  int64_t nviews;  // views a batch may hold (max_views)
  int64_t cb_floats;  // VQ pools: floats of the SH codebook (0 otherwise)
};

Dims make_dims(const vm3dgs_scene *s, const vm3dgs_params *p, int64_t P);
Layout make_layout(const Dims &d);

constexpr int kScanItems = 4096;     // elements per scan block
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxPasses = 8;
constexpr int64_t kCopySeg = 65536;

// Blocks of `threads` threads (and `smem` dynamic shared bytes) that all SMs
// of the current device hold at once: the grid of a grid-stride kernel that
// runs as one full wave, without a partial last wave.  Cached per kernel.
int full_wave(const void *kernel, int threads, size_t smem);
// Asks for the largest shared-memory carveout for a kernel that lives on
// shared memory (so that as many CTAs fit as registers allow); once per kernel.
void prefer_shared(const void *kernel);
// Raises a kernel's dynamic shared-memory limit to `bytes`, once per kernel
// and device (kernel attributes belong to a device).
void max_dynamic_smem(const void *kernel, int bytes);
// min(blocks needed for n items at `per_block` items each, full_wave), >= 1
int wave_grid(const void *kernel, int threads, size_t smem, int64_t n, int64_t per_block);

// ----- launchers (one per kernel family)
// fb (n pixels) to empty and qcount (8 words) to 0; with req also req,
// direct and dreq (NP each; dreq may be null) to 0
void launch_feedback_clear(uint64_t *fb, int64_t n, uint32_t *qcount, uint32_t *req, uint8_t *direct, uint32_t *dreq,
                           int64_t NP, cudaStream_t st);
// A run of at most 32 consecutive proxy triangles of one page with the
// axis-aligned box of their vertices (world units).
struct Cluster {
  float lo[3];
  uint32_t first;
  float hi[3];
  uint32_t count;
};
// Groups the triangles by page (stable), in clusters of at most 32; writes
// the regrouped triangles de-indexed (three planes of ntri float4 vertices,
// the page id's bits in the w of the first) and the clusters, returns their
// count.
int64_t build_clusters(const float *verts, const int32_t *tris, const int32_t *face_page, int64_t ntri, int64_t NP,
                       float *tv_out, Cluster *cl_out);
// large triangles (more than 16 pixels) are queued: queue holds qcap records of
// kRasterRecord bytes, qcount is eight device words (32 bytes, 8-aligned)
constexpr int64_t kRasterRecord = 64;
// live: ncl words for the clusters that pass the frustum test
void launch_feedback_raster(const float4 *tv, const Cluster *cl, int64_t ncl, int64_t ntri,
                            const vm3dgs_camera &cam, int ds, uint64_t *fb, void *queue,
                            uint32_t *qcount, uint32_t qcap, uint64_t *bands, uint32_t bcap, uint32_t *vis,
                            uint32_t *clip, uint32_t *live, cudaStream_t st);
// per-page maximum of the pixel codes into dst (atomic max), direct flags
void launch_feedback_reduce(const uint64_t *fb, int64_t npix, uint32_t *dst, uint8_t *direct, cudaStream_t st);
// req[p] and req of p's linked pages raised to dreq[p], for every page with dreq[p] != 0
void launch_feedback_links(const uint32_t *dreq, int64_t NP, const int64_t *link_ptr, const int32_t *link_col,
                           uint32_t *req, cudaStream_t st);
void launch_request_all(uint32_t *req, uint8_t *direct, int64_t NP, cudaStream_t st);

struct ResidencyArgs {
  Ctl *ctl;
  const uint32_t *req;
  const uint8_t *direct;
  int32_t *reqlev, *draw_info;
  uint8_t *matched;
  int4 *requests;
  uint64_t *ukeys, *free_keys;
  int32_t *open_list, *open_off, *admitted_pos;
  int4 *copies;
  int64_t *copy_seg;
  int4 *draw;
  int64_t *draw_off;
  int32_t *missing;
  int32_t *pt_lod, *pt_last, *pt_slot;
  uint8_t *required, *any_req, *pf_flag;
  // LOD cross-fade: per page the persistent state (level drawn last frame
  // + 1, fade's old level + 1, age; 0 = none), this frame's old level (-1
  // none) and its required slot (-1 none); weights of the draw items
  int32_t *fade_state, *fade_frame, *fade_lev, *fade_info;
  float *draw_w;
  int32_t fade_frames;
  const float *err;
  int32_t NP, P, Smax, levels, fanout, page_size;
  int32_t lod_on;
  int64_t budget;
  int32_t rec;        // bytes per Gaussian in the pool
  float f_px;
  float usage_lo, usage_hi;
  int32_t ukey_cap, free_cap;
};
void launch_residency(const ResidencyArgs &a, cudaStream_t st);

struct StreamArgs {
  const int32_t *count;         // number of copies (device)
  const int4 *copies;
  const int64_t *copy_seg;
  const uint8_t *host;          // device-visible pointer to the scene's page data (the pool's record)
  const int64_t *staged_off;    // null, or the byte offset in `host` of each copy (a staging buffer)
  int64_t level_off[kMaxLevels];
  int32_t page_size, fanout, rec;
  uint8_t *pool;
  int64_t slot_bytes;
};
void launch_stream(const StreamArgs &a, cudaStream_t st);

// Tensor maps of the pool, one per level: the record's float rows (a) and,
// for fp16 and VQ pools, its 16-bit rows (b), each as (Gaussian of the level block,
// row, level block of the whole pool), loaded `chunk` Gaussians at a time
// (64, or 32 when a level block holds 32 Gaussians).
struct ProjMaps {
  CUtensorMap a[kMaxLevels];
  CUtensorMap b[kMaxLevels];
  int32_t chunk;
};
struct ProjectArgs {
  const Ctl *ctl;   // the page table's control block (drawn count, draw list length)
  Ctl *rctl;        // the render context's control block (receives the drawn count as projected)
  const int4 *draw;
  const int64_t *draw_off;
  const float *draw_w;  // opacity weight of each draw item (LOD cross-fade)
  const uint8_t *pool;
  int64_t slot_bytes;
  int32_t page_size, fanout, K, fmt;  // fmt: kFmt32, kFmt16 or kFmtVQ
  const float *codebook;              // VQ pools: the SH codebook [codes][3 (K - 1)] in device memory
  int64_t ncap;
  Splats sp;
  const ProjMaps *maps;  // host copy; null: gather from the pool with plain loads
};
// Encodes the pool's tensor maps; false when a level block is not a multiple
// of 32 Gaussians or the driver refuses (the projection then gathers).
bool encode_proj_maps(const vm3dgs_scene *s, const uint8_t *pool, int64_t P, int fmt, ProjMaps *out);
void launch_project(const ProjectArgs &a, const vm3dgs_camera &cam, cudaStream_t st);

// Cameras of a batched render, in device memory.
constexpr int kMaxViews = 64;
struct ViewTable {
  vm3dgs_camera cam[kMaxViews];
  int32_t tile_off[kMaxViews + 1];   // first global tile of each view
  int32_t gx[kMaxViews];             // tiles per row
  float *img[kMaxViews];
  int32_t n;
};
void launch_project_batched(const ProjectArgs &a, const ViewTable *views, int n_views, cudaStream_t st);
void launch_scan_emit_batched(Ctl *ctl, const Splats &sp, int64_t ncap, int views, const ViewTable *vt,
                              uint32_t *block_sums, uint32_t *offsets, uint64_t *keys, uint32_t *vals,
                              int64_t pair_cap, uint64_t *pieces, uint32_t *piece_ctr, int64_t piece_cap,
                              cudaStream_t st);
void launch_blend_batched(const uint2 *ranges, const uint32_t *vals, const Splats &sp, int64_t ncap_total,
                          const ViewTable *vt, int ntiles, const float bg[3], uint32_t *order, uint32_t *work,
                          cudaStream_t st);

// Sort key of the single-view path (all fields unsigned):
//   key = tile << tshift | min(bits(depth) - base, 2^R - 1) << ib | (packed ? splat : 0)
// with depth > 0.2 for every drawn splat.  With base = bits(0.2f) and R wide
// enough for the farthest possible depth, the depth field orders exactly like
// the float bits; packed keys carry the splat index in their low ib bits and
// need no value array (emission order is splat order, and the sort is stable).
struct KeyFormat {
  int tshift, ib, R;
  uint32_t base;
  bool packed;
};
// The digit histograms of the coming sort (passes of 8 bits from lo_bit),
// counted by the emission itself, which also clears the sort's look-back
// words and tile counters (each sort pass scans its own histogram into digit
// bases).  hist null: none.
struct SortHist {
  uint32_t *hist;
  uint32_t *lookback;
  int64_t max_tiles;
  uint32_t *tile_ctr;
  int lo_bit, passes;
};
// pieces (piece_cap words) and piece_ctr: the list of kPiece-pair pieces of
// the splats with more than 32 pairs, written by the first emission kernel
// (also zeroes ranges[0 .. ntiles) for the ranges of the coming sort)
void launch_scan_emit(const Ctl *ctl, Ctl *ctl_w, const Splats &sp, int64_t ncap, uint32_t *block_sums,
                      uint32_t *offsets, uint64_t *keys, uint32_t *vals, int64_t pair_cap, const TileGeom &tg, int gx,
                      const KeyFormat &kf, const SortHist &sh, uint64_t *pieces, uint32_t *piece_ctr,
                      int64_t piece_cap, uint2 *ranges, int ntiles, cudaStream_t st);

// sorts keys/vals (pairs = ctl->pairs, capped at pair_cap) on the low `bits` bits;
// returns the index (0 or 1) of the buffer holding the result
// Stable LSD sort of the pairs on key bits [lo_bit, hi_bit); vals[0] null
// sorts the keys alone.  Returns the buffer holding the result.
int launch_sort(Ctl *ctl, uint64_t *keys[2], uint32_t *vals[2], int64_t pair_cap, int lo_bit, int hi_bit,
                uint32_t *hist, uint32_t *lookback, int64_t lookback_words, uint32_t *tile_ctr, cudaStream_t st);
// All passes in one cooperative launch (the chunk-per-CTA sort with grid
// barriers): hist holds the passes' digit counts of all pairs (counted by the
// emission), scratch 2 x 256 x grid words, bar two zeroed words.  Returns the
// buffer holding the result, -1 bad bits, -2 no cooperative launch or too
// little scratch, -3 launch refused.
int launch_sort_coop(Ctl *ctl, uint64_t *keys[2], uint32_t *vals[2], int64_t pair_cap, int lo_bit, int hi_bit,
                     const uint32_t *hist, uint32_t *scratch, int64_t scratch_words, uint32_t *bar, cudaStream_t st);
// CTAs of the cooperative sort on the current device (0: not available)
int coop_sort_grid();
// the same in two steps: digit histograms (0 or -1), then the passes
int launch_sort_prep(Ctl *ctl, const uint64_t *keys, int64_t pair_cap, int lo_bit, int hi_bit, uint32_t *hist,
                     uint32_t *lookback, int64_t lookback_words, uint32_t *tile_ctr, cudaStream_t st);
int launch_sort_passes(Ctl *ctl, uint64_t *keys[2], uint32_t *vals[2], int64_t pair_cap, int lo_bit, int hi_bit,
                       uint32_t *hist, uint32_t *lookback, uint32_t *tile_ctr, cudaStream_t st);

// zeroed: ranges[0 .. ntiles) are already zero (else they are cleared first)
void launch_ranges(const Ctl *ctl, const uint64_t *keys, int64_t pair_cap, uint2 *ranges, int ntiles, int tshift,
                   cudaStream_t st, bool zeroed = false);
// Tile processing order by descending pair count (empty tiles last); also
// resets the work counters work[0..2] (the blend uses work[1]).
void launch_tile_order(const uint2 *ranges, int ntiles, uint32_t *order, uint32_t *work, cudaStream_t st);

// req: the request words the features count (the live ones or a snapshot)
void launch_prefetch_features(const vm3dgs_renderer *r, const uint32_t *req, int n_out, const vm3dgs_camera &cam,
                              const vm3dgs_camera &prev, float *x, int32_t *base, cudaStream_t st);

// The splat of pair j is vals[j], or the low bits (idx_mask) of packed[j]
// when packed is not null; tiles are taken in `order` from the counter *work
// (reset by launch_tile_order).
// With rec_map (the tensor map of the context's splat records, rows of 48
// bytes) each batch of the tile's splats is staged by TMA: one bulk copy of
// its sorted keys, then gather loads of four records each; without, by plain
// loads.  A staging wait that expires records VM3DGS_E_TIMEOUT in ctl.
void launch_blend(const uint2 *ranges, const uint32_t *vals, const uint64_t *packed, uint32_t idx_mask,
                  const Splats &sp, int64_t ncap, const vm3dgs_camera &cam, const float bg[3], float *image,
                  uint32_t *order, uint32_t *work, const CUtensorMap *rec_map, Ctl *ctl, cudaStream_t st);
// The 2-D tensor map of n splat records (12 floats a row, one row per box):
// false when the driver refuses it.
bool encode_rec_map(const float4 *rec, int64_t n, CUtensorMap *out);

}  // namespace vm

struct vm3dgs_renderer {
  const vm3dgs_scene *scene = nullptr;
  vm3dgs_params prm{};
  uint8_t *pool = nullptr;
  int64_t pool_bytes = 0, slot_bytes = 0;
  int32_t P = 0;
  int32_t rec = 0;
  int32_t fmt = 0;  // pool record: vm::kFmt32, kFmt16 or kFmtVQ
  uint8_t *scratch = nullptr;
  vm::Dims dims{};
  vm::Layout lay{};
  const uint8_t *host_dev = nullptr;   // device-visible pointer to the pages streamed
  // scene opened from a file: the frame's pages pass through a page-locked
  // staging buffer the host fills from the file mapping (Sec. 4.1, Transfer)
  bool staged = false;
  uint8_t *staging = nullptr;           // page-locked, staging_bytes
  int32_t *h_count = nullptr;           // page-locked copy-list readback
  int4 *h_copies = nullptr;
  int64_t *h_off = nullptr;             // mapped page-locked byte offsets of the copies in staging
  const int64_t *h_off_dev = nullptr;   // its device-visible pointer
  int staged_err = 0;                   // set by the host gather, reported by the next update
  int state = 0;                        // 0 idle, 1 feedback done, 2 residency done
  float f_px = 0.0f;
  cudaEvent_t copy_done = nullptr;
  bool copy_pending = false;
  cudaEvent_t res_done = nullptr;   // recorded after each page-table update
  // request words and direct flags are double-buffered: page determination
  // writes buffer fb_buf ^ 1 while the update may still read buffer fb_buf
  int fb_buf = 1;                   // buffer of the last page determination
  cudaEvent_t res_done_buf[2] = {nullptr, nullptr};  // the last update that read buffer k
  bool res_recorded_buf[2] = {false, false};
  int pf_req_buf = 0;               // buffer the pending prefetch copies
  int res_buf = 0;                  // buffer the last update read
  uint32_t *req_buf(int k) const { return at<uint32_t>(lay.req) + k * dims.NP; }
  uint8_t *direct_buf(int k) const { return at<uint8_t>(lay.direct) + k * dims.NP; }
  cudaEvent_t fb_done = nullptr;    // recorded after each page determination
  cudaEvent_t upd_done = nullptr;   // recorded after each page-table update and its in-line copies
  cudaEvent_t proj_done = nullptr;  // recorded after each render's last projection (pool reads done)
  bool res_recorded = false, fb_recorded = false, upd_recorded = false, proj_recorded = false;
  cudaEvent_t pf_done = nullptr;    // recorded after a prefetch's page-table and pool writes
  cudaEvent_t pf_req_done = nullptr;  // recorded after a prefetch took its copy of the request words
  bool pf_pending = false, pf_req_pending = false;
  int64_t last_fb_pixels = 0;
  int64_t ncl = 0;  // proxy clusters in use
  double gbox_lo[3] = {0, 0, 0}, gbox_hi[3] = {0, 0, 0};  // holds every Gaussian mean
  vm::KeyFormat kf{32, 0, 32, 0u, false};  // of the last sort
  bool maps_ok = false;
  vm::ProjMaps maps{};
  bool rec_maps_ok = false;        // the blend stages splat records by TMA
  CUtensorMap rec_map[vm::kContexts];
  float scene_center[3] = {0, 0, 0}, scene_half = 1.0f;
  // captured batch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraphNode_t graph_views_node = nullptr;
  vm::ViewTable graph_table{};
  int tuned_shape[4] = {0, 0, 0, 0};
  int sorted_buf = 0;     // pair buffer (0/1) holding the last view's sorted pairs
  int ctx = 0;            // render context the next single-view render takes
  int last_ctx = 0;       // render context of the last render
  cudaEvent_t ctx_free[vm::kContexts] = {nullptr, nullptr};  // recorded after each render's last kernel
  bool ctx_recorded[vm::kContexts] = {false, false};
  int last_ntiles = 0;
  // per-stage timing
  struct TimedSpan { int stage; int launches; cudaEvent_t a, b; };
  bool timing = false;
  std::vector<TimedSpan> spans;
  std::vector<cudaEvent_t> spare_events;
  cudaEvent_t take_event() {
    cudaEvent_t e = nullptr;
    if (!spare_events.empty()) { e = spare_events.back(); spare_events.pop_back(); }
    else cudaEventCreate(&e);
    return e;
  }
  int span_begin(int stage, cudaStream_t st) {
    if (!timing) return -1;
    TimedSpan t{stage, 0, take_event(), take_event()};
    cudaEventRecord(t.a, st);
    spans.push_back(t);
    return (int)spans.size() - 1;
  }
  void span_end(int idx, int launches, cudaStream_t st) {
    if (idx < 0) return;
    spans[idx].launches = launches;
    cudaEventRecord(spans[idx].b, st);
  }
  template <class T>
  T *at(int64_t off) const { return reinterpret_cast<T *>(scratch + off); }
};

namespace vm {
// the splat arrays of render context k
Splats splats_of(const vm3dgs_renderer *r, int k);
}  // namespace vm
