/*
 * vm3dgs — virtual-memory 3D Gaussian Splatting, per-frame path on one GPU.
 *
 * C ABI of the library libvm3dgs.so.  Every function is extern "C", takes
 * plain pointers and sizes, and returns 0 (VM3DGS_OK) or a negative error
 * code; vm3dgs_last_error() then holds a one-line, thread-local message.
 * Streams are cudaStream_t values passed as void*.  The library never calls
 * cudaMalloc: device memory (the page pool, the scratch area, the images) is
 * owned by the caller and only borrowed.  Host input arrays are borrowed for
 * the duration of a call and copied.
 *
 * The calls follow the problem the paper (Haberl et al., "Virtual Memory for
 * 3D Gaussian Splatting", arXiv 2506.19415) sets: a trained scene in the
 * Kerbl 3DGS format is prepared once into pages with links, levels of detail
 * and a proxy mesh (Sec. 3), then every frame determines the visible pages
 * from a page-ID visibility buffer (Sec. 4.1 "Page Determination"), updates
 * a page table and streams missing pages into a fixed device buffer
 * (Sec. 4.1 "Page Table Management"), and renders only the resident
 * Gaussians (Sec. 4.2 "Rendering").
 *
 * Frame protocol: vm3dgs_render_feedback -> vm3dgs_update_residency ->
 * vm3dgs_render.  Calls on one renderer are not thread safe.  Each call may
 * be given a stream of its own; the renderer orders them with CUDA events so
 * that the results equal those of one stream:
 *   - page determination writes one of two request buffers, after the update
 *     that read that buffer (two page determinations ago) and after the
 *     previous page determination, so it may run a frame ahead;
 *   - the update reads the latest page determination's buffer, after it and
 *     after the previous render's projection (its last read of the pool and
 *     draw list);
 *   - a render takes one of two render contexts (splat, pair and sort
 *     buffers), after the update and after the last render that used that
 *     context, so consecutive renders may overlap.
 */
#ifndef VM3DGS_H
#define VM3DGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- errors */
#define VM3DGS_OK 0
#define VM3DGS_E_INVAL (-1)    /* null pointer, out-of-range size, NaN camera */
#define VM3DGS_E_CAPACITY (-2) /* pool, scratch or pair capacity too small */
#define VM3DGS_E_CUDA (-3)     /* a CUDA runtime call failed */
#define VM3DGS_E_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define VM3DGS_E_STATE (-5)    /* call order violated */
#define VM3DGS_E_NOMEM (-6)    /* host allocation failed */

typedef struct vm3dgs_scene vm3dgs_scene;       /* built pages in host memory */
typedef struct vm3dgs_renderer vm3dgs_renderer; /* page table, pool view, scratch view */

/* Raw Gaussians in the layout of the 3DGS PLY export (Kerbl et al.), with
 * the normals already dropped.  K = (sh_degree+1)^2. */
typedef struct {
  int64_t n;
  int32_t sh_degree;       /* 0..3 */
  const float *pos;        /* [n][3] world position */
  const float *log_scale;  /* [n][3] log of the axis scales */
  const float *rot;        /* [n][4] quaternion (w,x,y,z), any non-zero norm */
  const float *op_logit;   /* [n] opacity before the logistic function */
  const float *f_dc;       /* [n][3] degree-0 SH coefficient per colour channel */
  const float *f_rest;     /* [n][3][K-1] higher SH, channel-major; NULL if K == 1 */
} vm3dgs_gaussians;

/* Offline preparation parameters (Sec. 3). */
typedef struct {
  int32_t page_size;       /* Gaussians per level-0 page (Sec. 3.2) */
  int32_t paging;          /* 0: Morton order in chunks; 1: octree leaves merged greedily */
  int32_t lod_levels;      /* levels incl. level 0 (Sec. 3.4); 1 = no LOD */
  int32_t lod_fanout;      /* children merged per parent; page size shrinks by it per level */
  double lo[3], hi[3];     /* scene box: crop (Sec. 3.5), Morton quantisation, voxel grid */
  double voxel;            /* proxy voxel edge in world units */
  double kappa;            /* voxel occupied when its means' opacities sum to >= kappa */
  int32_t closing;         /* 1: one 3x3x3 closing of the occupancy */
  int32_t link_samples;    /* random points per Gaussian for page linking (Sec. 3.3) */
  double link_sigma;       /* ellipsoid extent of the samples, in standard deviations */
  uint64_t seed;           /* SplitMix64 key of the link samples */
  int32_t links;           /* 0: build no links */
  int32_t fp16;            /* 1: also build the fp16 page records */
  int32_t n_threads;       /* host threads, 0 = all */
  /* LOD construction (Sec. 3.4).  0: moment matching of `lod_fanout`
   * consecutive children.  1: the paper's k-means -- per page, the real
   * Gaussians of level l-1 are clustered into ceil(n / lod_fanout) clusters
   * (Lloyd's iterations from evenly spaced seeds, at most kmeans_iters) on
   * features: position centred and divided by the page's RMS radius, then
   * kmeans_attr_weight x (quaternion with w >= 0, degree-0 SH colour,
   * opacity); each non-empty cluster becomes one parent with the mean
   * position, quaternion, opacity and SH and the mean scale times
   * kmeans_scale (0: lod_fanout^(1/3)) when it merges two or more.  The
   * page's error at a level is the largest member distance from its parent
   * plus that member's largest scale.  E_INVAL for another method,
   * kmeans_iters < 1 or a negative scale or weight. */
  int32_t lod_method;
  int32_t kmeans_iters;
  double kmeans_scale;
  double kmeans_attr_weight;
  /* paging = 2, the paper's mesh proxy and page assignment (Sec. 3.1, 3.2),
   * computed on the current CUDA device: the scene box is sampled at voxel
   * centres lo + (i + 1/2) voxel; a sample point is occupied when it lies in
   * the mesh_kappa-sigma ellipsoid of a Gaussian of opacity >= mesh_op_min
   * (the points of each scene slice inside the ellipse where the slice cuts
   * the ellipsoid); the occupancy is closed with the cube of radius
   * mesh_closing voxels; its boundary is extracted cube by cube from the 6
   * tetrahedra of each cube (vertices at inside-outside midpoints); quadric
   * edge collapses keep mesh_qem_ratio of the triangles.  Gaussians go to
   * their nearest triangle; a triangle with more than page_size is split at
   * the midpoint of its first edge (rotated vertex order) until none has;
   * triangles merge breadth-first into pages of at most page_size (a
   * triangle that would overflow starts the next page; the nearest
   * unassigned triangle continues a page without neighbours left).  Links:
   * the nearest triangle of each link sample.  The proxy is that mesh. */
  double mesh_kappa;
  double mesh_op_min;
  int32_t mesh_closing;
  double mesh_qem_ratio;
} vm3dgs_build_params;

/* Pinhole camera, OpenCV axes (+x right, +y down, +z forward). */
typedef struct {
  float view[12];          /* world -> camera [R|t], rows */
  float campos[3];         /* camera centre, world */
  float fx, fy, cx, cy;    /* pixels; pixel (i,j) covers [i,i+1) x [j,j+1) */
  int32_t width, height;
  int32_t tile_w, tile_h;  /* splat tile: 8x8, 16x16 or 32x8 */
} vm3dgs_camera;

/* Renderer parameters. */
typedef struct {
  int64_t staging_bytes;   /* bytes streamed per update at most (the staging budget) */
  int32_t feedback_ds;     /* visibility buffer is ceil(W/ds) x ceil(H/ds); ceil(max_height/ds) <= 16000 */
  int32_t links;           /* follow page links in the reduction */
  int32_t lod;             /* choose levels by screen-space error, adapt the threshold */
  int32_t fp16_pool;       /* pool records: 0 fp32; 1 fp16 (scene built with fp16 = 1); 2 VQ with the
                              SH codebook (after vm3dgs_scene_quantize_sh); all arithmetic is FP32 */
  float usage_lo, usage_hi;/* target band of pool usage (0.5, 0.8) */
  float tau0, step0;       /* initial screen-space error threshold and step, pixels */
  int32_t max_width, max_height; /* largest view rendered */
  int32_t max_views;       /* largest n_cams passed to vm3dgs_render */
  int64_t max_pairs;       /* (Gaussian, tile) pairs per view; 0 = max(8 x pool Gaussians, 2^22) */
  float bg[3];             /* background colour */
  int32_t separate_values; /* 0: the splat index rides in the low bits of the sort key whenever tile, depth and
                              index bits fit in 64 (a keys-only sort); 1: always sort (key, splat) pairs.  The
                              rendered image and the pairs read back are the same either way. */
  int32_t sort_mode;       /* radix sort of a single-view render: 0 = one onesweep launch per pass (decoupled
                              look-back; the default), 1 = all passes in one cooperative launch (a chunk per CTA,
                              bounded grid barriers; where the device supports cooperative launches, else as 0).
                              Same sorted pairs either way. */
  int32_t lod_fade_frames; /* LOD cross-fade (Sec. 4.1 and 4.3 leave blending between levels, with both levels
                              resident during a transition, to a renderer with 3DGS alpha blending): 0 = off; F in
                              1..255: a page drawn last frame at a level other than the one it now needs keeps its
                              old copy required (if resident; it is never copied for this) for F frames and is
                              drawn at both levels, the old one after the new with opacity weight 1 - w, the new
                              one with w = (age + 1) / (F + 1) (float32; one of them alone: weight 1); the fade
                              ends at age F or when the page needs its old level again; a page not requested
                              forgets its fade.  Draw lists may then hold two items of a page (the draw list
                              capacity is 2 n_pages). */
} vm3dgs_params;

typedef struct {
  int32_t frame;
  int32_t requested;       /* pages in the request list */
  int32_t direct;          /* of which seen directly (not only through links) */
  int32_t resident;        /* requested and already resident at the chosen level */
  int32_t missing;         /* requested but neither resident nor streamed */
  int32_t streamed_pages;
  int64_t streamed_bytes;
  int32_t drawn_pages;
  int64_t drawn_gaussians;
  int64_t pairs;           /* (Gaussian, tile) pairs of the last rendered view */
  float usage;             /* drawn Gaussian capacity / pool capacity */
  float tau;               /* threshold used for the next frame */
  int32_t status;          /* device error word: 0 ok, else VM3DGS_E_* */
  /* running sums since the renderer was created or the sums were reset */
  int64_t acc_frames, acc_views, acc_pairs, acc_drawn_gaussians, acc_streamed_bytes, acc_streamed_pages,
      acc_missing, acc_requested;
  int64_t acc_prefetched_pages, acc_prefetched_bytes, acc_prefetch_hits;  /* hits: requested pages found resident
                                                                            because a prefetch brought them */
  int32_t staged_projection; /* 1: the projection stages records with tensor-map tile loads (every level block a
                                multiple of 32 Gaussians); 0: it gathers them with plain loads */
  /* sort key of the last rendered view: tile, depth and splat-index field
   * widths in bits (index 0 when the index travels in a value array, i.e.
   * key_packed = 0); the sort orders the key's tile and depth fields */
  int32_t key_tile_bits, key_depth_bits, key_index_bits, key_packed;
  int32_t fading;          /* pages drawn at two levels this frame (LOD cross-fade) */
} vm3dgs_stats;

typedef struct {
  int32_t n_pages;         /* virtual pages */
  int32_t page_size, lod_levels, lod_fanout, sh_degree;
  int64_t n_gaussians;     /* real level-0 Gaussians after cropping */
  int32_t record_bytes;    /* fp32 record: 4*(11 + 3K) */
  int32_t record_bytes16;  /* fp16 record, 0 if not built */
  int64_t n_tris;          /* proxy triangles */
  int64_t n_verts;
  int64_t n_links;
  int64_t host_bytes;      /* all page data held */
  int32_t record_bytes_vq; /* VQ record (40 bytes), 0 until vm3dgs_scene_quantize_sh */
  int32_t n_codes;         /* SH codebook entries, 0 until then */
} vm3dgs_scene_info;

/* Offline preparation (Sec. 3): decode (Sec. 3.5), page (Sec. 3.2), LOD
 * (Sec. 3.4), voxel proxy with page-marked faces (Sec. 3.1 stand-in), links
 * (Sec. 3.3).  Runs on the host; needs no GPU.  *out owns its memory. */
int vm3dgs_build_pages(const vm3dgs_gaussians *in, const vm3dgs_build_params *bp, vm3dgs_scene **out);

/* Wraps already-prepared pages (for example from another preparation tool)
 * into a scene.  Arrays are per level l, [n_pages][m_l][...] with
 * m_l = page_size / fanout^l; sh is [..][K][3]; err is [n_pages][levels];
 * the proxy is verts[n_verts][3], tris[n_tris][3], face_page[n_tris] (-1 =
 * none); links are a CSR link_ptr[n_pages+1], link_col[n_links]. */
typedef struct {
  int32_t n_pages, page_size, lod_levels, lod_fanout, sh_degree, fp16;
  const float *const *pos;      /* [levels] */
  const float *const *scale;    /* [levels] */
  const float *const *rot;      /* [levels] */
  const float *const *opacity;  /* [levels] */
  const float *const *sh;       /* [levels] */
  const float *err;
  const int64_t *count;         /* [n_pages] real level-0 Gaussians */
  int64_t n_verts, n_tris, n_links;
  const float *verts;
  const int32_t *tris;
  const int32_t *face_page;
  const int64_t *link_ptr;
  const int32_t *link_col;
} vm3dgs_scene_desc;
int vm3dgs_scene_import(const vm3dgs_scene_desc *d, vm3dgs_scene **out);

int vm3dgs_scene_info_get(const vm3dgs_scene *s, vm3dgs_scene_info *out);

/* Copies one internal array of the scene to host memory for inspection.
 * what: see VM3DGS_SCENE_*; level selects the LOD level where it applies.
 * Returns E_CAPACITY (with *needed set) when bytes is too small. */
enum {
  VM3DGS_SCENE_PAGE_COUNT = 0,  /* int64 [n_pages] */
  VM3DGS_SCENE_PAGE_SRC = 1,    /* int64 [n_pages][page_size] input index, -1 padding */
  VM3DGS_SCENE_PAGES = 2,       /* the level's page blocks, fp32 SoA, [n_pages][rec*m_l] bytes */
  VM3DGS_SCENE_PAGES16 = 3,     /* same in the fp16 record */
  VM3DGS_SCENE_ERR = 4,         /* float [n_pages][levels] */
  VM3DGS_SCENE_VERTS = 5,       /* float [n_verts][3] */
  VM3DGS_SCENE_TRIS = 6,        /* int32 [n_tris][3] */
  VM3DGS_SCENE_FACE_PAGE = 7,   /* int32 [n_tris] */
  VM3DGS_SCENE_LINK_PTR = 8,    /* int64 [n_pages+1] */
  VM3DGS_SCENE_LINK_COL = 9,    /* int32 [n_links] */
  VM3DGS_SCENE_CODEBOOK = 10,   /* float [n_codes][3 (K - 1)] SH codebook */
  VM3DGS_SCENE_PAGES_VQ = 11    /* the level's page blocks in the VQ record */
};
int vm3dgs_scene_export(const vm3dgs_scene *s, int32_t what, int32_t level, void *dst, int64_t bytes,
                        int64_t *needed);
void vm3dgs_scene_destroy(vm3dgs_scene *s);

/* Scene files (Sec. 3.5, "Scene Storage": the proxy loads at once, the
 * Gaussians stay in a memory-mapped file that the OS reads on demand, so a
 * scene may exceed host memory).
 *
 * vm3dgs_scene_save writes everything a scene holds to `path` (a
 * little-endian binary of this library's own layout: a header, the per-page
 * counts, sources, errors, proxy mesh, links and centroids, then the fp32 and,
 * if built, fp16 page data, each at a 4096-byte aligned offset).  E_INVAL if
 * the file cannot be written.
 *
 * vm3dgs_scene_open reads the header and the small arrays and maps the page
 * data read-only; *out owns the mapping.  E_INVAL for a missing, truncated or
 * inconsistent file, E_NOMEM if the mapping fails.  A renderer on an opened
 * scene moves pages as the paper does: vm3dgs_update_residency reads the copy
 * list back, copies the pages from the mapping into a page-locked staging
 * buffer of staging_bytes with host threads, and streams from there, all on
 * `stream` (the gather is a host function in stream order, so the call does
 * not wait; its copy_stream is not used); the frame's results equal those of
 * the in-memory scene.  vm3dgs_prefetch returns E_STATE on such a renderer. */
int vm3dgs_scene_save(const vm3dgs_scene *s, const char *path);
int vm3dgs_scene_open(const char *path, vm3dgs_scene **out);

/* Compressed pages (Sec. 6 leaves them to future work: codebooks of
 * quantised attributes kept in GPU memory, so that pages carry an index and
 * less data is copied; Sec. 2, Compression, names k-means vector
 * quantisation of the spherical harmonics).  Adds to the scene an SH
 * codebook and a third page record, the VQ record (40 bytes at any SH
 * degree, against 128 fp16 / 236 fp32 bytes at degree 3):
 *   floats   position x, y, z, opacity
 *   16 bit   scale (3), rotation (4), SH band 0 (3) as half; the index of
 *            the Gaussian's codeword for SH bands 1..3; one padding word
 * Codebook: n_codes vectors of the 3 (K - 1) view-dependent coefficients,
 * (coefficient, channel) order, by Lloyd's iterations (at most `iters`,
 * stopping when an assignment repeats; squared Euclidean distance in FP64,
 * features summed in order, lowest index on a tie; a codeword without
 * vectors stays) on the real level-0 Gaussians in slot order, or, when there
 * are more than n_train, those at positions floor(j T / n_train); started
 * from the training vectors at floor(j T' / n_codes); rounded to fp32.  Every
 * Gaussian of every level (padding too) takes the nearest fp32 codeword.
 * Host computation (OpenMP); the records are the scene's own memory.  A
 * renderer with params.fp16_pool = 2 holds VQ records in its pool and the
 * codebook in its scratch.  E_INVAL: SH degree 0, n_codes outside
 * 1..65536, fewer training Gaussians than codes; E_STATE: the scene already
 * holds VQ records (they are made once, before any renderer uses them).
 * Not written by vm3dgs_scene_save (quantise again after opening). */
int vm3dgs_scene_quantize_sh(vm3dgs_scene *s, int32_t n_codes, int32_t iters, int64_t n_train);

/* Device memory the caller must provide for a renderer. */
/* fp16_pool selects the record: 0 fp32, 1 fp16, 2 VQ (E_STATE if the scene
 * lacks it) */
int vm3dgs_pool_slot_bytes(const vm3dgs_scene *s, int32_t fp16_pool, int64_t *out);
int vm3dgs_scratch_bytes(const vm3dgs_scene *s, const vm3dgs_params *p, int64_t pool_bytes, int64_t *out);

/* Creates a renderer over caller-owned device memory: pool (whole slots of
 * vm3dgs_pool_slot_bytes each) and scratch (vm3dgs_scratch_bytes).  Makes the
 * scene's host pages readable by the GPU (page-locks them) on first use.
 * Clears the page table; returns E_CAPACITY if the pool holds no slot. */
int vm3dgs_renderer_create(const vm3dgs_scene *s, const vm3dgs_params *p, void *pool_dev, int64_t pool_bytes,
                           void *scratch_dev, int64_t scratch_bytes, void *stream, vm3dgs_renderer **out);
void vm3dgs_renderer_destroy(vm3dgs_renderer *r);

/* Page determination (Sec. 4.1): rasterises the proxy with per-face page
 * IDs into the low-resolution visibility buffer of each camera and reduces
 * it to one word per page, the maximum over its pixels (and over pixels of
 * pages linking to it) of a code that decreases with depth. */
int vm3dgs_render_feedback(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams, void *stream);

/* Requests every page at level 0 with the nearest depth (the no-virtual-
 * memory reference, when the pool holds the scene). */
int vm3dgs_request_all(vm3dgs_renderer *r, void *stream);

/* Page-table update (Sec. 4.1 "Page Table Management"): compaction of the
 * request words, LOD choice by screen-space error, the two-stage table
 * update with LRU replacement within the staging budget, the copy of the
 * new pages from host memory into the pool on copy_stream (which may equal
 * stream; the render on stream waits for it), and the LOD controller. */
int vm3dgs_update_residency(vm3dgs_renderer *r, void *stream, void *copy_stream);

/* Renders the resident, required Gaussians (Sec. 4.2) for each camera into
 * images[v], a caller-owned device float array [3][height][width] (CHW):
 * projection + SH colour, tile binning, (tile, depth) radix sort, tile
 * ranges, front-to-back blending. */
int vm3dgs_render(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams, float *const *images, void *stream);

/* Many views at once over the same resident pages (the union of their
 * requests was made resident by render_feedback on all of them): one
 * projection over (view, Gaussian), one pair sort over all views (the key's
 * tile field is a global tile id), one persistent blend over every (view,
 * tile) with each view's own tile shape.  n_cams <= max_views (<= 64). */
int vm3dgs_render_batched(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams, float *const *images,
                          void *stream);
/* Captures vm3dgs_render_batched for these views (their resolutions, tile
 * shapes and images) into a CUDA graph held by the renderer; stream must not
 * be the legacy default stream.  vm3dgs_batch_graph_launch replays it with
 * new camera poses (same count, sizes and tile shapes). */
int vm3dgs_batch_graph_capture(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams, float *const *images,
                               void *stream);
int vm3dgs_batch_graph_launch(vm3dgs_renderer *r, const vm3dgs_camera *cams, int32_t n_cams, void *stream);
/* Tile-shape autotuner: per resolution class (< 0.5, < 1, < 1.5, >= 1.5
 * megapixels) tries 16x16, 8x8 and 32x8 on the batch (median of `repeats`
 * timed runs), keeps the fastest, and writes the choice into cams[].tile_w /
 * tile_h.  Renders into images; synchronises stream. */
int vm3dgs_autotune_tiles(vm3dgs_renderer *r, vm3dgs_camera *cams, int32_t n_cams, float *const *images,
                          int32_t repeats, void *stream);

/* Copies the last frame's statistics (synchronises stream). */
int vm3dgs_get_stats(vm3dgs_renderer *r, vm3dgs_stats *out, void *stream);
/* Clears the running sums of the statistics (enqueued on stream). */
int vm3dgs_reset_sums(vm3dgs_renderer *r, void *stream);

/* Copies one device array of the renderer to host memory for inspection
 * (synchronises stream).  *needed receives the byte size of the array. */
enum {
  VM3DGS_DBG_FEEDBACK = 0,   /* uint64 [Hf][Wf] visibility buffer of the last feedback view */
  VM3DGS_DBG_REQ = 1,        /* uint32 [n_pages] request words */
  VM3DGS_DBG_DIRECT = 2,     /* uint8 [n_pages] */
  VM3DGS_DBG_REQUESTS = 3,   /* int32 [n][4] (page, enc, direct, level) request list */
  VM3DGS_DBG_PT_LOD = 4,     /* int32 [entries] */
  VM3DGS_DBG_PT_LAST = 5,    /* int32 [entries] */
  VM3DGS_DBG_PT_SLOT = 6,    /* int32 [entries][fanout^(levels-1)] */
  VM3DGS_DBG_COPIES = 7,     /* int32 [n][4] (page, level, entry, subslot), priority order */
  VM3DGS_DBG_DRAW = 8,       /* int32 [n][4] (page, level, entry, subslot), ascending page */
  VM3DGS_DBG_MISSING = 9,    /* int32 [n] ascending page */
  VM3DGS_DBG_SPLAT_RECT = 10,/* int32 [N][4] tile rectangle per drawn Gaussian (0s if culled) */
  VM3DGS_DBG_SPLAT_DEPTH = 11, /* float [N] view z (0 if culled) */
  VM3DGS_DBG_SPLAT_RADIUS = 12,/* float [N] (0 if culled) */
  VM3DGS_DBG_KEYS = 13,      /* uint64 [M] sorted keys of the last rendered view */
  VM3DGS_DBG_VALUES = 14,    /* uint32 [M] drawn-Gaussian index per sorted key */
  VM3DGS_DBG_RANGES = 15,    /* uint32 [tiles][2] */
  VM3DGS_DBG_SPLAT_XY = 16,  /* float [N][2] centre */
  VM3DGS_DBG_SPLAT_CONIC = 17, /* float [N][4] (A, B, C, opacity) */
  VM3DGS_DBG_SPLAT_RGB = 18, /* float [N][3] */
  VM3DGS_DBG_POOL = 19,      /* the pool bytes */
  VM3DGS_DBG_RASTER = 20,    /* uint32 [5] of the last feedback view: triangles queued for a warp, triangles left
                                in front of the near plane by the frustum test, huge triangles queued, their bands
                                of 4 rows, triangles crossing the near plane */
  VM3DGS_DBG_SPLAT_TMASK = 21, /* uint64 [N] the splat's tiles (those of its rectangle whose box of pixel centres
                                meets its 3-sigma ellipse, by the row rule of Sec. 4.2's tiled rendering reading) as
                                row-major bits of a rectangle of at most 64 tiles; 0 for larger rectangles and culled
                                splats */
  VM3DGS_DBG_SPLAT_TOUCHED = 22, /* uint32 [N] number of the splat's tiles (0 if culled) */
  VM3DGS_DBG_DRAW_W = 23        /* float [n_draw] opacity weight of each draw item (LOD cross-fade; else 1) */
};
int vm3dgs_debug_read(vm3dgs_renderer *r, int32_t what, void *host_dst, int64_t bytes, int64_t *needed, void *stream);

/* Per-stage GPU time.  When enabled, each stage of every later frame call is
 * bracketed by CUDA events on the stream it runs on, and its kernel launches
 * are counted.  vm3dgs_timing_read synchronises the device, adds the elapsed
 * milliseconds and launch counts of each stage since the last read into
 * ms_total[stage] and launches[stage] (arrays of n entries), and
 * forgets them (n <= 9).  Stages: */
enum {
  VM3DGS_STAGE_FEEDBACK = 0,  /* visibility buffer raster + reduction */
  VM3DGS_STAGE_RESIDENCY = 1, /* request compaction, LOD, page table, controller */
  VM3DGS_STAGE_STREAM = 2,    /* host -> pool page copies */
  VM3DGS_STAGE_PROJECT = 3,   /* gather + projection + SH */
  VM3DGS_STAGE_SCAN_EMIT = 4, /* tiles-touched scan, pair emission */
  VM3DGS_STAGE_SORT = 5,      /* radix sort passes over the pairs */
  VM3DGS_STAGE_RANGES = 6,    /* tile ranges and the tiles' processing order */
  VM3DGS_STAGE_BLEND = 7,     /* per-tile blending */
  VM3DGS_STAGE_PREFETCH = 8,  /* prefetch input, network, placement and copies */
  VM3DGS_STAGE_SORT_PREP = 9, /* reserved (the single-view sort's histograms are counted by the emission) */
  VM3DGS_N_STAGES = 10
};
int vm3dgs_timing_enable(vm3dgs_renderer *r, int32_t on);
int vm3dgs_timing_read(vm3dgs_renderer *r, double *ms_total, int64_t *launches, int32_t n);

/* ------------------------------------------------------------ prefetcher
 * A learned page prefetcher (the paper has none; its limitations, Sec. 4.3,
 * ask to copy earlier and with priorities).  Network: n_in inputs -> ReLU
 * n_hidden -> ReLU n_hidden -> n_out logits, one per page of a window of
 * n_out consecutive pages; bf16 weights and activations on the tensor cores,
 * FP32 accumulation, FP32 master weights and Adam state.  Device memory is
 * the caller's (vm3dgs_prefetcher_bytes). */
typedef struct vm3dgs_prefetcher vm3dgs_prefetcher;
typedef struct {
  int32_t n_in, n_hidden, n_out, max_batch;
  uint64_t seed;           /* weights U(-1/sqrt(fan_in), +1/sqrt(fan_in)) from SplitMix64(seed ^ index); biases 0 */
  float lr, beta1, beta2, eps;  /* Adam */
} vm3dgs_mlp_config;
enum { VM3DGS_PARAMS_GET = 0, VM3DGS_PARAMS_SET = 1, VM3DGS_PARAMS_GRAD = 2 };
int vm3dgs_prefetcher_bytes(const vm3dgs_mlp_config *c, int64_t *out);
int vm3dgs_prefetcher_create(const vm3dgs_mlp_config *c, void *dev, int64_t bytes, void *stream,
                             vm3dgs_prefetcher **out);
void vm3dgs_prefetcher_destroy(vm3dgs_prefetcher *p);
/* logits_dev[batch][n_out] = net(x_dev[batch][n_in]) (device pointers, fp32) */
int vm3dgs_prefetcher_forward(vm3dgs_prefetcher *p, const float *x_dev, int32_t batch, float *logits_dev, void *stream);
/* One Adam step on mean binary cross-entropy with logits over the entries
 * where mask = 1 (mask_sum = number of such entries); *loss_dev (optional)
 * receives the loss before the step.  Gradients stay readable until the next
 * step (VM3DGS_PARAMS_GRAD).  With lr = 0 no update is made. */
int vm3dgs_prefetcher_train_step(vm3dgs_prefetcher *p, const float *x_dev, const float *target_dev,
                                 const float *mask_dev, int32_t batch, float mask_sum, float *loss_dev, void *stream);
/* Host exchange of the packed fp32 parameters W1[n_in][h] b1 W2[h][h] b2
 * W3[h][n_out] b3 (GET / SET, SET also resets Adam) or of the last gradients
 * (GRAD).  n must equal the parameter count.  Synchronises stream. */
int vm3dgs_prefetcher_params(vm3dgs_prefetcher *p, int32_t what, float *host, int64_t n, void *stream);

/* Network input for the current frame, on the device: x_dev[0..11] = camera
 * position relative to the scene centre in units of the scene half-extent,
 * forward axis, velocity (position change since prev, in 1% of the half-
 * extent), change of the forward axis times 10; x_dev[12 + b] = fraction of
 * the 16 pages of window bin b requested by the last vm3dgs_render_feedback.
 * The window is the n_out pages centred, in page order, on the page whose
 * centroid is nearest the camera; its first page goes to *base_dev (device
 * int32, may be null).  prev may equal cam (no motion). */
int vm3dgs_prefetch_features(vm3dgs_renderer *r, int32_t n_out, const vm3dgs_camera *cam, const vm3dgs_camera *prev,
                             float *x_dev, int32_t *base_dev, void *stream);
/* Training targets from the last vm3dgs_render_feedback for a window:
 * y_dev[j] = 1 if page base + j was requested, else 0; mask_dev[j] = 1 if
 * base + j is a page of the scene, else 0 (base read from base_dev).  With
 * accumulate != 0, y_dev[j] becomes the OR (maximum) of its value and that
 * label, so calls over the frames of a horizon leave the pages requested in
 * any of them. */
int vm3dgs_prefetch_labels(vm3dgs_renderer *r, int32_t n_out, const int32_t *base_dev, float *y_dev, float *mask_dev,
                           int32_t accumulate, void *stream);
/* Prefetch for the next frame, after vm3dgs_render of this one: builds the
 * input as vm3dgs_prefetch_features does, runs the network, and spends the
 * staging budget this frame left unused on the window pages whose logit
 * exceeds threshold, highest first, that are neither requested this frame
 * nor resident at the level the screen-space-error rule gives for their
 * distance: they take entries not used this frame, least recently used first,
 * and are copied on copy_stream (the next vm3dgs_render waits for them). */
int vm3dgs_prefetch(vm3dgs_renderer *r, vm3dgs_prefetcher *p, const vm3dgs_camera *cam, const vm3dgs_camera *prev,
                    float threshold, void *stream, void *copy_stream);

/* ------------------------------------------------- sort without allocation
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory: a host application that reserves the device's
 * memory for itself and hands libraries only its own buffers, or a frame loop
 * that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * Sorts n (key, value) pairs in place, stably, by the low key_bits bits of the
 * keys (the renderer's onesweep radix sort), enqueued on stream.  keys_dev and
 * vals_dev are the caller's device arrays (input and output; they may be null
 * when n is 0).  Bits above key_bits are kept but do not order.  All scratch is
 * a fixed array inside the library (about 8.4 MB, held on every device that
 * loads the library until the process exits); n above
 * VM3DGS_NOALLOC_MAX_PAIRS is rejected with VM3DGS_E_CAPACITY before any
 * work.  Every call looks up the array's device address in the current
 * context (a host-side lookup once the library's module is loaded there; the
 * first call on a device loads it, so make that first call before any stream
 * capture and before time-critical use).  Every call shares the array and the
 * array keeps the last call's contents (each call clears what must start at
 * zero); calls that overlap on one device race.  A CUDA error left pending by
 * earlier work is reported as VM3DGS_E_CUDA before anything is enqueued (and
 * is not cleared).  If status_dev is not null it receives 0, VM3DGS_E_TIMEOUT
 * if a bounded wait of the sort gave up (the output is then not sorted), or
 * VM3DGS_E_CUDA if the call failed after enqueueing its first kernel.  Calls
 * no cudaMalloc, cudaFree or allocating library routine. */
#define VM3DGS_NOALLOC_MAX_PAIRS (1 << 19)
int vm3dgs_sort_pairs_noalloc(uint64_t *keys_dev, uint32_t *vals_dev, int64_t n, int32_t key_bits,
                              int32_t *status_dev, void *stream);

/* ------------------------------------------------ mesh proxy, host steps
 * The host steps of vm3dgs_build_pages with paging = 2, callable alone (no
 * GPU needed) to inspect or test them.
 * vm3dgs_mesh_simplify: quadric edge collapses (Sec. 3.1: "simplified using
 * a quadric error metric") of the mesh (verts [nv][3] FP64, tris [nt][3]) in
 * place, until at most target triangles live; the surviving vertices keep
 * their order, the triangles theirs; *nv_out, *nt_out the new counts.
 * vm3dgs_mesh_assign_pages: page assignment of Sec. 3.2 for n means (FP32
 * xyz): nearest triangle, subdivision of triangles holding more than
 * page_size, greedy merging.  Writes the subdivided mesh (verts_out up to
 * cap_v vertices, tris_out and face_page_out up to cap_t triangles), the
 * means in page order (order_out[n]), the pages' counts (counts_out, at
 * most n entries) and, if parent_out is not null, each page's parent (-1, or
 * for the extra pages of a triangle whose means splitting could not bring
 * within page_size -- 16 splits in a row that moved them all to one child --
 * the page that triangle carries; the build links them from it);
 * sizes_out[3] = vertices, triangles, pages (also when the caps are too
 * small: VM3DGS_E_CAPACITY).  E_INVAL for bad arrays. */
int vm3dgs_mesh_simplify(double *verts, int64_t nv, int32_t *tris, int64_t nt, int64_t target, int64_t *nv_out,
                         int64_t *nt_out);
int vm3dgs_mesh_assign_pages(int64_t n, const float *mu, int64_t page_size, const double *verts, int64_t nv,
                             const int32_t *tris, int64_t nt, int64_t cap_v, double *verts_out, int64_t cap_t,
                             int32_t *tris_out, int32_t *face_page_out, int64_t *order_out, int64_t *counts_out,
                             int64_t *parent_out, int64_t *sizes_out);

const char *vm3dgs_last_error(void);
const char *vm3dgs_version(void);

#ifdef __cplusplus
}
#endif
#endif
