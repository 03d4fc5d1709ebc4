// Tile binning and depth sort of the splats (Sec. 4.2: the paper sorts its
// index buffer globally by camera distance with a radix sort before drawing;
// here the sort key is (tile, depth) so each image tile receives its splats
// front to back, as in the tiled renderer of Kerbl et al.).
//
//   scan + emit   exclusive scan of tiles-touched per splat, then one
//                 (tile << 32 | float bits of depth, splat index) pair per
//                 (splat, tile of its rectangle), in ascending splat order.
//   onesweep      stable LSD radix sort, 8-bit digits, one pass per digit
//                 over the significant key bits: a histogram kernel counts
//                 every digit position at once, then each pass ranks a tile
//                 of keys in shared memory (warp match + per-warp counters),
//                 obtains its global digit offsets by decoupled look-back
//                 over predecessor tiles and scatters through shared memory.
//                 Every look-back wait is bounded: on expiry the kernel
//                 records VM3DGS_E_TIMEOUT in the control block and goes on.
//   ranges        [first, last+1) of every tile in the sorted keys.
// Stability plus ascending emission order gives the order (tile, depth,
// drawn index), and the drawn index ascends with the virtual Gaussian id.
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <unordered_set>

#include "coverage.cuh"
#include "renderer.cuh"

namespace vm {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = kScanItems / kScanThreads;   // 4
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kFlagMask = 3u << 30, kValMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookWindow = 8;  // look-back words read per round trip

__device__ __forceinline__ int64_t n_drawn(const Ctl *c, int64_t cap) { return c->r_drawn < cap ? c->r_drawn : cap; }
// splat records of all views (views x drawn)
__device__ __forceinline__ int64_t n_total(const Ctl *c, int64_t cap, int views) { return n_drawn(c, cap) * views; }

// exclusive scan across a 1024-thread block (64-bit); returns the block total in *total
__device__ uint64_t block_excl_scan_1024(uint64_t v, uint64_t *total) {
  __shared__ uint64_t warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  uint64_t wpre = warp == 0 ? 0 : warp_tot[warp - 1];
  *total = warp_tot[31];
  __syncthreads();
  return wpre + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const Ctl *ctl, const uint32_t *touched, int64_t ncap,
                                                                  int views, uint64_t *block_sums) {
  const int64_t N = n_total(ctl, ncap, views);
  const int64_t base = (int64_t)blockIdx.x * kScanItems;
  if (base >= N) return;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < N) s += touched[i];
  }
  uint64_t tot;
  block_excl_scan_1024(s, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// (also zeroes the n0 words at z0 and the n1 at z1: the emission's counters)
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(Ctl *ctl, int64_t ncap, int views,
                                                                  uint64_t *block_sums, uint32_t *z0, int n0,
                                                                  uint32_t *z1, int n1) {
  for (int i = threadIdx.x; i < n0; i += kScanThreads) z0[i] = 0;
  for (int i = threadIdx.x; i < n1; i += kScanThreads) z1[i] = 0;
  const int64_t N = n_total(ctl, ncap, views);
  const int64_t nb = (N + kScanItems - 1) / kScanItems;
  uint64_t carry = 0;
  for (int64_t c = 0; c < nb; c += kScanThreads) {
    int64_t i = c + threadIdx.x;
    uint64_t v = i < nb ? block_sums[i] : 0, tot;
    uint64_t ex = block_excl_scan_1024(v, &tot);
    if (i < nb) block_sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    ctl->pairs = (int64_t)carry;
    ctl->acc_pairs += (int64_t)carry;
    ctl->acc_views += views;
  }
}

// Per-splat exclusive pair offsets (saturated to 32 bits: offsets past the
// pair capacity are never written).
__global__ void __launch_bounds__(kScanThreads) scan_offsets_kernel(const Ctl *ctl, const uint32_t *touched,
                                                                   int64_t ncap, int views, const uint64_t *block_off,
                                                                   uint32_t *offsets) {
  const int64_t N = n_total(ctl, ncap, views);
  const int64_t base = (int64_t)blockIdx.x * kScanItems;
  if (base >= N) return;
  const int64_t i0 = base + (int64_t)threadIdx.x * kScanPer;
  uint32_t cnt[kScanPer];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    cnt[k] = (i0 + k < N) ? touched[i0 + k] : 0;
    s += cnt[k];
  }
  uint64_t tot;
  uint64_t off = block_off[blockIdx.x] + block_excl_scan_1024(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (i0 + k < N) offsets[i0 + k] = off < 0xFFFFFFFFull ? (uint32_t)off : 0xFFFFFFFFu;
    off += cnt[k];
  }
}

// Rectangle position (row-major) of the q-th covered tile of a splat whose
// rectangle has at most 64 tiles (m: its tile mask, q < popcount(m)): the
// q-th set bit, by halving the word with population counts.
__device__ __forceinline__ uint32_t covered_tile(uint64_t m, uint32_t q) {
  uint32_t pos = 0, x = (uint32_t)m, c = __popc(x);
  if (q >= c) {
    q -= c;
    pos = 32;
    x = (uint32_t)(m >> 32);
  }
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    c = __popc(x & ((1u << h) - 1u));
    if (q >= c) {
      q -= c;
      pos += (uint32_t)h;
      x >>= h;
    }
  }
  return pos;
}

// n / w for n < 64 and 1 <= w <= 64 by one multiply: with
// mag = ceil(2^16 / w), n * mag / 2^16 exceeds n / w by less than
// 64 / 2^16, below the gap 1/w between n / w and the next integer
__device__ __forceinline__ uint32_t div_small(uint32_t n, uint32_t mag) { return (n * mag) >> 16; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Where a splat's pairs go: its view's image and tile size, the view's first
// global tile and its tiles per row.  One view (vt null): g and gx; a batch:
// splat record i belongs to view i / nv of the device table.
struct EmitViews {
  const ViewTable *vt;
  TileGeom g;
  int gx;
  __device__ __forceinline__ void of(int64_t i, int64_t nv, TileGeom &tg, int &tgx, int &toff) const {
    if (!vt) {
      tg = g;
      tgx = gx;
      toff = 0;
      return;
    }
    const int v = (int)(i / nv);
    const vm3dgs_camera &c = vt->cam[v];
    tg = TileGeom{c.width, c.height, c.tile_w, c.tile_h};
    tgx = vt->gx[v];
    toff = vt->tile_off[v];
  }
};

// adds n to the depth-field digits 0 .. dpass-1 of the shifted key kd
__device__ __forceinline__ void count_run(uint32_t (*hs)[256], uint64_t kd, int dpass, uint32_t n) {
  for (int d = 0; d < dpass; ++d) atomicAdd(&hs[d][(kd >> (8 * d)) & 255u], n);
}

// What the emission writes per pair: the packed key (and value), and the
// sort's digit counts in the CTA's shared-memory histograms.
struct PairOut {
  uint64_t *keys;
  uint32_t *vals;
  int64_t M;
  KeyFormat kf;
  uint32_t (*hs)[256];
  bool hist;
  int lo_bit, passes, dpass;  // digits 0 .. dpass-1 lie in the depth field (counted once per splat)
  // (valid: this lane has a pair)
  __device__ __forceinline__ void put(bool valid, int64_t j, uint32_t tile, uint64_t dkey, uint32_t i) const {
    const uint64_t key = ((uint64_t)tile << kf.tshift) | dkey;
    if (valid && j < M) {
      if (kf.packed) {
        keys[j] = key | (uint64_t)i;
      } else {
        keys[j] = key;
        vals[j] = i;
      }
    }
    if (hist && valid) {
      const uint64_t kd = key >> lo_bit;
      for (int d = dpass; d < passes; ++d) atomicAdd(&hs[d][(kd >> (8 * d)) & 255u], 1u);
    }
  }
};

__device__ __forceinline__ PairOut pair_out(const Ctl *ctl, uint64_t *keys, uint32_t *vals, int64_t pair_cap,
                                            const KeyFormat &kf, const SortHist &sh, uint32_t (*hs)[256]) {
  PairOut po;
  po.keys = keys;
  po.vals = vals;
  po.M = ctl->pairs < pair_cap ? ctl->pairs : pair_cap;
  po.kf = kf;
  po.hs = hs;
  po.hist = sh.hist != nullptr;
  po.lo_bit = sh.lo_bit;
  po.passes = sh.passes;
  po.dpass = po.hist ? max(0, min(sh.passes, (kf.tshift - sh.lo_bit) / 8)) : 0;
  return po;
}

// the depth field of a splat's keys (its view depth's bits above 0.2f, clamped)
__device__ __forceinline__ uint64_t depth_key(uint32_t db, const KeyFormat &kf) {
  const uint64_t dmax = (1ull << kf.R) - 1ull;
  return min((uint64_t)(db >= kf.base ? db - kf.base : 0u), dmax) << kf.ib;
}

__device__ __forceinline__ void hist_flush(const SortHist &sh, uint32_t (*hs)[256]) {
  __syncthreads();
  for (int i2 = threadIdx.x; i2 < sh.passes * 256; i2 += blockDim.x) {
    const uint32_t v2 = (&hs[0][0])[i2];
    if (v2) atomicAdd(&sh.hist[i2], v2);
  }
}

constexpr uint32_t kSmallSplat = 32;  // pairs a splat may have to be dealt out with others
constexpr uint32_t kPiece = 256;      // pairs per piece of a larger splat

// Pairs [qa, qb) of splat i whose rectangle has more than 64 tiles, by the
// whole warp: its rows are walked 32 at a time (a lane per row computes the
// row's run of kept columns, a warp scan gives the rows' first pairs, and each
// pair in those rows finds its row by a binary search over the scan).
__device__ __forceinline__ void emit_rows(const PairOut &po, const SplatEllipse &el, int x0, int x1, int y0, int y1,
                                          uint32_t qa, uint32_t qb, uint32_t off, uint64_t dkey, uint32_t i,
                                          const TileGeom &tg, int tgx, int toff, int lane) {
  uint32_t base = 0;  // pairs in the rows before this group of 32
  for (int r0 = y0; r0 < y1 && base < qb; r0 += 32) {
    const int ty = r0 + lane;
    const int2 sp2 = ty < y1 ? row_span(el, ty, x0, x1, tg) : make_int2(0, 0);
    const uint32_t nr = sp2.y > sp2.x ? (uint32_t)(sp2.y - sp2.x) : 0u;
    uint32_t incl = nr;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += o;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t lo = max(qa, base), hi = min(qb, base + tot);
    for (uint32_t g0 = lo; g0 < hi; g0 += 32) {
      const uint32_t q = g0 + (uint32_t)lane, rel = q - base;
      // row: the number of rows whose inclusive count is <= rel
      int L = 0;
#pragma unroll
      for (int st = 16; st >= 1; st >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, incl, L + st - 1);
        if (v <= rel) L += st;
      }
      L = min(L, 31);
      const uint32_t Li = __shfl_sync(0xffffffffu, incl, L), Ln = __shfl_sync(0xffffffffu, nr, L);
      const int Lc0 = __shfl_sync(0xffffffffu, sp2.x, L);
      po.put(q < hi, (int64_t)off + q, (uint32_t)(toff + (r0 + L) * tgx + Lc0 + (int)(rel - (Li - Ln))), dkey, i);
    }
    base += tot;
  }
}

// Pair emission (pairs of a splat: its kept tiles in row-major order, at its
// scanned offset), part 1: a warp takes 32 consecutive splats, a lane each,
// with coalesced loads of their records.  The pairs of the splats with at
// most 32 of them are dealt out to the lanes together (lane g of a round
// writes pair g of the concatenation, its splat found by a binary search over
// the lanes' inclusive counts and its record fetched by shuffles), so stores
// are contiguous and no lane walks the offsets; a pair's tile comes from the
// splat's tile mask.  A splat of at most 32 pairs whose rectangle has more
// than 64 tiles (no mask) has its rows walked by the whole warp (emit_rows).
// Larger splats are cut into pieces of kPiece pairs, listed for part 2.
// Digits that lie in the depth field are
// the same for all pairs of a splat and are counted once per splat.  With
// sh.hist the kernel also counts the sort's digits (shared-memory histograms
// merged into sh.hist) and clears the sort's look-back words and tile
// counters.  A batch (ev.vt) emits the records of all its views.
__global__ void __launch_bounds__(256, 4) emit_kernel(const Ctl *ctl, Splats sp, int64_t ncap, int views, EmitViews ev,
                                                   const uint32_t *offsets, uint64_t *keys, uint32_t *vals,
                                                   int64_t pair_cap, KeyFormat kf, SortHist sh, uint64_t *pieces,
                                                   uint32_t *piece_ctr, int64_t piece_cap, uint2 *ranges, int ntiles) {
  __shared__ uint32_t hs[kMaxPasses][256];
  if (sh.hist) {
    for (int i = threadIdx.x; i < sh.passes * 256; i += blockDim.x) (&hs[0][0])[i] = 0;
    __syncthreads();
  }
  const PairOut po = pair_out(ctl, keys, vals, pair_cap, kf, sh, hs);
  const int64_t Nv = n_drawn(ctl, ncap);
  const int64_t N = Nv * views;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // a task's records are loaded together (one round trip, culled splats
  // included) and the next task's while this one is dealt out
  struct Rec {
    uint32_t cnt, off, rx, ry, db;
    uint64_t tm;
  };
  auto load = [&](int64_t i) {
    Rec q{0u, 0u, 0u, 0u, 0u, 0ull};
    if (i < N) {
      q.cnt = sp.touched[i];
      q.off = offsets[i];
      q.rx = sp.rect[2 * i];
      q.ry = sp.rect[2 * i + 1];
      q.tm = sp.tmask[i];
      q.db = sp.depth[i];
    }
    return q;
  };
  Rec nx = load(warp0 * 32 + lane);
  for (int64_t b = warp0 * 32; b < N; b += nwarps * 32) {
    const int64_t i = b + lane;
    const Rec cur = nx;
    nx = load(b + nwarps * 32 + lane);
    const uint32_t cnt = cur.cnt;
    uint32_t off = 0, rx = 0, ry = 0;
    uint64_t tm = 0, dkey = 0;
    // dealt out here: splats of at most 32 pairs whose tiles the mask lists;
    // those of at most 32 pairs in a rectangle of more than 64 tiles (no
    // mask) are walked by the warp together below; larger ones are pieces
    const uint32_t rw = (cur.rx >> 16) - (cur.rx & 0xFFFFu), rh = (cur.ry >> 16) - (cur.ry & 0xFFFFu);
    const bool big = cnt > kSmallSplat;
    const bool rows = cnt && !big && rw * rh > 64u;
    uint32_t mag = 0;
    if (cnt && !big && !rows) {
      off = cur.off;
      rx = cur.rx;
      ry = cur.ry;
      tm = cur.tm;
      mag = (65536u + rw - 1u) / rw;
      dkey = depth_key(cur.db, kf);
      if (po.hist) count_run(hs, dkey >> po.lo_bit, po.dpass, cnt);
    }
    const uint32_t small = (big || rows) ? 0u : cnt;
    uint32_t incl = small;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += o;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t g0 = 0; g0 < total; g0 += 32) {
      const uint32_t g = g0 + (uint32_t)lane;
      // owner: the number of lanes whose inclusive count is <= g
      int L = 0;
#pragma unroll
      for (int st = 16; st >= 1; st >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, incl, L + st - 1);
        if (v <= g) L += st;
      }
      L = min(L, 31);
      const uint32_t Li = __shfl_sync(0xffffffffu, incl, L), Ln = __shfl_sync(0xffffffffu, small, L);
      const uint32_t Lrx = __shfl_sync(0xffffffffu, rx, L), Lry = __shfl_sync(0xffffffffu, ry, L);
      const uint64_t Ltm = __shfl_sync(0xffffffffu, tm, L), Ld = __shfl_sync(0xffffffffu, dkey, L);
      const uint32_t Loff = __shfl_sync(0xffffffffu, off, L), Lmag = __shfl_sync(0xffffffffu, mag, L);
      const bool valid = g < total;
      const int64_t si = b + L;
      const uint32_t q = g - (Li - Ln);
      const uint32_t x0 = Lrx & 0xFFFFu, w = (Lrx >> 16) - x0, y0 = Lry & 0xFFFFu;
      TileGeom tg;
      int tgx, toff;
      ev.of(si, Nv, tg, tgx, toff);
      const uint32_t qt = valid ? covered_tile(Ltm, q) : 0u;
      const uint32_t dy = div_small(qt, Lmag);
      const uint32_t tx = x0 + (qt - dy * w), ty = y0 + dy;
      po.put(valid, (int64_t)Loff + q, (uint32_t)toff + ty * (uint32_t)tgx + tx, Ld, (uint32_t)si);
    }
    // splats of a few pairs in a large rectangle: the warp walks each one's rows
    for (uint32_t m = __ballot_sync(0xffffffffu, rows); m; m &= m - 1u) {
      const int L = __ffs(m) - 1;
      const int64_t si = b + L;
      const uint32_t Lrx = __shfl_sync(0xffffffffu, cur.rx, L), Lry = __shfl_sync(0xffffffffu, cur.ry, L);
      const uint32_t Lcnt = __shfl_sync(0xffffffffu, cnt, L), Loff = __shfl_sync(0xffffffffu, cur.off, L);
      const uint64_t Ld = depth_key(__shfl_sync(0xffffffffu, cur.db, L), kf);
      if (po.hist && lane == L) count_run(hs, Ld >> po.lo_bit, po.dpass, Lcnt);
      TileGeom tg;
      int tgx, toff;
      ev.of(si, Nv, tg, tgx, toff);
      const float4 s0 = sp.rec[3 * si];
      const SplatEllipse el = splat_ellipse(s0.x, s0.y, s0.z, s0.w, sp.rec[3 * si + 1].x);
      emit_rows(po, el, (int)(Lrx & 0xFFFFu), (int)(Lrx >> 16), (int)(Lry & 0xFFFFu), (int)(Lry >> 16), 0u, Lcnt, Loff,
                Ld, (uint32_t)si, tg, tgx, toff, lane);
    }
    // larger splats: their pieces to the list (one reservation per warp)
    const uint32_t np = big ? (cnt + kPiece - 1) / kPiece : 0u;
    uint32_t pincl = np;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, pincl, d);
      if (lane >= d) pincl += o;
    }
    const uint32_t ptotal = __shfl_sync(0xffffffffu, pincl, 31);
    if (ptotal) {
      uint32_t pb = 0;
      if (lane == 0) pb = atomicAdd(piece_ctr, ptotal);
      pb = __shfl_sync(0xffffffffu, pb, 0);
      for (uint32_t k = 0; k < np; ++k) {
        const int64_t slot = (int64_t)pb + (pincl - np) + k;
        if (slot < piece_cap) pieces[slot] = ((uint64_t)i << 32) | k;
      }
    }
  }
  if (sh.hist) {
    hist_flush(sh, hs);
    // the look-back words and tile counters of the coming sort
    const int64_t ntiles = (po.M + kSortTile - 1) / kSortTile;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int d = 0; d < sh.passes && sh.lookback; ++d) {
      uint32_t *lb = sh.lookback + (int64_t)d * sh.max_tiles * 256;
      for (int64_t q2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q2 < ntiles * 256; q2 += stride) lb[q2] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < kMaxPasses) sh.tile_ctr[threadIdx.x] = 0;
  }
  // the tile ranges, written only for tiles with pairs, start empty
  for (int64_t q2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q2 < ntiles; q2 += (int64_t)gridDim.x * blockDim.x)
    ranges[q2] = make_uint2(0u, 0u);
}

// Pair emission, part 2: a warp per piece of kPiece pairs of a larger splat.
// A rectangle of at most 64 tiles reads its tile mask; a larger one has its
// rows walked by the warp (emit_rows).
__global__ void __launch_bounds__(256) emit_pieces_kernel(const Ctl *ctl, Splats sp, int64_t ncap, EmitViews ev,
                                                          const uint32_t *offsets, uint64_t *keys, uint32_t *vals,
                                                          int64_t pair_cap, KeyFormat kf, SortHist sh,
                                                          const uint64_t *pieces, const uint32_t *piece_ctr,
                                                          int64_t piece_cap) {
  __shared__ uint32_t hs[kMaxPasses][256];
  if (sh.hist) {
    for (int i = threadIdx.x; i < sh.passes * 256; i += blockDim.x) (&hs[0][0])[i] = 0;
    __syncthreads();
  }
  const PairOut po = pair_out(ctl, keys, vals, pair_cap, kf, sh, hs);
  const int64_t Nv = n_drawn(ctl, ncap);
  const int64_t n = min((int64_t)*piece_ctr, piece_cap);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp0; p < n; p += nwarps) {
    const uint64_t e = pieces[p];
    const int64_t i = (int64_t)(e >> 32);
    const uint32_t k = (uint32_t)e;
    const uint32_t cnt = sp.touched[i], off = offsets[i];
    const uint32_t rx = sp.rect[2 * i], ry = sp.rect[2 * i + 1];
    const uint64_t dkey = depth_key(sp.depth[i], kf);
    if (po.hist && k == 0 && lane == 0) count_run(hs, dkey >> po.lo_bit, po.dpass, cnt);
    const int x0 = (int)(rx & 0xFFFFu), x1 = (int)(rx >> 16), y0 = (int)(ry & 0xFFFFu), y1 = (int)(ry >> 16);
    const int w = x1 - x0;
    TileGeom tg;
    int tgx, toff;
    ev.of(i, Nv, tg, tgx, toff);
    const uint32_t qa = k * kPiece, qb = min(cnt, qa + kPiece);
    if (w * (y1 - y0) <= 64) {
      const uint64_t tm = sp.tmask[i];
      const uint32_t mag = (65536u + (uint32_t)w - 1u) / (uint32_t)w;
      for (uint32_t q0 = qa; q0 < qb; q0 += 32) {
        const uint32_t q = q0 + (uint32_t)lane;
        const bool valid = q < qb;
        const uint32_t qt = valid ? covered_tile(tm, q) : 0u;
        const uint32_t dy = div_small(qt, mag);
        po.put(valid, (int64_t)off + q, (uint32_t)(toff + (y0 + (int)dy) * tgx + x0 + (int)(qt - dy * (uint32_t)w)), dkey,
               (uint32_t)i);
      }
      continue;
    }
    const float4 s0 = sp.rec[3 * i];
    const SplatEllipse el = splat_ellipse(s0.x, s0.y, s0.z, s0.w, sp.rec[3 * i + 1].x);
    emit_rows(po, el, x0, x1, y0, y1, qa, qb, off, dkey, (uint32_t)i, tg, tgx, toff, lane);
  }
  if (sh.hist) hist_flush(sh, hs);
}

// ------------------------------------------------------------------ onesweep
// (the last pass's digit holds the bits left below hi_bit: last_mask)
__global__ void __launch_bounds__(256) sort_hist_kernel(const Ctl *ctl, const uint64_t *keys, int64_t cap, int lo_bit,
                                                        int passes, uint32_t last_mask, uint32_t *hist,
                                                        uint32_t *lookback, int64_t max_tiles, uint32_t *tile_ctr) {
  __shared__ uint32_t h[kMaxPasses][256];
  const int64_t M = ctl->pairs < cap ? ctl->pairs : cap;
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
    const uint64_t k = keys[j] >> lo_bit;
    for (int d = 0; d < passes; ++d) atomicAdd(&h[d][(k >> (8 * d)) & (d == passes - 1 ? last_mask : 255u)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
    uint32_t v = (&h[0][0])[i];
    if (v) atomicAdd(&hist[i], v);
  }
  // clear the look-back words this sort will use (pass d owns words
  // [d * max_tiles * 256, +ntiles * 256)), and the tile counters
  const int64_t ntiles = (M + kSortTile - 1) / kSortTile;
  for (int d = 0; d < passes; ++d) {
    uint32_t *lb = lookback + (int64_t)d * max_tiles * 256;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ntiles * 256; j += stride) lb[j] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x < kMaxPasses) tile_ctr[threadIdx.x] = 0;
}

// Lanes of the warp holding the same digit as this lane (d < 0: an empty
// slot, in no lane's set): the AND of the eight ballots on the digit's bits
// (a warp multisplit, cheaper here than the match instruction).
__device__ __forceinline__ uint32_t digit_peers(int d) {
  uint32_t peers = __ballot_sync(0xffffffffu, d >= 0);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const bool bit = (d >> j) & 1;
    const uint32_t bj = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bj : ~bj;
  }
  return peers;
}

// one radix digit per thread: the digit scans and count loads index by tid
static_assert(kSortThreads == 256, "onesweep assumes one thread per 8-bit digit");

template <bool VALS>
__global__ void __launch_bounds__(kSortThreads, 4) onesweep_kernel(Ctl *ctl, const uint64_t *kin, const uint32_t *vin,
                                                                uint64_t *kout, uint32_t *vout, int64_t cap, int shift,
                                                                uint32_t dmask, const uint32_t *counts,
                                                                uint32_t *status, uint32_t *tile_ctr) {
  constexpr int W = kSortThreads / 32;
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *s_keys = reinterpret_cast<uint64_t *>(smem);
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + kSortTile);
  uint32_t *s_wc = s_vals + kSortTile;          // [W][256]
  uint32_t *s_doff = s_wc + W * 256;            // [256]
  uint32_t *s_glob = s_doff + 256;              // [256]
  __shared__ int64_t s_tile;
  __shared__ uint32_t s_scan[W];
  const int64_t M = ctl->pairs < cap ? ctl->pairs : cap;
  const int64_t ntiles = (M + kSortTile - 1) / kSortTile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  // global offset of digit tid: exclusive scan of the pass's digit counts
  uint32_t dbase;
  {
    const uint32_t c = counts[tid];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_scan[w];
    dbase = wpre + x - c;
    __syncthreads();
  }
  for (;;) {
    if (tid == 0) s_tile = (int64_t)atomicAdd(tile_ctr, 1u);
    for (int i = tid; i < W * 256; i += kSortThreads) s_wc[i] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t t0 = tile * kSortTile;
    uint64_t k[kSortItems];
    uint32_t v[kSortItems], rk[kSortItems];
    int dg[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const int64_t idx = t0 + (int64_t)warp * 32 * kSortItems + it * 32 + lane;
      const bool valid = idx < M;
      k[it] = valid ? kin[idx] : 0ull;
      v[it] = (VALS && valid) ? vin[idx] : 0u;
      dg[it] = valid ? (int)((k[it] >> shift) & dmask) : -1;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      // (the match instruction: the pairs of a splat share their depth
      // digits, so groups are large and it is cheaper here than ballots)
      const int d = dg[it];
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = 0;
      if (d >= 0) before = s_wc[warp * 256 + d];
      rk[it] = before + __popc(peers & lt);
      __syncwarp();
      if (d >= 0 && (peers & lt) == 0) s_wc[warp * 256 + d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, tile count
    uint32_t cnt = 0;
    for (int w = 0; w < W; ++w) {
      const uint32_t c = s_wc[w * 256 + tid];
      s_wc[w * 256 + tid] = cnt;
      cnt += c;
    }
    volatile uint32_t *st = status + tile * 256 + tid;
    *st = (tile == 0 ? kFlagInc : kFlagAgg) | cnt;
    // tile-local exclusive scan of the digit counts
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_scan[w];
    s_doff[tid] = wpre + x - cnt;
    __syncthreads();
    // the tile in digit order in shared memory (its keys leave the registers
    // before the look-back)
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const int d = dg[it];
      if (d < 0) continue;
      const uint32_t pos = s_doff[d] + s_wc[warp * 256 + d] + rk[it];
      s_keys[pos] = k[it];
      if (VALS) s_vals[pos] = v[it];
    }
    // decoupled look-back, kLookWindow predecessors per round trip: the
    // words of tiles j, j-1, .. are read together and summed from the nearest
    // until an inclusive one (done) or one not yet published (read again from
    // there next round)
    uint32_t excl = 0;
    if (tile > 0) {
      int64_t j = tile - 1;
      int spins = 0;
      for (;;) {
        uint32_t w[kLookWindow];
#pragma unroll
        for (int i = 0; i < kLookWindow; ++i)
          w[i] = j - i >= 0 ? *(const volatile uint32_t *)(status + (j - i) * 256 + tid) : 0u;
        int used = 0;
        bool inc = false;
#pragma unroll
        for (int i = 0; i < kLookWindow; ++i) {
          if (used != i || inc) break;
          const uint32_t f = w[i] & kFlagMask;
          if (f == 0) break;
          excl += w[i] & kValMask;
          ++used;
          inc = f == kFlagInc;
        }
        if (inc) break;
        j -= used;
        if (used == 0) {
          if (++spins > kSpinLimit) {
            atomicCAS(&ctl->status, 0, VM3DGS_E_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
      }
      *st = kFlagInc | ((excl + cnt) & kValMask);
    }
    s_glob[tid] = dbase + excl;
    __syncthreads();
    const int nvalid = (int)((M - t0) < kSortTile ? (M - t0) : kSortTile);
    for (int i = tid; i < nvalid; i += kSortThreads) {
      const uint64_t key = s_keys[i];
      const int d = (int)((key >> shift) & dmask);
      const uint32_t o = s_glob[d] + (uint32_t)i - s_doff[d];
      if ((int64_t)o < M) {  // always true unless a look-back wait timed out
        kout[o] = key;
        if (VALS) vout[o] = s_vals[i];
      }
    }
    __syncthreads();
  }
}


// ------------------------------------------------------------ cooperative sort
// All passes of the LSD radix sort in one cooperative launch: CTA b owns the
// fixed chunk [b c, (b + 1) c) of the pairs (c = ceil(M / G)), and each pass
// runs in three phases separated by grid barriers:
//   count   the chunk's digit histogram -> column b of colhist[256][G]
//   scan    CTA d (d < 256) scans digit d's column over the CTAs into the
//           global output offsets offs[d][b] = (pairs with a smaller digit,
//           from the pass's digit histogram counted by the emission) + (pairs
//           of digit d in earlier chunks)
//   scatter the chunk, in sub-tiles of kCoopTile pairs in order, ranked
//           stably (warp multisplit by ballots + per-warp digit counters taken
//           by one shared atomic per digit group; otherwise as in the onesweep
//           pass) and written through shared memory to offs + the digit's
//           running count in the chunk.
// No look-back chain and one launch for all passes: the pass costs two reads
// and one write of the keys (in L2 at these sizes) and three barriers.  Each
// barrier wait is bounded: on expiry the kernel sets an error word that every
// CTA checks, records VM3DGS_E_TIMEOUT and returns (writes stay in bounds:
// every scatter checks its position against the pair count).
constexpr int kCoopThreads = 512;
constexpr int kCoopWarps = kCoopThreads / 32;
constexpr int kCoopItems = 8;
constexpr int kCoopTile = kCoopThreads * kCoopItems;
constexpr int kCoopMaxGrid = kCoopThreads;  // the column scan holds one CTA per thread
constexpr uint32_t kBarrierSpins = 1u << 22;

struct CoopSortArgs {
  Ctl *ctl;
  uint64_t *keys[2];
  uint32_t *vals[2];
  int64_t cap;
  int lo_bit, passes;
  uint32_t last_mask;
  const uint32_t *hist;  // [passes][256] digit counts of all pairs
  uint32_t *colhist;     // [256][G]
  uint32_t *offs;        // [256][G]
  uint32_t *bar;         // [0] barrier arrivals, [1] error word (both zero at launch)
};

// exclusive scan of one value per thread over the 512-thread block; *total
// gets the block's sum
__device__ __forceinline__ uint32_t coop_block_scan(uint32_t v, uint32_t *total, uint32_t *s_scan) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_scan[warp] = x;
  __syncthreads();
  uint32_t wpre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kCoopWarps; ++w) {
    const uint32_t t = s_scan[w];
    if (w < warp) wpre += t;
    tot += t;
  }
  __syncthreads();
  *total = tot;
  return wpre + x - v;
}

// Grid barrier: every CTA arrives once per call; returns false (in every
// thread) when the bounded wait expired or another CTA reported an error.
__device__ __forceinline__ bool coop_grid_sync(uint32_t *bar, uint32_t target, int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(&bar[0], 1u);
    uint32_t spins = 0;
    for (;;) {
      if (*(volatile uint32_t *)&bar[1]) {
        ok = 0;
        break;
      }
      if (*(volatile uint32_t *)&bar[0] >= target) break;
      if (++spins > kBarrierSpins) {
        atomicExch(&bar[1], 1u);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

template <bool VALS>
__global__ void __launch_bounds__(kCoopThreads, 2) coop_sort_kernel(CoopSortArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *s_keys = reinterpret_cast<uint64_t *>(smem);
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + kCoopTile);
  uint32_t *s_wc = s_vals + (VALS ? kCoopTile : 0);  // [kCoopWarps][256]
  __shared__ uint32_t s_hist[256], s_base[256], s_run[256], s_doff[256], s_cnt[256], s_scan[kCoopWarps];
  __shared__ int s_ok;
  const int64_t M = a.ctl->pairs < a.cap ? a.ctl->pairs : a.cap;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  const int64_t c = (M + G - 1) / G;
  const int64_t lo = min(M, (int64_t)b * c), hi = min(M, lo + c);
  uint32_t nbar = 0;
  bool ok = true;
  for (int p = 0; p < a.passes && ok; ++p) {
    const bool odd = p & 1;  // (selects, not indexing: the parameter arrays stay in registers)
    const uint64_t *kin = odd ? a.keys[1] : a.keys[0];
    uint64_t *kout = odd ? a.keys[0] : a.keys[1];
    const uint32_t *vin = odd ? a.vals[1] : a.vals[0];
    uint32_t *vout = odd ? a.vals[0] : a.vals[1];
    const int shift = a.lo_bit + 8 * p;
    const uint32_t dmask = p == a.passes - 1 ? a.last_mask : 255u;
    // ---- count (eight independent loads per thread in flight; the first
    // sub-tile is loaded as the scatter reads it and kept in registers)
    for (int d = tid; d < 256; d += kCoopThreads) s_hist[d] = 0;
    __syncthreads();
    {
      uint64_t k0[kCoopItems];
#pragma unroll
      for (int it = 0; it < kCoopItems; ++it) {
        const int64_t idx = lo + (int64_t)warp * 32 * kCoopItems + it * 32 + lane;
        k0[it] = idx < hi ? kin[idx] : 0ull;
      }
#pragma unroll
      for (int it = 0; it < kCoopItems; ++it) {
        // parked where the scatter's first sub-tile reads it (s_keys is free until then)
        s_keys[warp * 32 * kCoopItems + it * 32 + lane] = k0[it];
        if (lo + (int64_t)warp * 32 * kCoopItems + it * 32 + lane < hi) atomicAdd(&s_hist[(k0[it] >> shift) & dmask], 1u);
      }
    }
    for (int64_t t0 = lo + kCoopTile; t0 < hi; t0 += kCoopTile) {
      uint32_t dd[kCoopItems];
#pragma unroll
      for (int it = 0; it < kCoopItems; ++it) {
        const int64_t idx = t0 + (int64_t)it * kCoopThreads + tid;
        dd[it] = idx < hi ? (uint32_t)((kin[idx] >> shift) & dmask) : 0xFFFFFFFFu;
      }
#pragma unroll
      for (int it = 0; it < kCoopItems; ++it)
        if (dd[it] != 0xFFFFFFFFu) atomicAdd(&s_hist[dd[it]], 1u);
    }
    __syncthreads();
    for (int d = tid; d < 256; d += kCoopThreads) a.colhist[(int64_t)d * G + b] = s_hist[d];
    if (!(ok = coop_grid_sync(a.bar, ++nbar * (uint32_t)G, &s_ok))) break;
    // ---- scan: digit d's column, by CTA d (and d + G, ... when G < 256)
    for (int d = b; d < 256; d += G) {
      uint32_t tot;
      const uint32_t below = coop_block_scan(tid < 256 && tid < d ? a.hist[p * 256 + tid] : 0u, &tot, s_scan);
      (void)below;
      const uint32_t base = tot;  // pairs with a digit below d
      const uint32_t x = tid < G ? a.colhist[(int64_t)d * G + tid] : 0u;
      const uint32_t ex = coop_block_scan(x, &tot, s_scan);
      if (tid < G) a.offs[(int64_t)d * G + tid] = base + ex;
    }
    if (!(ok = coop_grid_sync(a.bar, ++nbar * (uint32_t)G, &s_ok))) break;
    // ---- scatter
    for (int d = tid; d < 256; d += kCoopThreads) {
      s_base[d] = a.offs[(int64_t)d * G + b];
      s_run[d] = 0;
    }
    for (int64_t t0 = lo; t0 < hi; t0 += kCoopTile) {
      for (int i = tid; i < kCoopWarps * 256; i += kCoopThreads) s_wc[i] = 0;
      __syncthreads();
      uint64_t k[kCoopItems];
      uint32_t v[kCoopItems], rk[kCoopItems];
      int dg[kCoopItems];
#pragma unroll
      for (int it = 0; it < kCoopItems; ++it) {
        const int64_t idx = t0 + (int64_t)warp * 32 * kCoopItems + it * 32 + lane;
        const bool valid = idx < hi;
        k[it] = t0 == lo ? s_keys[warp * 32 * kCoopItems + it * 32 + lane] : (valid ? kin[idx] : 0ull);
        v[it] = (VALS && valid) ? vin[idx] : 0u;
        dg[it] = valid ? (int)((k[it] >> shift) & dmask) : -1;
      }
#pragma unroll
      for (int it = 0; it < kCoopItems; ++it) {
        const int d = dg[it];
        // the lowest lane of each digit group takes the group's places from the
        // warp's counter (a shared atomic returns the places taken before it)
        const uint32_t peers = digit_peers(d);
        const int leader = peers ? __ffs(peers) - 1 : lane;
        uint32_t old = 0;
        if (d >= 0 && leader == lane) old = atomicAdd(&s_wc[warp * 256 + d], (uint32_t)__popc(peers));
        rk[it] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
      }
      __syncthreads();
      // per digit: exclusive prefix over the warps, and the sub-tile's count
      uint32_t cnt = 0;
      if (tid < 256) {
        for (int w = 0; w < kCoopWarps; ++w) {
          const uint32_t cw = s_wc[w * 256 + tid];
          s_wc[w * 256 + tid] = cnt;
          cnt += cw;
        }
      }
      uint32_t tot;
      const uint32_t dofs = coop_block_scan(tid < 256 ? cnt : 0u, &tot, s_scan);
      if (tid < 256) {
        s_doff[tid] = dofs;
        s_cnt[tid] = cnt;
      }
      __syncthreads();
#pragma unroll
      for (int it = 0; it < kCoopItems; ++it) {
        const int d = dg[it];
        if (d < 0) continue;
        const uint32_t pos = s_doff[d] + s_wc[warp * 256 + d] + rk[it];
        s_keys[pos] = k[it];
        if (VALS) s_vals[pos] = v[it];
      }
      __syncthreads();
      const int nvalid = (int)((hi - t0) < kCoopTile ? (hi - t0) : kCoopTile);
      for (int i = tid; i < nvalid; i += kCoopThreads) {
        const uint64_t key = s_keys[i];
        const int d = (int)((key >> shift) & dmask);
        const int64_t o = (int64_t)s_base[d] + s_run[d] + (i - (int)s_doff[d]);
        if (o < M) {
          kout[o] = key;
          if (VALS) vout[o] = s_vals[i];
        }
      }
      __syncthreads();
      if (tid < 256) s_run[tid] += s_cnt[tid];
      __syncthreads();
    }
    if (p + 1 < a.passes && !(ok = coop_grid_sync(a.bar, ++nbar * (uint32_t)G, &s_ok))) break;
  }
  if (!ok && tid == 0) atomicCAS(&a.ctl->status, 0, VM3DGS_E_TIMEOUT);
}

__global__ void ranges_kernel(const Ctl *ctl, const uint64_t *keys, int64_t cap, uint2 *ranges, uint32_t ntiles,
                              int tshift) {
  const int64_t M = ctl->pairs < cap ? ctl->pairs : cap;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
    const uint64_t t = keys[j] >> tshift;
    if (t >= ntiles) continue;  // only after a timed-out sort
    if (j == 0 || (keys[j - 1] >> tshift) != t) ranges[t].x = (uint32_t)j;
    if (j == M - 1 || (keys[j + 1] >> tshift) != t) ranges[t].y = (uint32_t)(j + 1);
  }
}

}  // namespace

void launch_scan_emit(const Ctl *ctl, Ctl *ctl_w, const Splats &sp, int64_t ncap, uint32_t *block_sums,
                      uint32_t *offsets, uint64_t *keys, uint32_t *vals, int64_t pair_cap, const TileGeom &tg, int gx,
                      const KeyFormat &kf, const SortHist &sh, uint64_t *pieces, uint32_t *piece_ctr,
                      int64_t piece_cap, uint2 *ranges, int ntiles, cudaStream_t st) {
  const int64_t nb = (ncap + kScanItems - 1) / kScanItems;
  uint64_t *bs = reinterpret_cast<uint64_t *>(block_sums);
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, 1, bs);
  // the scan of the block sums also zeroes the digit histograms and the piece counter
  scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(ctl_w, ncap, 1, bs, sh.hist, sh.hist ? kMaxPasses * 256 : 0, piece_ctr,
                                                 1);
  scan_offsets_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, 1, bs, offsets);
  const EmitViews ev{nullptr, tg, gx};
  emit_kernel<<<full_wave((const void *)emit_kernel, 256, 0), 256, 0, st>>>(ctl, sp, ncap, 1, ev, offsets, keys, vals,
                                                                            pair_cap, kf, sh, pieces, piece_ctr,
                                                                            piece_cap, ranges, ntiles);
  emit_pieces_kernel<<<full_wave((const void *)emit_pieces_kernel, 256, 0), 256, 0, st>>>(
      ctl, sp, ncap, ev, offsets, keys, vals, pair_cap, kf, sh, pieces, piece_ctr, piece_cap);
}

void launch_scan_emit_batched(Ctl *ctl, const Splats &sp, int64_t ncap, int views, const ViewTable *vt,
                              uint32_t *block_sums, uint32_t *offsets, uint64_t *keys, uint32_t *vals,
                              int64_t pair_cap, uint64_t *pieces, uint32_t *piece_ctr, int64_t piece_cap,
                              cudaStream_t st) {
  const int64_t nb = (ncap * views + kScanItems - 1) / kScanItems;
  uint64_t *bs = reinterpret_cast<uint64_t *>(block_sums);
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, views, bs);
  scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(ctl, ncap, views, bs, nullptr, 0, piece_ctr, 1);
  scan_offsets_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, views, bs, offsets);
  // keys (global tile << 32 | depth bits) with the record index as value
  const KeyFormat kf{32, 0, 32, 0u, false};
  const SortHist none{};
  const EmitViews ev{vt, TileGeom{0, 0, 1, 1}, 0};
  emit_kernel<<<full_wave((const void *)emit_kernel, 256, 0), 256, 0, st>>>(ctl, sp, ncap, views, ev, offsets, keys,
                                                                            vals, pair_cap, kf, none, pieces, piece_ctr,
                                                                            piece_cap, nullptr, 0);
  emit_pieces_kernel<<<full_wave((const void *)emit_pieces_kernel, 256, 0), 256, 0, st>>>(
      ctl, sp, ncap, ev, offsets, keys, vals, pair_cap, kf, none, pieces, piece_ctr, piece_cap);
}

int launch_sort_prep(Ctl *ctl, const uint64_t *keys, int64_t pair_cap, int lo_bit, int hi_bit, uint32_t *hist,
                     uint32_t *lookback, int64_t lookback_words, uint32_t *tile_ctr, cudaStream_t st) {
  const int passes = (hi_bit - lo_bit + 7) / 8;
  if (passes < 1 || passes > kMaxPasses || lo_bit < 0) return -1;
  const int64_t max_tiles = (pair_cap + kSortTile - 1) / kSortTile;
  if ((int64_t)passes * max_tiles * 256 > lookback_words) return -1;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kMaxPasses * 256, st);
  const int last_bits = hi_bit - lo_bit - 8 * (passes - 1);
  sort_hist_kernel<<<full_wave((const void *)sort_hist_kernel, 256, 0), 256, 0, st>>>(
      ctl, keys, pair_cap, lo_bit, passes, (1u << last_bits) - 1u, hist, lookback, max_tiles, tile_ctr);
  return 0;
}

int launch_sort_passes(Ctl *ctl, uint64_t *keys[2], uint32_t *vals[2], int64_t pair_cap, int lo_bit, int hi_bit,
                       uint32_t *hist, uint32_t *lookback, uint32_t *tile_ctr, cudaStream_t st) {
  const int passes = (hi_bit - lo_bit + 7) / 8;
  if (passes < 1 || passes > kMaxPasses || lo_bit < 0) return -1;
  const int smem = kSortTile * 12 + (kSortThreads / 32) * 256 * 4 + 2 * 256 * 4;
  {
    // kernel attributes belong to a device: set them once on each
    static std::mutex mu;
    static std::unordered_set<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!done.count(dev)) {
      if (cudaFuncSetAttribute(onesweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
          cudaFuncSetAttribute(onesweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -2;
      prefer_shared((const void *)onesweep_kernel<true>);
      prefer_shared((const void *)onesweep_kernel<false>);
      done.insert(dev);
    }
  }
  const int64_t max_tiles = (pair_cap + kSortTile - 1) / kSortTile;
  int grid = 148 * 4;
  if (grid > max_tiles) grid = (int)(max_tiles > 0 ? max_tiles : 1);
  int cur = 0;
  const int last_bits = hi_bit - lo_bit - 8 * (passes - 1);
  for (int d = 0; d < passes; ++d) {
    const int64_t lb_off = (int64_t)d * max_tiles * 256;
    // the digit of the last pass holds only the bits left below hi_bit
    const uint32_t dmask = d == passes - 1 ? (1u << last_bits) - 1u : 255u;
    if (vals[0])
      onesweep_kernel<true><<<grid, kSortThreads, smem, st>>>(ctl, keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1],
                                                              pair_cap, lo_bit + 8 * d, dmask, hist + d * 256,
                                                              lookback + lb_off, tile_ctr + d);
    else
      onesweep_kernel<false><<<grid, kSortThreads, smem, st>>>(ctl, keys[cur], nullptr, keys[cur ^ 1], nullptr,
                                                               pair_cap, lo_bit + 8 * d, dmask, hist + d * 256,
                                                               lookback + lb_off, tile_ctr + d);
    cur ^= 1;
  }
  return cur;
}

int coop_sort_grid() {
  static std::mutex mu;
  static std::unordered_map<int, int> grid;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = grid.find(dev);
  if (it != grid.end()) return it->second;
  int g = 0, coop = 0, sms = 0, per_sm = 0;
  const int smem = kCoopTile * 12 + kCoopWarps * 256 * 4;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaFuncSetAttribute(coop_sort_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
      cudaFuncSetAttribute(coop_sort_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_sort_kernel<true>, kCoopThreads, smem) == cudaSuccess) {
    int per_sm2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, coop_sort_kernel<false>, kCoopThreads, smem) ==
        cudaSuccess)
      per_sm = std::min(per_sm, per_sm2);
    g = std::min(per_sm * sms, kCoopMaxGrid);
  }
  cudaGetLastError();  // a refused attribute only means: no cooperative sort
  grid[dev] = g;
  return g;
}

int launch_sort_coop(Ctl *ctl, uint64_t *keys[2], uint32_t *vals[2], int64_t pair_cap, int lo_bit, int hi_bit,
                     const uint32_t *hist, uint32_t *scratch, int64_t scratch_words, uint32_t *bar, cudaStream_t st) {
  const int passes = (hi_bit - lo_bit + 7) / 8;
  if (passes < 1 || passes > kMaxPasses || lo_bit < 0) return -1;
  const int G = coop_sort_grid();
  if (G < 1 || (int64_t)2 * 256 * G > scratch_words) return -2;
  CoopSortArgs a;
  a.ctl = ctl;
  a.keys[0] = keys[0];
  a.keys[1] = keys[1];
  a.vals[0] = vals[0];
  a.vals[1] = vals[1];
  a.cap = pair_cap;
  a.lo_bit = lo_bit;
  a.passes = passes;
  a.last_mask = (1u << (hi_bit - lo_bit - 8 * (passes - 1))) - 1u;
  a.hist = hist;
  a.colhist = scratch;
  a.offs = scratch + (int64_t)256 * G;
  a.bar = bar;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kCoopThreads);
  cfg.dynamicSmemBytes = (size_t)(kCoopTile * (vals[0] ? 12 : 8) + kCoopWarps * 256 * 4);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = vals[0] ? cudaLaunchKernelEx(&cfg, coop_sort_kernel<true>, a)
                                : cudaLaunchKernelEx(&cfg, coop_sort_kernel<false>, a);
  if (e != cudaSuccess) return -3;
  return passes & 1;
}

int launch_sort(Ctl *ctl, uint64_t *keys[2], uint32_t *vals[2], int64_t pair_cap, int lo_bit, int hi_bit,
                uint32_t *hist, uint32_t *lookback, int64_t lookback_words, uint32_t *tile_ctr, cudaStream_t st) {
  const int rc = launch_sort_prep(ctl, keys[0], pair_cap, lo_bit, hi_bit, hist, lookback, lookback_words, tile_ctr, st);
  if (rc < 0) return rc;
  return launch_sort_passes(ctl, keys, vals, pair_cap, lo_bit, hi_bit, hist, lookback, tile_ctr, st);
}

void launch_ranges(const Ctl *ctl, const uint64_t *keys, int64_t pair_cap, uint2 *ranges, int ntiles, int tshift,
                   cudaStream_t st, bool zeroed) {
  if (!zeroed) cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, st);
  ranges_kernel<<<full_wave((const void *)ranges_kernel, 256, 0), 256, 0, st>>>(ctl, keys, pair_cap, ranges,
                                                                                (uint32_t)ntiles, tshift);
}

}  // namespace vm
