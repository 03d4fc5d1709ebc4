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

// Last index i in [0, N) with offsets[i] <= j (offsets ascending from 0),
// found by the whole warp: each round probes 32 evenly spaced entries and
// keeps the span between the last probe at or below j and the next one.
__device__ __forceinline__ int64_t warp_find(const uint32_t *offsets, int64_t N, uint32_t j, int lane) {
  int64_t lo = 0, hi = N;
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t p = lo + lane * step;
    const bool ok = p < hi && offsets[p] <= j;
    const uint32_t b = __ballot_sync(0xffffffffu, ok);
    const int last = 31 - __clz(b);
    lo += last * step;
    hi = min(hi, lo + step);
  }
  const int64_t p = lo + lane;
  const uint32_t b = __ballot_sync(0xffffffffu, p < hi && offsets[p] <= j);
  return lo + (31 - __clz(b));
}

// Rectangle position (row-major) of the q-th covered tile of a splat.
__device__ __forceinline__ uint32_t covered_tile(uint64_t m, uint32_t w, uint32_t h, uint32_t q) {
  if (w * h > 64) return q;
  const uint32_t lo = (uint32_t)m, c = __popc(lo);
  return q < c ? __fns(lo, 0, (int)q + 1) : 32u + __fns((uint32_t)(m >> 32), 0, (int)(q - c) + 1);
}

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
  __device__ __forceinline__ void put(int64_t j, uint32_t tile, uint64_t dkey, uint32_t i) const {
    const uint64_t key = ((uint64_t)tile << kf.tshift) | dkey;
    if (j < M) {
      if (kf.packed) {
        keys[j] = key | (uint64_t)i;
      } else {
        keys[j] = key;
        vals[j] = i;
      }
    }
    if (hist) {
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

// Pair emission (pairs of a splat: its covered tiles in row-major order, at
// its scanned offset), part 1: a warp takes 32 consecutive splats, a lane
// each, with coalesced loads of their records.  The pairs of the splats with
// at most 32 of them are dealt out to the lanes together (lane g of a round
// writes pair g of the concatenation, its splat found by a binary search over
// the lanes' inclusive counts and its record fetched by shuffles), so stores
// are contiguous and no lane walks the offsets.  Larger splats are cut into
// pieces of kPiece pairs, listed for part 2.  Digits that lie in the depth
// field are the same for all pairs of a splat and are counted once per
// splat.  With sh.hist the kernel also counts the sort's digits
// (shared-memory histograms merged into sh.hist) and clears the sort's
// look-back words and tile counters.
__global__ void __launch_bounds__(256) emit_kernel(const Ctl *ctl, Splats sp, int64_t ncap, const uint32_t *offsets,
                                                   uint64_t *keys, uint32_t *vals, int64_t pair_cap, int gx,
                                                   KeyFormat kf, SortHist sh, uint64_t *pieces,
                                                   uint32_t *piece_ctr, int64_t piece_cap, uint2 *ranges, int ntiles) {
  __shared__ uint32_t hs[kMaxPasses][256];
  if (sh.hist) {
    for (int i = threadIdx.x; i < sh.passes * 256; i += blockDim.x) (&hs[0][0])[i] = 0;
    __syncthreads();
  }
  const PairOut po = pair_out(ctl, keys, vals, pair_cap, kf, sh, hs);
  const int64_t N = n_drawn(ctl, ncap);
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
    const bool big = cnt > kSmallSplat;
    if (cnt && !big) {
      off = cur.off;
      rx = cur.rx;
      ry = cur.ry;
      tm = cur.tm;
      dkey = depth_key(cur.db, kf);
      if (po.hist) count_run(hs, dkey >> po.lo_bit, po.dpass, cnt);
    }
    const uint32_t small = big ? 0u : cnt;
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
      const uint32_t Loff = __shfl_sync(0xffffffffu, off, L);
      if (g < total) {
        const uint32_t q = g - (Li - Ln);
        const uint32_t x0 = Lrx & 0xFFFFu, w = (Lrx >> 16) - x0, y0 = Lry & 0xFFFFu, h = (Lry >> 16) - y0;
        const uint32_t qt = covered_tile(Ltm, w, h, q);
        po.put((int64_t)Loff + q, (y0 + qt / w) * (uint32_t)gx + x0 + qt % w, Ld, (uint32_t)(b + L));
      }
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
    for (int d = 0; d < sh.passes; ++d) {
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
__global__ void __launch_bounds__(256) emit_pieces_kernel(const Ctl *ctl, Splats sp, const uint32_t *offsets,
                                                          uint64_t *keys, uint32_t *vals, int64_t pair_cap, int gx,
                                                          KeyFormat kf, SortHist sh, const uint64_t *pieces,
                                                          const uint32_t *piece_ctr, int64_t piece_cap) {
  __shared__ uint32_t hs[kMaxPasses][256];
  if (sh.hist) {
    for (int i = threadIdx.x; i < sh.passes * 256; i += blockDim.x) (&hs[0][0])[i] = 0;
    __syncthreads();
  }
  const PairOut po = pair_out(ctl, keys, vals, pair_cap, kf, sh, hs);
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
    const uint64_t tm = sp.tmask[i], dkey = depth_key(sp.depth[i], kf);
    if (po.hist && k == 0 && lane == 0) count_run(hs, dkey >> po.lo_bit, po.dpass, cnt);
    const uint32_t x0 = rx & 0xFFFFu, w = (rx >> 16) - x0, y0 = ry & 0xFFFFu, h = (ry >> 16) - y0;
    const uint32_t q1 = min(cnt, (k + 1) * kPiece);
    for (uint32_t q = k * kPiece + lane; q < q1; q += 32) {
      const uint32_t qt = covered_tile(tm, w, h, q);
      po.put((int64_t)off + q, (y0 + qt / w) * (uint32_t)gx + x0 + qt % w, dkey, (uint32_t)i);
    }
  }
  if (sh.hist) hist_flush(sh, hs);
}

constexpr int kEmitChunk = 256;  // pairs per warp task of the batched emission

// Pairs of all views of a batch: splat record v * N + i belongs to view v;
// the key's tile field is the view's first global tile plus its local tile.
__global__ void __launch_bounds__(256) emit_batched_kernel(const Ctl *ctl, Splats sp, int64_t ncap, int views,
                                                           const ViewTable *vt, const uint32_t *offsets,
                                                           uint64_t *keys, uint32_t *vals, int64_t pair_cap) {
  const int64_t Nv = n_drawn(ctl, ncap);
  const int64_t N = Nv * views;
  int64_t M = ctl->pairs;
  if (M > pair_cap) M = pair_cap;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp0; c * kEmitChunk < M; c += nwarps) {
    const uint32_t j0 = (uint32_t)(c * kEmitChunk);
    int64_t i = warp_find(offsets, N, j0, lane);  // last splat with offset <= j0
    for (int k = 0; k < kEmitChunk / 32; ++k) {
      const uint32_t j = j0 + 32u * k + lane;
      if ((int64_t)j >= M) break;
      if (i + 1 < N && offsets[i + 1] <= j) {
        int64_t lo2 = i + 1, step = 1;
        while (lo2 + step < N && offsets[lo2 + step] <= j) { lo2 += step; step <<= 1; }
        int64_t hi2 = lo2 + step < N ? lo2 + step - 1 : N - 1;
        while (lo2 < hi2) {
          const int64_t mid = (lo2 + hi2 + 1) >> 1;
          if (offsets[mid] <= j) lo2 = mid; else hi2 = mid - 1;
        }
        i = lo2;
      }
      const int v = (int)(i / Nv);
      const uint32_t rx = sp.rect[2 * i], ry = sp.rect[2 * i + 1];
      const uint32_t x0 = rx & 0xFFFFu, w = (rx >> 16) - x0, y0 = ry & 0xFFFFu, h = (ry >> 16) - y0;
      const uint32_t q = covered_tile(sp.tmask[i], w, h, j - offsets[i]);
      const uint32_t tile = (uint32_t)vt->tile_off[v] + (y0 + q / w) * (uint32_t)vt->gx[v] + x0 + q % w;
      keys[j] = ((uint64_t)tile << 32) | sp.depth[i];
      vals[j] = (uint32_t)i;
    }
  }
}

// ------------------------------------------------------------------ onesweep
__global__ void __launch_bounds__(256) sort_hist_kernel(const Ctl *ctl, const uint64_t *keys, int64_t cap, int lo_bit,
                                                        int passes, uint32_t *hist, uint32_t *lookback,
                                                        int64_t max_tiles, uint32_t *tile_ctr) {
  __shared__ uint32_t h[kMaxPasses][256];
  const int64_t M = ctl->pairs < cap ? ctl->pairs : cap;
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
    const uint64_t k = keys[j] >> lo_bit;
    for (int d = 0; d < passes; ++d) atomicAdd(&h[d][(k >> (8 * d)) & 255u], 1u);
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

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// one radix digit per thread: the digit scans and count loads index by tid
static_assert(kSortThreads == 256, "onesweep assumes one thread per 8-bit digit");

template <bool VALS>
__global__ void __launch_bounds__(kSortThreads, 4) onesweep_kernel(Ctl *ctl, const uint64_t *kin, const uint32_t *vin,
                                                                uint64_t *kout, uint32_t *vout, int64_t cap, int shift,
                                                                const uint32_t *counts, uint32_t *status,
                                                                uint32_t *tile_ctr) {
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
      dg[it] = valid ? (int)((k[it] >> shift) & 255u) : -1;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
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
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const int d = dg[it];
      if (d < 0) continue;
      const uint32_t pos = s_doff[d] + s_wc[warp * 256 + d] + rk[it];
      s_keys[pos] = k[it];
      if (VALS) s_vals[pos] = v[it];
    }
    __syncthreads();
    const int nvalid = (int)((M - t0) < kSortTile ? (M - t0) : kSortTile);
    for (int i = tid; i < nvalid; i += kSortThreads) {
      const uint64_t key = s_keys[i];
      const int d = (int)((key >> shift) & 255u);
      const uint32_t o = s_glob[d] + (uint32_t)i - s_doff[d];
      if ((int64_t)o < M) {  // always true unless a look-back wait timed out
        kout[o] = key;
        if (VALS) vout[o] = s_vals[i];
      }
    }
    __syncthreads();
  }
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
                      uint32_t *offsets, uint64_t *keys, uint32_t *vals, int64_t pair_cap, int gx, const KeyFormat &kf,
                      const SortHist &sh, uint64_t *pieces, uint32_t *piece_ctr, int64_t piece_cap, uint2 *ranges,
                      int ntiles, cudaStream_t st) {
  const int64_t nb = (ncap + kScanItems - 1) / kScanItems;
  uint64_t *bs = reinterpret_cast<uint64_t *>(block_sums);
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, 1, bs);
  // the scan of the block sums also zeroes the digit histograms and the piece counter
  scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(ctl_w, ncap, 1, bs, sh.hist, sh.hist ? kMaxPasses * 256 : 0, piece_ctr,
                                                 1);
  scan_offsets_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, 1, bs, offsets);
  emit_kernel<<<full_wave((const void *)emit_kernel, 256, 0), 256, 0, st>>>(ctl, sp, ncap, offsets, keys, vals, pair_cap,
                                                                            gx, kf, sh, pieces, piece_ctr, piece_cap,
                                                                            ranges, ntiles);
  emit_pieces_kernel<<<full_wave((const void *)emit_pieces_kernel, 256, 0), 256, 0, st>>>(
      ctl, sp, offsets, keys, vals, pair_cap, gx, kf, sh, pieces, piece_ctr, piece_cap);
}

void launch_scan_emit_batched(Ctl *ctl, const Splats &sp, int64_t ncap, int views, const ViewTable *vt,
                              uint32_t *block_sums, uint32_t *offsets, uint64_t *keys, uint32_t *vals,
                              int64_t pair_cap, cudaStream_t st) {
  const int64_t nb = (ncap * views + kScanItems - 1) / kScanItems;
  uint64_t *bs = reinterpret_cast<uint64_t *>(block_sums);
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, views, bs);
  scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(ctl, ncap, views, bs, nullptr, 0, nullptr, 0);
  scan_offsets_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, sp.touched, ncap, views, bs, offsets);
  emit_batched_kernel<<<full_wave((const void *)emit_batched_kernel, 256, 0), 256, 0, st>>>(ctl, sp, ncap, views, vt,
                                                                                            offsets, keys, vals, pair_cap);
}

int launch_sort_prep(Ctl *ctl, const uint64_t *keys, int64_t pair_cap, int lo_bit, int hi_bit, uint32_t *hist,
                     uint32_t *lookback, int64_t lookback_words, uint32_t *tile_ctr, cudaStream_t st) {
  const int passes = (hi_bit - lo_bit + 7) / 8;
  if (passes < 1 || passes > kMaxPasses || lo_bit < 0) return -1;
  const int64_t max_tiles = (pair_cap + kSortTile - 1) / kSortTile;
  if ((int64_t)passes * max_tiles * 256 > lookback_words) return -1;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kMaxPasses * 256, st);
  sort_hist_kernel<<<full_wave((const void *)sort_hist_kernel, 256, 0), 256, 0, st>>>(ctl, keys, pair_cap, lo_bit,
                                                                                      passes, hist, lookback, max_tiles,
                                                                                      tile_ctr);
  return 0;
}

int launch_sort_passes(Ctl *ctl, uint64_t *keys[2], uint32_t *vals[2], int64_t pair_cap, int lo_bit, int hi_bit,
                       uint32_t *hist, uint32_t *lookback, uint32_t *tile_ctr, cudaStream_t st) {
  const int passes = (hi_bit - lo_bit + 7) / 8;
  if (passes < 1 || passes > kMaxPasses || lo_bit < 0) return -1;
  static bool attr_set = false;
  const int smem = kSortTile * 12 + (kSortThreads / 32) * 256 * 4 + 2 * 256 * 4;
  if (!attr_set) {
    if (cudaFuncSetAttribute(onesweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(onesweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return -2;
    prefer_shared((const void *)onesweep_kernel<true>);
    prefer_shared((const void *)onesweep_kernel<false>);
    attr_set = true;
  }
  const int64_t max_tiles = (pair_cap + kSortTile - 1) / kSortTile;
  int grid = 148 * 4;
  if (grid > max_tiles) grid = (int)(max_tiles > 0 ? max_tiles : 1);
  int cur = 0;
  for (int d = 0; d < passes; ++d) {
    const int64_t lb_off = (int64_t)d * max_tiles * 256;
    if (vals[0])
      onesweep_kernel<true><<<grid, kSortThreads, smem, st>>>(ctl, keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1],
                                                              pair_cap, lo_bit + 8 * d, hist + d * 256,
                                                              lookback + lb_off, tile_ctr + d);
    else
      onesweep_kernel<false><<<grid, kSortThreads, smem, st>>>(ctl, keys[cur], nullptr, keys[cur ^ 1], nullptr,
                                                               pair_cap, lo_bit + 8 * d, hist + d * 256,
                                                               lookback + lb_off, tile_ctr + d);
    cur ^= 1;
  }
  return cur;
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
