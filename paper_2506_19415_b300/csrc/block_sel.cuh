// Block-wide primitives of the one-CTA page-table steps (update and
// prefetch placement): a CTA of RT threads, an exclusive scan, a bitonic
// sort through shared memory, and a radix select of the k smallest keys.
// Included into one translation unit each (internal linkage).
#pragma once
#include <cstdint>

namespace vm {
namespace {

constexpr int RT = 1024;
constexpr int kSmemKeys = 16384;

struct ScanSmem {
  int64_t warp[32];
  int64_t total;
};

// exclusive block scan (all 1024 threads call it); returns prefix, sets total
__device__ int64_t bscan(int64_t v, int64_t *total, ScanSmem &sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm.warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t t = sm.warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sm.warp[lane] = t;
  }
  __syncthreads();
  const int64_t pre = (warp ? sm.warp[warp - 1] : 0) + x - v;
  *total = sm.warp[31];
  __syncthreads();
  return pre;
}

// The k smallest of the distinct keys g[0, n) (0 < k < n, k <= kSmemKeys),
// ascending, into g[0, k): a most-significant-digit radix select of the k-th
// smallest key (8 bits a round), the keys at or below it compacted through
// shared memory and sorted there.
__device__ void select_smallest(uint64_t *g, int n, int k, uint64_t *sh, ScanSmem &sm) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t s_pref;
  __shared__ int s_rank;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    s_pref = 0;
    s_rank = k - 1;
  }
  uint64_t mask = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += RT) hist[i] = 0;
    __syncthreads();
    const uint64_t pref = s_pref;
    for (int i = tid; i < n; i += RT) {
      const uint64_t key = g[i];
      if ((key & mask) == pref) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid < 32) {
      uint32_t c[8], sum = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        c[b] = hist[8 * lane + b];
        sum += c[b];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int target = s_rank;
      const uint32_t excl = incl - sum;
      if ((int)excl <= target && target < (int)incl) {
        int t = target - (int)excl, b = 0;
        while (t >= (int)c[b]) {
          t -= (int)c[b];
          ++b;
        }
        s_pref = pref | ((uint64_t)(8 * lane + b) << shift);
        s_rank = t;
      }
    }
    mask |= 0xFFull << shift;
    __syncthreads();
  }
  const uint64_t thr = s_pref;  // the k-th smallest key
  int64_t base = 0, tot;
  for (int c = 0; c < n; c += RT) {
    const int i = c + tid;
    const int f = (i < n && g[i] <= thr) ? 1 : 0;
    const int64_t pos = bscan(f, &tot, sm);
    if (f) sh[base + pos] = g[i];
    base += tot;
  }
  int m = 1;
  while (m < k) m <<= 1;
  for (int i = k + tid; i < m; i += RT) sh[i] = ~0ull;
  __syncthreads();
  for (int kk = 2; kk <= m; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < m; i += RT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = sh[i], y = sh[ixj];
          if ((x > y) == ((i & kk) == 0)) {
            sh[i] = y;
            sh[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int i = tid; i < k; i += RT) g[i] = sh[i];
  __syncthreads();
}

// bitonic sort of n_pow2 keys, staged through shared memory when they fit
__device__ void bitonic(uint64_t *g, int n_pow2, uint64_t *sh) {
  uint64_t *a = n_pow2 <= kSmemKeys ? sh : g;
  if (a == sh) {
    for (int i = threadIdx.x; i < n_pow2; i += RT) sh[i] = g[i];
    __syncthreads();
  }
  for (int k = 2; k <= n_pow2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n_pow2; i += RT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = a[i], y = a[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) { a[i] = y; a[ixj] = x; }
        }
      }
      __syncthreads();
    }
  if (a == sh) {
    for (int i = threadIdx.x; i < n_pow2; i += RT) g[i] = sh[i];
    __syncthreads();
  }
}

__device__ int pow2_at_least(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

}  // namespace
}  // namespace vm
