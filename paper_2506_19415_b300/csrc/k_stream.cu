// Page streaming (Sec. 4.1 "Page Table Management" and evaluation
// "Transfer"): the pages of the copy list move from the scene's page-locked
// host memory into their pool sub-slots.  The paper copies through a staging
// buffer with the graphics driver; here the GPU pulls the bytes itself over
// the host link with 16-byte loads, so the copy list never returns to the
// CPU.  Work is cut into 64 KiB segments spread over a persistent grid;
// every copied page is one contiguous block on both sides.  A thread issues
// kInFlight loads before its stores, so a segment crosses the host link in
// one round trip.  For a scene opened from a file the host first gathers the
// frame's pages into a page-locked staging buffer, and the kernel reads each
// copy at its staging offset instead.
#include "renderer.cuh"

namespace vm {
namespace {

constexpr int kStreamThreads = 512, kInFlight = 8;  // 512 x 8 x 16 B = one 64 KiB segment

__global__ void __launch_bounds__(kStreamThreads) stream_kernel(StreamArgs a) {
  const int n = *a.count;
  const int64_t nseg = a.copy_seg[n];
  for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    // copy holding this segment
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.copy_seg[mid] <= sg) lo = mid; else hi = mid - 1;
    }
    const int4 c = a.copies[lo];
    int m = a.page_size;
    for (int l = 0; l < c.y; ++l) m /= a.fanout;
    const int64_t bytes = (int64_t)m * a.rec;
    const int64_t off = (sg - a.copy_seg[lo]) * kCopySeg;
    const int64_t len = bytes - off < kCopySeg ? bytes - off : kCopySeg;
    const uint4 *src = reinterpret_cast<const uint4 *>(
        a.host + (a.staged_off ? a.staged_off[lo] : a.level_off[c.y] + (int64_t)c.x * bytes) + off);
    uint4 *dst = reinterpret_cast<uint4 *>(a.pool + (int64_t)c.z * a.slot_bytes + (int64_t)c.w * bytes + off);
    const int64_t n16 = len / 16;
    for (int64_t i0 = threadIdx.x; i0 < n16; i0 += (int64_t)kInFlight * kStreamThreads) {
      uint4 v[kInFlight];
#pragma unroll
      for (int u = 0; u < kInFlight; ++u) {
        const int64_t i = i0 + (int64_t)u * kStreamThreads;
        if (i < n16) v[u] = src[i];
      }
#pragma unroll
      for (int u = 0; u < kInFlight; ++u) {
        const int64_t i = i0 + (int64_t)u * kStreamThreads;
        if (i < n16) dst[i] = v[u];
      }
    }
  }
}

}  // namespace

void launch_stream(const StreamArgs &a, cudaStream_t st) { stream_kernel<<<148 * 2, kStreamThreads, 0, st>>>(a); }

}  // namespace vm
