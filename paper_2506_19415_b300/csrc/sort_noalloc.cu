// Stable radix sort of (key, value) pairs that allocates no memory: the same
// onesweep kernels as the renderer's sort, with their scratch (the second
// key/value buffers, digit histograms, look-back words, tile counters and a
// small control block) in one file-scope device array of fixed size.
//
// Who needs it: callers that cannot call cudaMalloc or take memory from a
// caching allocator, for example a host application that reserves all device
// memory for itself at start-up and hands libraries only its own buffers, or
// a frame loop that must not pay the device-wide synchronisation cudaMalloc
// and cudaFree imply.  They pass only their keys and values.
//
// Limits and sharing.  At most VM3DGS_NOALLOC_MAX_PAIRS pairs per call.  The
// array belongs to the library and stays on every device that loads it until
// the process exits.  Every call on a device uses the same array, and it keeps
// what the last call left in it; the control block and counters are cleared
// by each call before use.  Calls whose work overlaps on a device (on
// different streams, or from different threads) race on the array.
#include <cuda_runtime.h>

#include <string>

#include "renderer.cuh"

namespace vm {
namespace {

constexpr int64_t kMaxPairs = VM3DGS_NOALLOC_MAX_PAIRS;
constexpr int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }
constexpr int64_t kMaxTiles = (kMaxPairs + kSortTile - 1) / kSortTile;
constexpr int64_t kLookbackWords = (int64_t)kMaxPasses * kMaxTiles * 256;
constexpr int64_t kOffCtl = 0;
constexpr int64_t kOffHist = align256(kOffCtl + (int64_t)sizeof(Ctl));
constexpr int64_t kOffTiles = align256(kOffHist + 4 * kMaxPasses * 256);
constexpr int64_t kOffLook = align256(kOffTiles + 4 * kMaxPasses);
constexpr int64_t kOffKeys = align256(kOffLook + 4 * kLookbackWords);
constexpr int64_t kOffVals = align256(kOffKeys + 8 * kMaxPairs);
constexpr int64_t kScratchBytes = align256(kOffVals + 4 * kMaxPairs);

// the scratch of every call on this device
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

__global__ void begin_kernel(Ctl *ctl, int64_t n) {
  ctl->pairs = n;
  ctl->status = 0;
}

// copies the call's status out (forced, when non-zero, replaces it) and
// clears it for the next call
__global__ void end_kernel(Ctl *ctl, int32_t *status_out, int32_t forced) {
  if (status_out) *status_out = forced ? forced : ctl->status;
  ctl->status = 0;
}

}  // namespace
}  // namespace vm

using namespace vm;

extern "C" int vm3dgs_sort_pairs_noalloc(uint64_t *keys_dev, uint32_t *vals_dev, int64_t n, int32_t key_bits,
                                         int32_t *status_dev, void *stream) {
  if ((!keys_dev || !vals_dev) && n > 0) return fail(VM3DGS_E_INVAL, "null keys or values");
  if (n < 0 || n > kMaxPairs)
    return fail(VM3DGS_E_CAPACITY, "at most " + std::to_string(kMaxPairs) + " pairs per call, got " + std::to_string(n));
  if (key_bits < 1 || key_bits > 64) return fail(VM3DGS_E_INVAL, "key_bits must be 1..64");
  // an error left by the caller's earlier work is not this call's to report
  // (or to clear): refuse to start on top of it
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return fail(VM3DGS_E_CUDA, std::string("a CUDA error from earlier work is pending: ") + cudaGetErrorString(pending));
  // the array's address in the current context, looked up on every call: a
  // host-side lookup once the library's module is loaded there (the first
  // call on a device loads it), and never stale after a device reset or in
  // another context of the same device
  void *p = nullptr;
  const cudaError_t ea = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (ea != cudaSuccess || !p) return fail(VM3DGS_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ea));
  unsigned char *base = static_cast<unsigned char *>(p);
  cudaStream_t st = (cudaStream_t)stream;
  Ctl *ctl = reinterpret_cast<Ctl *>(base + kOffCtl);
  begin_kernel<<<1, 1, 0, st>>>(ctl, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VM3DGS_E_CUDA, std::string("sort: ") + cudaGetErrorString(e));
  int32_t forced = 0;
  std::string why;
  if (n > 1) {
    uint64_t *keys[2] = {keys_dev, reinterpret_cast<uint64_t *>(base + kOffKeys)};
    uint32_t *vals[2] = {vals_dev, reinterpret_cast<uint32_t *>(base + kOffVals)};
    const int cur = launch_sort(ctl, keys, vals, n, 0, key_bits, reinterpret_cast<uint32_t *>(base + kOffHist),
                                reinterpret_cast<uint32_t *>(base + kOffLook), kLookbackWords,
                                reinterpret_cast<uint32_t *>(base + kOffTiles), st);
    if (cur < 0) {
      forced = VM3DGS_E_CUDA;
      why = "sort launch refused";
    } else if ((e = cudaGetLastError()) != cudaSuccess) {
      forced = VM3DGS_E_CUDA;
      why = std::string("sort: ") + cudaGetErrorString(e);
    } else if (cur == 1) {
      cudaError_t c1 = cudaMemcpyAsync(keys_dev, keys[1], 8 * (size_t)n, cudaMemcpyDeviceToDevice, st);
      cudaError_t c2 = c1 == cudaSuccess ? cudaMemcpyAsync(vals_dev, vals[1], 4 * (size_t)n, cudaMemcpyDeviceToDevice, st)
                                         : c1;
      if (c2 != cudaSuccess) {
        forced = VM3DGS_E_CUDA;
        why = std::string("copy back: ") + cudaGetErrorString(c2);
      }
    }
  }
  // the status word is written on the failure path too, so a stream-ordered
  // reader of it sees the failure
  end_kernel<<<1, 1, 0, st>>>(ctl, status_dev, forced);
  e = cudaGetLastError();
  if (forced) return fail(VM3DGS_E_CUDA, why);
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, std::string("sort: ") + cudaGetErrorString(e));
}
