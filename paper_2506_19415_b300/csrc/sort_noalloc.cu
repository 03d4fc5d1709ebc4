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

#include <mutex>
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

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

__global__ void begin_kernel(Ctl *ctl, int64_t n) {
  ctl->pairs = n;
  ctl->status = 0;
}

__global__ void end_kernel(Ctl *ctl, int32_t *status_out) {
  if (status_out) *status_out = ctl->status;
  ctl->status = 0;
}

}  // namespace
}  // namespace vm

using namespace vm;

extern "C" int vm3dgs_sort_pairs_noalloc(uint64_t *keys_dev, uint32_t *vals_dev, int64_t n, int32_t key_bits,
                                         int32_t *status_dev, void *stream) {
  if (!keys_dev || !vals_dev) return fail(VM3DGS_E_INVAL, "null keys or values");
  if (n < 0 || n > kMaxPairs)
    return fail(VM3DGS_E_CAPACITY, "at most " + std::to_string(kMaxPairs) + " pairs per call, got " + std::to_string(n));
  if (key_bits < 1 || key_bits > 64) return fail(VM3DGS_E_INVAL, "key_bits must be 1..64");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(VM3DGS_E_CUDA, "no usable current device");
  unsigned char *base = nullptr;
  {
    // first call on this device: look up the device address of the array
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
      if (e != cudaSuccess || !p) return fail(VM3DGS_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = static_cast<unsigned char *>(p);
    }
    base = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  Ctl *ctl = reinterpret_cast<Ctl *>(base + kOffCtl);
  begin_kernel<<<1, 1, 0, st>>>(ctl, n);
  if (n > 1) {
    uint64_t *keys[2] = {keys_dev, reinterpret_cast<uint64_t *>(base + kOffKeys)};
    uint32_t *vals[2] = {vals_dev, reinterpret_cast<uint32_t *>(base + kOffVals)};
    const int cur = launch_sort(ctl, keys, vals, n, 0, key_bits, reinterpret_cast<uint32_t *>(base + kOffHist),
                                reinterpret_cast<uint32_t *>(base + kOffLook), kLookbackWords,
                                reinterpret_cast<uint32_t *>(base + kOffTiles), st);
    if (cur < 0) return fail(VM3DGS_E_CUDA, "sort launch refused");
    if (cur == 1) {
      cudaMemcpyAsync(keys_dev, keys[1], 8 * (size_t)n, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(vals_dev, vals[1], 4 * (size_t)n, cudaMemcpyDeviceToDevice, st);
    }
  }
  end_kernel<<<1, 1, 0, st>>>(ctl, status_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, std::string("sort: ") + cudaGetErrorString(e));
}
