// Internal scene representation shared by the host builder and the renderer.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vm3dgs.h"

struct vm3dgs_scene;

#ifdef __CUDACC__
#define VM_HD __host__ __device__
#else
#define VM_HD
#endif

namespace vm {

constexpr int kMaxLevels = 6;

// Error reporting: a thread-local message plus the return code.
int fail(int code, const std::string &msg);

// IEEE binary32 -> binary16, round to nearest even
uint16_t f32_to_f16(float f);

// Page centroids and the box around them (for the prefetch window and LOD of
// prefetched pages); called at the end of every scene construction.
void finish_scene(vm3dgs_scene *s);

// fp32 record: attributes of one Gaussian as float arrays of a page block.
//   0..2 pos, 3..5 scale, 6..9 rot (w,x,y,z), 10 opacity, 11 + 3k + c  SH coefficient k, channel c
VM_HD constexpr int n_attr32(int K) { return 11 + 3 * K; }
// fp16 record: float arrays pos x,y,z, opacity; then half arrays
//   0..2 scale, 3..6 rot, 7 + 3k + c SH, padded to an even count.
VM_HD constexpr int n_half16(int K) { return ((7 + 3 * K) + 1) & ~1; }
VM_HD constexpr int rec_bytes32(int K) { return 4 * n_attr32(K); }
VM_HD constexpr int rec_bytes16(int K) { return 16 + 2 * n_half16(K); }
// VQ record (compressed pages): float arrays pos x,y,z, opacity; then 16-bit
// arrays 0..2 scale, 3..6 rot, 7..9 SH band 0 (half), 10 the codebook index
// of the SH bands 1..3 (unsigned), 11 padding: 40 bytes at every SH degree.
constexpr int kHalfVQ = 12;
VM_HD constexpr int rec_bytes_vq() { return 16 + 2 * kHalfVQ; }
// pool formats: 0 fp32 records, 1 fp16 records, 2 VQ records
constexpr int kFmt32 = 0, kFmt16 = 1, kFmtVQ = 2;
// a codeword in device memory: per channel c its bands-1..3 coefficients at
// floats [16 c, 16 c + K - 1), zero padded (aligned 16-byte loads)
constexpr int kCodeRow = 48;

}  // namespace vm

struct vm3dgs_scene {
  int32_t n_pages = 0, page_size = 0, levels = 1, fanout = 8, sh_degree = 0, K = 1;
  int64_t n_gauss = 0;
  int32_t rec32 = 0, rec16 = 0;
  std::vector<int64_t> count;    // real level-0 Gaussians per page
  std::vector<int64_t> src;      // [n_pages * page_size] input index or -1
  // page blocks: level l page p occupies bytes [off32[l] + p * m_l * rec32, +m_l * rec32)
  uint8_t *data32 = nullptr;
  int64_t bytes32 = 0;
  int64_t off32[vm::kMaxLevels] = {0};
  uint8_t *data16 = nullptr;
  int64_t bytes16 = 0;
  int64_t off16[vm::kMaxLevels] = {0};
  std::vector<float> err;        // [n_pages * levels]
  std::vector<float> verts;      // [n_verts * 3]
  std::vector<int32_t> tris;     // [n_tris * 3]
  std::vector<int32_t> face_page;
  std::vector<int64_t> link_ptr; // [n_pages + 1]
  std::vector<int32_t> link_col;
  std::vector<float> centroid;   // [n_pages * 4]: mean of the level-0 means, radius incl. 3 sigma
  float box_center[3] = {0, 0, 0}, box_half = 1.0f;
  bool registered32 = false, registered16 = false, registered_vq = false;
  // compressed pages: the SH codebook [n_codes][code_dim] (code_dim = 3 (K - 1))
  // and the VQ records, laid out like the others (vm3dgs_scene_quantize_sh)
  int32_t rec_vq = 0, n_codes = 0, code_dim = 0;
  std::vector<float> codebook;
  uint8_t *data_vq = nullptr;
  int64_t bytes_vq = 0;
  int64_t off_vq[vm::kMaxLevels] = {0};
  // opened from a scene file: data32/data16 point into a read-only mapping of
  // the file, read by the OS on first touch (Sec. 3.5, memory-mapped scene)
  bool mapped = false;
  void *map_base = nullptr;
  size_t map_len = 0;

  // page data, byte offsets of the levels and record size of a pool format
  uint8_t *fmt_data(int f) const { return f == vm::kFmtVQ ? data_vq : f == vm::kFmt16 ? data16 : data32; }
  int64_t fmt_bytes(int f) const { return f == vm::kFmtVQ ? bytes_vq : f == vm::kFmt16 ? bytes16 : bytes32; }
  const int64_t *fmt_off(int f) const { return f == vm::kFmtVQ ? off_vq : f == vm::kFmt16 ? off16 : off32; }
  int32_t fmt_rec(int f) const { return f == vm::kFmtVQ ? rec_vq : f == vm::kFmt16 ? rec16 : rec32; }
  bool &fmt_registered(int f) { return f == vm::kFmtVQ ? registered_vq : f == vm::kFmt16 ? registered16 : registered32; }

  int32_t m(int l) const {
    int32_t v = page_size;
    for (int i = 0; i < l; ++i) v /= fanout;
    return v;
  }
  ~vm3dgs_scene();
};
