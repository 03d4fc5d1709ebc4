// Scene object: error reporting, import of prepared pages, inspection.
#include <cuda_runtime.h>
#include <fcntl.h>
#include <sys/mman.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "scene.h"

namespace vm {
thread_local std::string g_last_error;
int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}
void finish_scene(vm3dgs_scene *S) {
  const int64_t NP = S->n_pages, ps = S->page_size;
  const int NA = n_attr32(S->K);
  S->centroid.assign(4 * NP, 0.0f);
  const float *L0 = (const float *)(S->data32 + S->off32[0]);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t p = 0; p < NP; ++p) {
    const float *b = L0 + p * ps * NA;
    const int64_t n = S->count[p];
    double c[3] = {0, 0, 0};
    for (int64_t g = 0; g < n; ++g)
      for (int a = 0; a < 3; ++a) c[a] += b[a * ps + g];
    for (int a = 0; a < 3; ++a) c[a] /= (n > 0 ? n : 1);
    double r = 0;
    for (int64_t g = 0; g < n; ++g) {
      double d2 = 0, smax = 0;
      for (int a = 0; a < 3; ++a) {
        const double d = b[a * ps + g] - c[a];
        d2 += d * d;
        smax = std::max(smax, (double)b[(3 + a) * ps + g]);
      }
      r = std::max(r, std::sqrt(d2) + 3.0 * smax);
    }
    for (int a = 0; a < 3; ++a) S->centroid[4 * p + a] = (float)c[a];
    S->centroid[4 * p + 3] = (float)r;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t p = 0; p < NP; ++p)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], (double)S->centroid[4 * p + a]);
      hi[a] = std::max(hi[a], (double)S->centroid[4 * p + a]);
    }
  double half = 0;
  for (int a = 0; a < 3; ++a) {
    S->box_center[a] = NP ? (float)(0.5 * (lo[a] + hi[a])) : 0.0f;
    half = std::max(half, NP ? 0.5 * (hi[a] - lo[a]) : 0.0);
  }
  S->box_half = (float)(half > 0 ? half : 1.0);
}
}  // namespace vm

vm3dgs_scene::~vm3dgs_scene() {
  // (VQ records are built in host memory, for mapped scenes too)
  if (registered_vq && data_vq) cudaHostUnregister(data_vq);
  std::free(data_vq);
  if (mapped) {
    if (map_base) munmap(map_base, map_len);
    return;
  }
  if (registered32 && data32) cudaHostUnregister(data32);
  if (registered16 && data16) cudaHostUnregister(data16);
  std::free(data32);
  std::free(data16);
}

// ---------------------------------------------------------------- scene files
// Layout: FileHeader, then the arrays count, src, err, verts, tris, face_page,
// link_ptr, link_col, centroid in that order; the fp32 page data at a
// 4096-aligned offset, then the fp16 page data (if built) at the next one.
namespace {
constexpr char kMagic[8] = {'V', 'M', '3', 'D', 'G', 'S', 'f', '1'};
struct FileHeader {
  char magic[8];
  int32_t n_pages, page_size, levels, fanout, sh_degree, K, rec32, rec16;
  int64_t n_gauss, bytes32, bytes16;
  int64_t off32[vm::kMaxLevels], off16[vm::kMaxLevels];
  int64_t n_count, n_src, n_err, n_verts, n_tris, n_face, n_lptr, n_lcol, n_centroid;
  float box_center[3], box_half;
  int64_t data32_at, data16_at, file_bytes;
};
int64_t align4k(int64_t x) { return (x + 4095) / 4096 * 4096; }
// pread until `bytes` have arrived (one call returns at most about 2 GB)
bool pread_all(int fd, void *dst, int64_t bytes, int64_t at) {
  auto *p = static_cast<uint8_t *>(dst);
  while (bytes > 0) {
    const ssize_t got = pread(fd, p, (size_t)std::min<int64_t>(bytes, int64_t(1) << 30), (off_t)at);
    if (got <= 0) return false;
    p += got;
    at += got;
    bytes -= got;
  }
  return true;
}
}  // namespace

extern "C" int vm3dgs_scene_save(const vm3dgs_scene *s, const char *path) {
  if (!s || !path) return vm::fail(VM3DGS_E_INVAL, "null argument");
  FileHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.n_pages = s->n_pages; h.page_size = s->page_size; h.levels = s->levels; h.fanout = s->fanout;
  h.sh_degree = s->sh_degree; h.K = s->K; h.rec32 = s->rec32; h.rec16 = s->rec16;
  h.n_gauss = s->n_gauss; h.bytes32 = s->bytes32; h.bytes16 = s->data16 ? s->bytes16 : 0;
  for (int l = 0; l < vm::kMaxLevels; ++l) { h.off32[l] = s->off32[l]; h.off16[l] = s->off16[l]; }
  h.n_count = (int64_t)s->count.size(); h.n_src = (int64_t)s->src.size(); h.n_err = (int64_t)s->err.size();
  h.n_verts = (int64_t)s->verts.size(); h.n_tris = (int64_t)s->tris.size(); h.n_face = (int64_t)s->face_page.size();
  h.n_lptr = (int64_t)s->link_ptr.size(); h.n_lcol = (int64_t)s->link_col.size();
  h.n_centroid = (int64_t)s->centroid.size();
  for (int a = 0; a < 3; ++a) h.box_center[a] = s->box_center[a];
  h.box_half = s->box_half;
  const int64_t arrays = 8 * (h.n_count + h.n_src) + 4 * (h.n_err + h.n_verts + h.n_tris + h.n_face) + 8 * h.n_lptr +
                         4 * (h.n_lcol + h.n_centroid);
  h.data32_at = align4k((int64_t)sizeof(FileHeader) + arrays);
  h.data16_at = align4k(h.data32_at + h.bytes32);
  h.file_bytes = h.bytes16 > 0 ? h.data16_at + h.bytes16 : h.data32_at + h.bytes32;
  FILE *f = std::fopen(path, "wb");
  if (!f) return vm::fail(VM3DGS_E_INVAL, std::string("cannot create ") + path);
  bool ok = std::fwrite(&h, sizeof h, 1, f) == 1;
  auto put = [&](const void *p, int64_t n) { if (ok && n > 0) ok = std::fwrite(p, 1, (size_t)n, f) == (size_t)n; };
  put(s->count.data(), 8 * h.n_count);
  put(s->src.data(), 8 * h.n_src);
  put(s->err.data(), 4 * h.n_err);
  put(s->verts.data(), 4 * h.n_verts);
  put(s->tris.data(), 4 * h.n_tris);
  put(s->face_page.data(), 4 * h.n_face);
  put(s->link_ptr.data(), 8 * h.n_lptr);
  put(s->link_col.data(), 4 * h.n_lcol);
  put(s->centroid.data(), 4 * h.n_centroid);
  ok = ok && std::fseek(f, (long)h.data32_at, SEEK_SET) == 0;
  put(s->data32, h.bytes32);
  if (h.bytes16 > 0) {
    ok = ok && std::fseek(f, (long)h.data16_at, SEEK_SET) == 0;
    put(s->data16, h.bytes16);
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return vm::fail(VM3DGS_E_INVAL, std::string("write failed: ") + path);
  return VM3DGS_OK;
}

extern "C" int vm3dgs_scene_open(const char *path, vm3dgs_scene **out) {
  if (!path || !out) return vm::fail(VM3DGS_E_INVAL, "null argument");
  *out = nullptr;
  const int fd = ::open(path, O_RDONLY);
  if (fd < 0) return vm::fail(VM3DGS_E_INVAL, std::string("cannot open ") + path);
  struct stat sb{};
  FileHeader h{};
  const bool head = fstat(fd, &sb) == 0 && pread_all(fd, &h, (int64_t)sizeof h, 0);
  auto bad = [&](const char *why) {
    ::close(fd);
    return vm::fail(VM3DGS_E_INVAL, std::string("not a scene file (") + why + "): " + path);
  };
  if (!head || std::memcmp(h.magic, kMagic, 8) != 0) return bad("header");
  if (h.n_pages <= 0 || h.page_size <= 0 || h.levels < 1 || h.levels > vm::kMaxLevels || h.fanout < 2 ||
      h.sh_degree < 0 || h.sh_degree > 3 || h.K != (h.sh_degree + 1) * (h.sh_degree + 1) ||
      h.rec32 != vm::rec_bytes32(h.K) || (h.bytes16 > 0 && h.rec16 != vm::rec_bytes16(h.K)) ||
      h.n_count != h.n_pages || h.n_src != (int64_t)h.n_pages * h.page_size ||
      h.n_err != (int64_t)h.n_pages * h.levels || h.n_lptr != h.n_pages + 1 || h.n_tris != 3 * h.n_face ||
      h.n_verts % 3 || h.n_centroid != 4 * (int64_t)h.n_pages || h.bytes32 <= 0 || h.bytes16 < 0 ||
      h.data32_at % 4096 || h.data16_at % 4096 || h.file_bytes != (int64_t)sb.st_size ||
      h.data32_at + h.bytes32 > h.file_bytes || (h.bytes16 > 0 && h.data16_at + h.bytes16 > h.file_bytes))
    return bad("fields");
  auto *S = new (std::nothrow) vm3dgs_scene;
  if (!S) { ::close(fd); return vm::fail(VM3DGS_E_NOMEM, "scene"); }
  S->n_pages = h.n_pages; S->page_size = h.page_size; S->levels = h.levels; S->fanout = h.fanout;
  S->sh_degree = h.sh_degree; S->K = h.K; S->rec32 = h.rec32; S->rec16 = h.bytes16 > 0 ? h.rec16 : 0;
  S->n_gauss = h.n_gauss; S->bytes32 = h.bytes32; S->bytes16 = h.bytes16;
  for (int l = 0; l < vm::kMaxLevels; ++l) { S->off32[l] = h.off32[l]; S->off16[l] = h.off16[l]; }
  for (int a = 0; a < 3; ++a) S->box_center[a] = h.box_center[a];
  S->box_half = h.box_half;
  int64_t at = (int64_t)sizeof h;
  bool ok = true;
  auto get = [&](auto &vec, int64_t n) {
    vec.resize((size_t)n);
    const int64_t bytes = n * (int64_t)sizeof(vec[0]);
    if (ok && bytes > 0) ok = pread_all(fd, vec.data(), bytes, at);
    at += bytes;
  };
  get(S->count, h.n_count);
  get(S->src, h.n_src);
  get(S->err, h.n_err);
  get(S->verts, h.n_verts);
  get(S->tris, h.n_tris);
  get(S->face_page, h.n_face);
  get(S->link_ptr, h.n_lptr);
  get(S->link_col, h.n_lcol);
  get(S->centroid, h.n_centroid);
  if (!ok || at > h.data32_at) { delete S; ::close(fd); return vm::fail(VM3DGS_E_INVAL, "short scene file"); }
  void *base = mmap(nullptr, (size_t)h.file_bytes, PROT_READ, MAP_SHARED, fd, 0);
  ::close(fd);
  if (base == MAP_FAILED) { delete S; return vm::fail(VM3DGS_E_NOMEM, "mmap of the scene file failed"); }
  S->mapped = true;
  S->map_base = base;
  S->map_len = (size_t)h.file_bytes;
  S->data32 = (uint8_t *)base + h.data32_at;
  S->data16 = h.bytes16 > 0 ? (uint8_t *)base + h.data16_at : nullptr;
  *out = S;
  return VM3DGS_OK;
}

extern "C" const char *vm3dgs_last_error(void) { return vm::g_last_error.c_str(); }
extern "C" const char *vm3dgs_version(void) { return "vm3dgs 0.1 sm_103a"; }

extern "C" void vm3dgs_scene_destroy(vm3dgs_scene *s) { delete s; }

extern "C" int vm3dgs_scene_info_get(const vm3dgs_scene *s, vm3dgs_scene_info *o) {
  if (!s || !o) return vm::fail(VM3DGS_E_INVAL, "null argument");
  o->n_pages = s->n_pages;
  o->page_size = s->page_size;
  o->lod_levels = s->levels;
  o->lod_fanout = s->fanout;
  o->sh_degree = s->sh_degree;
  o->n_gaussians = s->n_gauss;
  o->record_bytes = s->rec32;
  o->record_bytes16 = s->rec16;
  o->n_tris = (int64_t)s->face_page.size();
  o->n_verts = (int64_t)s->verts.size() / 3;
  o->n_links = (int64_t)s->link_col.size();
  o->host_bytes = s->bytes32 + s->bytes16 + s->bytes_vq;
  o->record_bytes_vq = s->data_vq ? s->rec_vq : 0;
  o->n_codes = s->data_vq ? s->n_codes : 0;
  return VM3DGS_OK;
}

namespace {
int copy_out(const void *src, int64_t n, void *dst, int64_t bytes, int64_t *needed) {
  if (needed) *needed = n;
  if (!dst) return VM3DGS_OK;
  if (bytes < n) return vm::fail(VM3DGS_E_CAPACITY, "destination too small");
  if (n) std::memcpy(dst, src, (size_t)n);
  return VM3DGS_OK;
}
}  // namespace

extern "C" int vm3dgs_scene_export(const vm3dgs_scene *s, int32_t what, int32_t level, void *dst, int64_t bytes,
                                   int64_t *needed) {
  if (!s) return vm::fail(VM3DGS_E_INVAL, "null scene");
  if (level < 0 || level >= s->levels) return vm::fail(VM3DGS_E_INVAL, "level out of range");
  const int64_t NP = s->n_pages;
  switch (what) {
    case VM3DGS_SCENE_PAGE_COUNT: return copy_out(s->count.data(), 8 * NP, dst, bytes, needed);
    case VM3DGS_SCENE_PAGE_SRC: return copy_out(s->src.data(), 8 * (int64_t)s->src.size(), dst, bytes, needed);
    case VM3DGS_SCENE_PAGES:
      return copy_out(s->data32 + s->off32[level], NP * s->m(level) * (int64_t)s->rec32, dst, bytes, needed);
    case VM3DGS_SCENE_PAGES16:
      if (!s->data16) return vm::fail(VM3DGS_E_STATE, "scene built without fp16 records");
      return copy_out(s->data16 + s->off16[level], NP * s->m(level) * (int64_t)s->rec16, dst, bytes, needed);
    case VM3DGS_SCENE_ERR: return copy_out(s->err.data(), 4 * (int64_t)s->err.size(), dst, bytes, needed);
    case VM3DGS_SCENE_VERTS: return copy_out(s->verts.data(), 4 * (int64_t)s->verts.size(), dst, bytes, needed);
    case VM3DGS_SCENE_TRIS: return copy_out(s->tris.data(), 4 * (int64_t)s->tris.size(), dst, bytes, needed);
    case VM3DGS_SCENE_FACE_PAGE:
      return copy_out(s->face_page.data(), 4 * (int64_t)s->face_page.size(), dst, bytes, needed);
    case VM3DGS_SCENE_LINK_PTR: return copy_out(s->link_ptr.data(), 8 * (int64_t)s->link_ptr.size(), dst, bytes, needed);
    case VM3DGS_SCENE_LINK_COL: return copy_out(s->link_col.data(), 4 * (int64_t)s->link_col.size(), dst, bytes, needed);
    case VM3DGS_SCENE_CODEBOOK:
      if (!s->data_vq) return vm::fail(VM3DGS_E_STATE, "scene has no SH codebook");
      return copy_out(s->codebook.data(), 4 * (int64_t)s->codebook.size(), dst, bytes, needed);
    case VM3DGS_SCENE_PAGES_VQ:
      if (!s->data_vq) return vm::fail(VM3DGS_E_STATE, "scene has no VQ records");
      return copy_out(s->data_vq + s->off_vq[level], NP * s->m(level) * (int64_t)s->rec_vq, dst, bytes, needed);
    default: return vm::fail(VM3DGS_E_INVAL, "unknown export item");
  }
}

namespace {
uint16_t to_half(float f) {
  // IEEE binary32 -> binary16, round to nearest even
  uint32_t x;
  std::memcpy(&x, &f, 4);
  uint32_t sign = (x >> 16) & 0x8000u, mant = x & 0x7FFFFFu;
  int exp = (int)((x >> 23) & 0xFF);
  if (exp == 0xFF) return (uint16_t)(sign | 0x7C00u | (mant ? 0x200u : 0));
  int e = exp - 127 + 15;
  if (e >= 31) return (uint16_t)(sign | 0x7C00u);
  if (e <= 0) {
    if (e < -10) return (uint16_t)sign;
    mant |= 0x800000u;
    int shift = 14 - e;
    uint32_t h = mant >> shift, rem = mant & ((1u << shift) - 1), half = 1u << (shift - 1);
    if (rem > half || (rem == half && (h & 1))) ++h;
    return (uint16_t)(sign | h);
  }
  uint32_t h = ((uint32_t)e << 10) | (mant >> 13), rem = mant & 0x1FFFu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1))) ++h;
  return (uint16_t)(sign | h);
}
}  // namespace

extern "C" int vm3dgs_scene_import(const vm3dgs_scene_desc *d, vm3dgs_scene **out) {
  using namespace vm;
  if (!d || !out) return fail(VM3DGS_E_INVAL, "null argument");
  *out = nullptr;
  if (d->n_pages <= 0 || d->page_size <= 0 || d->lod_levels < 1 || d->lod_levels > kMaxLevels || d->lod_fanout < 2 ||
      d->sh_degree < 0 || d->sh_degree > 3 || !d->pos || !d->scale || !d->rot || !d->opacity || !d->sh || !d->err ||
      !d->count || !d->link_ptr || (d->n_tris > 0 && (!d->verts || !d->tris || !d->face_page)))
    return fail(VM3DGS_E_INVAL, "bad scene description");
  auto *S = new (std::nothrow) vm3dgs_scene();
  if (!S) return fail(VM3DGS_E_NOMEM, "scene");
  const int K = (d->sh_degree + 1) * (d->sh_degree + 1), NA = n_attr32(K);
  S->n_pages = d->n_pages; S->page_size = d->page_size; S->levels = d->lod_levels; S->fanout = d->lod_fanout;
  S->sh_degree = d->sh_degree; S->K = K;
  S->rec32 = rec_bytes32(K); S->rec16 = d->fp16 ? rec_bytes16(K) : 0;
  const int64_t NP = d->n_pages;
  S->count.assign(d->count, d->count + NP);
  S->n_gauss = 0;
  for (int64_t p = 0; p < NP; ++p) S->n_gauss += S->count[p];
  S->src.assign(NP * d->page_size, -1);
  int64_t total = 0;
  for (int l = 0; l < S->levels; ++l) { S->off32[l] = total; total += NP * (int64_t)S->m(l) * S->rec32; }
  S->bytes32 = total;
  S->data32 = (uint8_t *)std::aligned_alloc(4096, (size_t)((total + 4095) / 4096 * 4096));
  if (!S->data32) { delete S; return fail(VM3DGS_E_NOMEM, "page data"); }
  for (int l = 0; l < S->levels; ++l) {
    const int64_t m = S->m(l);
    for (int64_t p = 0; p < NP; ++p) {
      float *blk = (float *)(S->data32 + S->off32[l]) + p * m * NA;
      for (int64_t g = 0; g < m; ++g) {
        const int64_t i = p * m + g;
        for (int a = 0; a < 3; ++a) blk[a * m + g] = d->pos[l][3 * i + a];
        for (int a = 0; a < 3; ++a) blk[(3 + a) * m + g] = d->scale[l][3 * i + a];
        for (int a = 0; a < 4; ++a) blk[(6 + a) * m + g] = d->rot[l][4 * i + a];
        blk[10 * m + g] = d->opacity[l][i];
        for (int k = 0; k < 3 * K; ++k) blk[(11 + k) * m + g] = d->sh[l][(size_t)i * 3 * K + k];
      }
    }
  }
  if (d->fp16) {
    const int NH = n_half16(K);
    int64_t t16 = 0;
    for (int l = 0; l < S->levels; ++l) { S->off16[l] = t16; t16 += NP * (int64_t)S->m(l) * S->rec16; }
    S->bytes16 = t16;
    S->data16 = (uint8_t *)std::aligned_alloc(4096, (size_t)((t16 + 4095) / 4096 * 4096));
    if (!S->data16) { delete S; return fail(VM3DGS_E_NOMEM, "fp16 page data"); }
    for (int l = 0; l < S->levels; ++l) {
      const int64_t m = S->m(l);
      for (int64_t p = 0; p < NP; ++p) {
        const float *src = (const float *)(S->data32 + S->off32[l]) + p * m * NA;
        uint8_t *dst = S->data16 + S->off16[l] + p * m * S->rec16;
        float *f = (float *)dst;
        uint16_t *h = (uint16_t *)(dst + 16 * m);
        for (int64_t g = 0; g < m; ++g) {
          for (int a = 0; a < 3; ++a) f[a * m + g] = src[a * m + g];
          f[3 * m + g] = src[10 * m + g];
          for (int a = 0; a < 3; ++a) h[a * m + g] = to_half(src[(3 + a) * m + g]);
          for (int a = 0; a < 4; ++a) h[(3 + a) * m + g] = to_half(src[(6 + a) * m + g]);
          for (int k = 0; k < 3 * K; ++k) h[(7 + k) * m + g] = to_half(src[(11 + k) * m + g]);
          for (int k = 7 + 3 * K; k < NH; ++k) h[k * m + g] = 0;
        }
      }
    }
  }
  S->err.assign(d->err, d->err + NP * S->levels);
  S->verts.assign(d->verts, d->verts + 3 * d->n_verts);
  S->tris.assign(d->tris, d->tris + 3 * d->n_tris);
  S->face_page.assign(d->face_page, d->face_page + d->n_tris);
  S->link_ptr.assign(d->link_ptr, d->link_ptr + NP + 1);
  if (S->link_ptr[NP] != d->n_links) { delete S; return fail(VM3DGS_E_INVAL, "link_ptr does not end at n_links"); }
  S->link_col.assign(d->link_col, d->link_col + d->n_links);
  for (int64_t t = 0; t < d->n_tris; ++t) {
    for (int k = 0; k < 3; ++k)
      if (S->tris[3 * t + k] < 0 || S->tris[3 * t + k] >= d->n_verts) { delete S; return fail(VM3DGS_E_INVAL, "triangle index"); }
    if (S->face_page[t] < -1 || S->face_page[t] >= NP) { delete S; return fail(VM3DGS_E_INVAL, "face page out of range"); }
  }
  for (int64_t k = 0; k < d->n_links; ++k)
    if (S->link_col[k] < 0 || S->link_col[k] >= NP) { delete S; return fail(VM3DGS_E_INVAL, "link column out of range"); }
  finish_scene(S);
  *out = S;
  return VM3DGS_OK;
}
