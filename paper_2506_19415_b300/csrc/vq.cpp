// Compressed pages: vector quantisation of the view-dependent spherical
// harmonics into a codebook kept in GPU memory (Sec. 6 names codebooks of
// quantised attributes in GPU memory as future work, to copy less data per
// page; Sec. 2, Compression, names k-means quantisation of the SH).
//
//   training  the real (opacity > 0) level-0 Gaussians in slot order, or the
//             n_train of them at positions floor(j T / n_train)
//   codebook  Lloyd's iterations from the training vectors at positions
//             floor(j T' / n_codes): nearest codeword (squared Euclidean
//             distance in FP64, features summed in order, lowest index on a
//             tie), then each codeword to the mean of its vectors (summed in
//             training order; one without vectors stays); at most `iters`
//             rounds, ending early when an assignment repeats; rounded to fp32
//   codes     every Gaussian of every level takes the nearest fp32 codeword
//   records   the VQ record of scene.h (40 bytes), built from the fp32 pages
// The distance loops run along the codewords (codebook stored feature-major),
// so vectorising them leaves every sum in its order: the codebook and codes
// equal the oracle's bit for bit.
#include <omp.h>

#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "scene.h"

namespace {

// Nearest codeword of rows [i0, i1) of X ([n][D]); C is feature-major [D][k].
template <int D>
__attribute__((target_clones("avx2", "default"))) void nearest_rows(const double *__restrict X, int64_t i0,
                                                                    int64_t i1, const double *__restrict C, int k,
                                                                    double *__restrict dist, int32_t *__restrict lab) {
  for (int64_t i = i0; i < i1; ++i) {
    const double *x = X + (size_t)i * D;
    for (int j = 0; j < k; ++j) dist[j] = 0.0;
    for (int a = 0; a < D; ++a) {
      const double xa = x[a];
      const double *__restrict ca = C + (size_t)a * k;
      for (int j = 0; j < k; ++j) {
        const double t = xa - ca[j];
        dist[j] += t * t;
      }
    }
    int best = 0;
    for (int j = 1; j < k; ++j)
      if (dist[j] < dist[best]) best = j;
    lab[i] = best;
  }
}

template <int D>
void nearest_all(const double *X, int64_t n, const double *C, int k, int32_t *lab) {
#pragma omp parallel
  {
    std::vector<double> dist((size_t)k);
    const int nt = omp_get_num_threads(), t = omp_get_thread_num();
    // contiguous blocks of 256 rows dealt out in turn
    for (int64_t b = (int64_t)t * 256; b < n; b += (int64_t)nt * 256)
      nearest_rows<D>(X, b, b + 256 < n ? b + 256 : n, C, k, dist.data(), lab);
  }
}

void nearest(int D, const double *X, int64_t n, const double *C, int k, int32_t *lab) {
  switch (D) {
    case 9: nearest_all<9>(X, n, C, k, lab); break;
    case 24: nearest_all<24>(X, n, C, k, lab); break;
    default: nearest_all<45>(X, n, C, k, lab); break;
  }
}

// The SH bands 1..3 of Gaussian g of a level block (fp32 SoA, attribute row
// 11 + 3 k + c) into x[3 (k - 1) + c].
inline void rest_of(const float *blk, int64_t m, int64_t g, int K, double *x) {
  for (int d = 0; d < 3 * (K - 1); ++d) x[d] = (double)blk[(11 + 3 + d) * m + g];
}

}  // namespace

extern "C" int vm3dgs_scene_quantize_sh(vm3dgs_scene *s, int32_t n_codes, int32_t iters, int64_t n_train) {
  using namespace vm;
  if (!s) return fail(VM3DGS_E_INVAL, "null scene");
  if (s->K < 2) return fail(VM3DGS_E_INVAL, "SH degree 0: no view-dependent coefficients to quantise");
  if (n_codes < 1 || n_codes > 65536) return fail(VM3DGS_E_INVAL, "n_codes must be 1..65536");
  if (iters < 0 || n_train < 1) return fail(VM3DGS_E_INVAL, "iters must be >= 0 and n_train >= 1");
  if (s->data_vq) return fail(VM3DGS_E_STATE, "the scene already holds VQ records");
  const int K = s->K, D = 3 * (K - 1), NA = n_attr32(K);
  const int64_t NP = s->n_pages, m0 = s->m(0);
  // ---- training set
  const float *L0 = (const float *)(s->data32 + s->off32[0]);
  std::vector<int64_t> real;  // (page, slot) in slot order as p * m0 + g
  for (int64_t p = 0; p < NP; ++p)
    for (int64_t g = 0; g < m0; ++g)
      if (L0[p * m0 * NA + 10 * m0 + g] > 0) real.push_back(p * m0 + g);
  const int64_t T = (int64_t)real.size(), nt = T < n_train ? T : n_train;
  if (nt < n_codes) return fail(VM3DGS_E_INVAL, "fewer training Gaussians than codes");
  std::vector<double> X;
  try {
    X.resize((size_t)(nt * D));
  } catch (const std::bad_alloc &) {
    return fail(VM3DGS_E_NOMEM, "training set");
  }
  for (int64_t j = 0; j < nt; ++j) {
    const int64_t pg = real[(size_t)(j * T / nt)], p = pg / m0, g = pg % m0;
    rest_of(L0 + p * m0 * NA, m0, g, K, &X[(size_t)(j * D)]);
  }
  // ---- Lloyd's iterations (codebook feature-major [D][k])
  const int k = n_codes;
  std::vector<double> C((size_t)D * k), acc((size_t)D * k);
  for (int j = 0; j < k; ++j) {
    const double *x = &X[(size_t)(((int64_t)j * nt / k) * D)];
    for (int a = 0; a < D; ++a) C[(size_t)a * k + j] = x[a];
  }
  std::vector<int32_t> lab((size_t)nt), prev((size_t)nt), cnt((size_t)k);
  for (int it = 0; it < iters; ++it) {
    nearest(D, X.data(), nt, C.data(), k, lab.data());
    if (it > 0 && lab == prev) break;
    std::fill(acc.begin(), acc.end(), 0.0);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t i = 0; i < nt; ++i) {
      const int j = lab[(size_t)i];
      ++cnt[(size_t)j];
      for (int a = 0; a < D; ++a) acc[(size_t)a * k + j] += X[(size_t)(i * D + a)];
    }
    for (int j = 0; j < k; ++j)
      if (cnt[(size_t)j] > 0)
        for (int a = 0; a < D; ++a) C[(size_t)a * k + j] = acc[(size_t)a * k + j] / cnt[(size_t)j];
    prev = lab;
  }
  // ---- the fp32 codebook (row-major for the renderer; feature-major FP64
  // copy of the rounded values for the codes)
  std::vector<float> cb((size_t)k * D);
  for (int j = 0; j < k; ++j)
    for (int a = 0; a < D; ++a) {
      cb[(size_t)j * D + a] = (float)C[(size_t)a * k + j];
      C[(size_t)a * k + j] = (double)cb[(size_t)j * D + a];
    }
  // ---- codes and VQ records, level by level
  const int rec = rec_bytes_vq();
  int64_t off[kMaxLevels] = {0}, total = 0;
  for (int l = 0; l < s->levels; ++l) { off[l] = total; total += NP * (int64_t)s->m(l) * rec; }
  auto *data = (uint8_t *)std::aligned_alloc(4096, (size_t)((total + 4095) / 4096 * 4096));
  if (!data) return fail(VM3DGS_E_NOMEM, "VQ page data");
  for (int l = 0; l < s->levels; ++l) {
    const int64_t m = s->m(l);
    const float *Ll = (const float *)(s->data32 + s->off32[l]);
    // pages in chunks of about 2^20 Gaussians (their vectors in FP64)
    const int64_t chunk = (int64_t(1) << 20) / m > 0 ? (int64_t(1) << 20) / m : 1;
    std::vector<double> Xl;
    std::vector<int32_t> code;
    try {
      Xl.resize((size_t)(chunk * m * D));
      code.resize((size_t)(chunk * m));
    } catch (const std::bad_alloc &) {
      std::free(data);
      return fail(VM3DGS_E_NOMEM, "codes");
    }
    for (int64_t p0 = 0; p0 < NP; p0 += chunk) {
      const int64_t np = NP - p0 < chunk ? NP - p0 : chunk, n = np * m;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) rest_of(Ll + (p0 + i / m) * m * NA, m, i % m, K, &Xl[(size_t)(i * D)]);
      nearest(D, Xl.data(), n, C.data(), k, code.data());
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < np; ++q) {
        const int64_t p = p0 + q;
        const float *src = Ll + p * m * NA;
        uint8_t *dst = data + off[l] + p * m * rec;
        float *f = (float *)dst;
        uint16_t *h = (uint16_t *)(dst + 16 * m);
        for (int64_t g = 0; g < m; ++g) {
          for (int a = 0; a < 3; ++a) f[a * m + g] = src[a * m + g];
          f[3 * m + g] = src[10 * m + g];
          for (int a = 0; a < 3; ++a) h[a * m + g] = f32_to_f16(src[(3 + a) * m + g]);
          for (int a = 0; a < 4; ++a) h[(3 + a) * m + g] = f32_to_f16(src[(6 + a) * m + g]);
          for (int c = 0; c < 3; ++c) h[(7 + c) * m + g] = f32_to_f16(src[(11 + c) * m + g]);
          h[10 * m + g] = (uint16_t)code[(size_t)(q * m + g)];
          h[11 * m + g] = 0;
        }
      }
    }
  }
  s->registered_vq = false;
  s->data_vq = data;
  s->bytes_vq = total;
  for (int l = 0; l < kMaxLevels; ++l) s->off_vq[l] = l < s->levels ? off[l] : 0;
  s->rec_vq = rec;
  s->n_codes = k;
  s->code_dim = D;
  s->codebook.swap(cb);
  return VM3DGS_OK;
}
