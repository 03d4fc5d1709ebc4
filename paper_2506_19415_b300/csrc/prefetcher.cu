// C ABI of the learned prefetcher: device memory layout, initialisation,
// forward pass, one training step (forward, binary cross-entropy with logits
// over unmasked outputs, backward, Adam), weight and gradient exchange.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mlp.cuh"
#include "prefetcher.cuh"
#include "scene.h"

namespace vm {
namespace {
int64_t al(int64_t x) { return (x + 255) & ~int64_t(255); }

uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

bool ok(cudaError_t e, const char *what, int *rc) {
  if (e == cudaSuccess) return true;
  *rc = fail(VM3DGS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return false;
}
}  // namespace

PfLayout pf_layout(const vm3dgs_mlp_config &c) {
  PfLayout L{};
  const int64_t I = c.n_in, H = c.n_hidden, O = c.n_out, B = c.max_batch;
  L.n_w1 = I * H; L.n_b1 = H; L.n_w2 = H * H; L.n_b2 = H; L.n_w3 = H * O; L.n_b3 = O;
  L.n_params = L.n_w1 + L.n_b1 + L.n_w2 + L.n_b2 + L.n_w3 + L.n_b3;
  int64_t o = 0;
  auto take = [&](int64_t bytes) { int64_t r = o; o = al(o + (bytes > 0 ? bytes : 1)); return r; };
  L.w = take(4 * L.n_params);       // fp32 master weights, packed W1 b1 W2 b2 W3 b3
  L.g = take(4 * L.n_params);       // gradients, same packing
  L.m = take(4 * L.n_params);
  L.v = take(4 * L.n_params);
  L.w1b = take(2 * L.n_w1);
  L.w2b = take(2 * L.n_w2);
  L.w3b = take(2 * L.n_w3);
  L.xb = take(2 * B * I);
  L.h1f = take(4 * B * H);
  L.h1b = take(2 * B * H);
  L.h2f = take(4 * B * H);
  L.h2b = take(2 * B * H);
  L.logits = take(4 * B * O);
  L.dy = take(4 * B * O);
  L.dyb = take(2 * B * O);
  L.dz2 = take(4 * B * H);
  L.dz2b = take(2 * B * H);
  L.dz1 = take(4 * B * H);
  L.dz1b = take(2 * B * H);
  L.loss = take(16);
  L.feat = take(4 * I);
  L.total = o;
  return L;
}

void pf_forward(vm3dgs_prefetcher *p, const float *x, int Bn, float *logits, cudaStream_t st) {
  const PfLayout &L = p->lay;
  const int I = p->cfg.n_in, H = p->cfg.n_hidden, O = p->cfg.n_out;
  float *w = p->at<float>(L.w);
  launch_to_bf16(x, p->at<__nv_bfloat16>(L.xb), (int64_t)Bn * I, st);
  GemmArgs g{};
  // layer 1: h1 = relu(x W1 + b1)
  g = GemmArgs{Bn, H, I, p->at<__nv_bfloat16>(L.xb), I, 0, p->at<__nv_bfloat16>(L.w1b), H, 0, w + L.n_w1, 1, nullptr,
               p->at<float>(L.h1f), p->at<__nv_bfloat16>(L.h1b), H};
  (Bn == 1 ? launch_gemv : launch_gemm)(g, st);
  // layer 2
  g = GemmArgs{Bn, H, H, p->at<__nv_bfloat16>(L.h1b), H, 0, p->at<__nv_bfloat16>(L.w2b), H, 0,
               w + L.n_w1 + L.n_b1 + L.n_w2, 1, nullptr, p->at<float>(L.h2f), p->at<__nv_bfloat16>(L.h2b), H};
  (Bn == 1 ? launch_gemv : launch_gemm)(g, st);
  // output logits
  g = GemmArgs{Bn, O, H, p->at<__nv_bfloat16>(L.h2b), H, 0, p->at<__nv_bfloat16>(L.w3b), O, 0,
               w + L.n_w1 + L.n_b1 + L.n_w2 + L.n_b2 + L.n_w3, 0, nullptr, logits, nullptr, O};
  (Bn == 1 ? launch_gemv : launch_gemm)(g, st);
}

}  // namespace vm

using namespace vm;

extern "C" int vm3dgs_prefetcher_bytes(const vm3dgs_mlp_config *c, int64_t *out) {
  if (!c || !out) return fail(VM3DGS_E_INVAL, "null argument");
  if (c->n_in <= 0 || c->n_hidden <= 0 || c->n_out <= 0 || c->max_batch <= 0)
    return fail(VM3DGS_E_INVAL, "bad network shape");
  *out = pf_layout(*c).total;
  return VM3DGS_OK;
}

extern "C" int vm3dgs_prefetcher_create(const vm3dgs_mlp_config *c, void *dev, int64_t bytes, void *stream,
                                        vm3dgs_prefetcher **out) {
  if (!c || !dev || !out) return fail(VM3DGS_E_INVAL, "null argument");
  *out = nullptr;
  int64_t need;
  int rc = vm3dgs_prefetcher_bytes(c, &need);
  if (rc) return rc;
  if (bytes < need) return fail(VM3DGS_E_CAPACITY, "prefetcher needs " + std::to_string(need) + " bytes");
  auto *p = new (std::nothrow) vm3dgs_prefetcher();
  if (!p) return fail(VM3DGS_E_NOMEM, "prefetcher");
  p->cfg = *c;
  p->lay = pf_layout(*c);
  p->mem = (uint8_t *)dev;
  cudaStream_t st = (cudaStream_t)stream;
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from SplitMix64(seed, index)
  const PfLayout &L = p->lay;
  std::vector<float> w(L.n_params, 0.0f);
  auto fill = [&](int64_t off, int64_t n, int fan_in) {
    const double a = 1.0 / std::sqrt((double)fan_in);
    for (int64_t i = 0; i < n; ++i) {
      const double u = (double)(sm64(c->seed ^ (uint64_t)(off + i)) >> 11) * (1.0 / 9007199254740992.0);
      w[off + i] = (float)((2.0 * u - 1.0) * a);
    }
  };
  fill(0, L.n_w1, c->n_in);
  fill(L.n_w1 + L.n_b1, L.n_w2, c->n_hidden);
  fill(L.n_w1 + L.n_b1 + L.n_w2 + L.n_b2, L.n_w3, c->n_hidden);
  bool good = ok(cudaMemsetAsync(p->mem, 0, (size_t)L.total, st), "memset", &rc);
  good = good && ok(cudaMemcpyAsync(p->at<void>(L.w), w.data(), 4 * L.n_params, cudaMemcpyHostToDevice, st), "copy", &rc);
  if (good) {
    float *wd = p->at<float>(L.w);
    launch_to_bf16(wd, p->at<__nv_bfloat16>(L.w1b), L.n_w1, st);
    launch_to_bf16(wd + L.n_w1 + L.n_b1, p->at<__nv_bfloat16>(L.w2b), L.n_w2, st);
    launch_to_bf16(wd + L.n_w1 + L.n_b1 + L.n_w2 + L.n_b2, p->at<__nv_bfloat16>(L.w3b), L.n_w3, st);
    good = ok(cudaStreamSynchronize(st), "sync", &rc);
  }
  if (!good) { delete p; return rc; }
  *out = p;
  return VM3DGS_OK;
}

extern "C" void vm3dgs_prefetcher_destroy(vm3dgs_prefetcher *p) { delete p; }

extern "C" int vm3dgs_prefetcher_forward(vm3dgs_prefetcher *p, const float *x_dev, int32_t batch, float *logits_dev,
                                         void *stream) {
  if (!p || !x_dev || !logits_dev) return fail(VM3DGS_E_INVAL, "null argument");
  if (batch <= 0 || batch > p->cfg.max_batch) return fail(VM3DGS_E_INVAL, "batch outside 1..max_batch");
  pf_forward(p, x_dev, batch, logits_dev, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, cudaGetErrorString(e));
}

extern "C" int vm3dgs_prefetcher_train_step(vm3dgs_prefetcher *p, const float *x_dev, const float *target_dev,
                                            const float *mask_dev, int32_t batch, float mask_sum, float *loss_dev,
                                            void *stream) {
  if (!p || !x_dev || !target_dev || !mask_dev) return fail(VM3DGS_E_INVAL, "null argument");
  if (batch <= 0 || batch > p->cfg.max_batch) return fail(VM3DGS_E_INVAL, "batch outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  const PfLayout &L = p->lay;
  const int I = p->cfg.n_in, H = p->cfg.n_hidden, O = p->cfg.n_out, Bn = batch;
  float *logits = p->at<float>(L.logits);
  pf_forward(p, x_dev, Bn, logits, st);
  float *loss = loss_dev ? loss_dev : p->at<float>(L.loss);
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  const float inv_n = 1.0f / (mask_sum > 1.0f ? mask_sum : 1.0f);
  launch_bce_grad(logits, target_dev, mask_dev, (int64_t)Bn * O, inv_n, p->at<float>(L.dy), p->at<__nv_bfloat16>(L.dyb),
                  loss, st);
  float *g = p->at<float>(L.g);
  float *gW1 = g, *gb1 = g + L.n_w1, *gW2 = gb1 + L.n_b1, *gb2 = gW2 + L.n_w2, *gW3 = gb2 + L.n_b2, *gb3 = gW3 + L.n_w3;
  // output layer
  launch_gemm(GemmArgs{H, O, Bn, p->at<__nv_bfloat16>(L.h2b), H, 1, p->at<__nv_bfloat16>(L.dyb), O, 0, nullptr, 0,
                       nullptr, gW3, nullptr, O}, st);
  launch_colsum(p->at<float>(L.dy), Bn, O, gb3, st);
  launch_gemm(GemmArgs{Bn, H, O, p->at<__nv_bfloat16>(L.dyb), O, 0, p->at<__nv_bfloat16>(L.w3b), O, 1, nullptr, 0,
                       p->at<float>(L.h2f), p->at<float>(L.dz2), p->at<__nv_bfloat16>(L.dz2b), H}, st);
  // hidden layer 2
  launch_gemm(GemmArgs{H, H, Bn, p->at<__nv_bfloat16>(L.h1b), H, 1, p->at<__nv_bfloat16>(L.dz2b), H, 0, nullptr, 0,
                       nullptr, gW2, nullptr, H}, st);
  launch_colsum(p->at<float>(L.dz2), Bn, H, gb2, st);
  launch_gemm(GemmArgs{Bn, H, H, p->at<__nv_bfloat16>(L.dz2b), H, 0, p->at<__nv_bfloat16>(L.w2b), H, 1, nullptr, 0,
                       p->at<float>(L.h1f), p->at<float>(L.dz1), p->at<__nv_bfloat16>(L.dz1b), H}, st);
  // hidden layer 1
  launch_gemm(GemmArgs{I, H, Bn, p->at<__nv_bfloat16>(L.xb), I, 1, p->at<__nv_bfloat16>(L.dz1b), H, 0, nullptr, 0,
                       nullptr, gW1, nullptr, H}, st);
  launch_colsum(p->at<float>(L.dz1), Bn, H, gb1, st);
  // Adam
  p->step += 1;
  const vm3dgs_mlp_config &c = p->cfg;
  float *w = p->at<float>(L.w), *m = p->at<float>(L.m), *v = p->at<float>(L.v);
  const int64_t offs[6] = {0, L.n_w1, L.n_w1 + L.n_b1, L.n_w1 + L.n_b1 + L.n_w2, L.n_w1 + L.n_b1 + L.n_w2 + L.n_b2,
                           L.n_w1 + L.n_b1 + L.n_w2 + L.n_b2 + L.n_w3};
  const int64_t sizes[6] = {L.n_w1, L.n_b1, L.n_w2, L.n_b2, L.n_w3, L.n_b3};
  __nv_bfloat16 *copies[6] = {p->at<__nv_bfloat16>(L.w1b), nullptr, p->at<__nv_bfloat16>(L.w2b), nullptr,
                              p->at<__nv_bfloat16>(L.w3b), nullptr};
  if (c.lr > 0.0f)
    for (int k = 0; k < 6; ++k)
      launch_adam(w + offs[k], g + offs[k], m + offs[k], v + offs[k], copies[k], sizes[k], c.lr, c.beta1, c.beta2,
                  c.eps, p->step, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VM3DGS_OK : fail(VM3DGS_E_CUDA, cudaGetErrorString(e));
}

extern "C" int vm3dgs_prefetcher_params(vm3dgs_prefetcher *p, int32_t what, float *host, int64_t n, void *stream) {
  if (!p || !host) return fail(VM3DGS_E_INVAL, "null argument");
  const PfLayout &L = p->lay;
  if (n != L.n_params) return fail(VM3DGS_E_INVAL, "parameter count is " + std::to_string(L.n_params));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = 0;
  if (what == VM3DGS_PARAMS_SET) {
    if (!ok(cudaMemcpyAsync(p->at<void>(L.w), host, 4 * n, cudaMemcpyHostToDevice, st), "copy", &rc)) return rc;
    float *wd = p->at<float>(L.w);
    launch_to_bf16(wd, p->at<__nv_bfloat16>(L.w1b), L.n_w1, st);
    launch_to_bf16(wd + L.n_w1 + L.n_b1, p->at<__nv_bfloat16>(L.w2b), L.n_w2, st);
    launch_to_bf16(wd + L.n_w1 + L.n_b1 + L.n_w2 + L.n_b2, p->at<__nv_bfloat16>(L.w3b), L.n_w3, st);
    cudaMemsetAsync(p->at<void>(L.m), 0, 4 * n, st);
    cudaMemsetAsync(p->at<void>(L.v), 0, 4 * n, st);
    p->step = 0;
  } else if (what == VM3DGS_PARAMS_GET || what == VM3DGS_PARAMS_GRAD) {
    const int64_t off = what == VM3DGS_PARAMS_GET ? L.w : L.g;
    if (!ok(cudaMemcpyAsync(host, p->at<void>(off), 4 * n, cudaMemcpyDeviceToHost, st), "copy", &rc)) return rc;
  } else {
    return fail(VM3DGS_E_INVAL, "unknown parameter request");
  }
  if (!ok(cudaStreamSynchronize(st), "sync", &rc)) return rc;
  return VM3DGS_OK;
}
