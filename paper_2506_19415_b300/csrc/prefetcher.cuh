// Internal state of the learned prefetcher.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/vm3dgs.h"

namespace vm {

struct PfLayout {
  int64_t n_w1, n_b1, n_w2, n_b2, n_w3, n_b3, n_params;
  int64_t w, g, m, v, w1b, w2b, w3b, xb, h1f, h1b, h2f, h2b, logits, dy, dyb, dz2, dz2b, dz1, dz1b, loss, feat, total;
};

PfLayout pf_layout(const vm3dgs_mlp_config &c);

}  // namespace vm

struct vm3dgs_prefetcher {
  vm3dgs_mlp_config cfg{};
  vm::PfLayout lay{};
  uint8_t *mem = nullptr;
  int step = 0;
  template <class T>
  T *at(int64_t off) const { return reinterpret_cast<T *>(mem + off); }
};

namespace vm {
void pf_forward(vm3dgs_prefetcher *p, const float *x, int Bn, float *logits, cudaStream_t st);
}
