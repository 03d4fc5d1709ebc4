// Internal interface of the prefetcher network kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace vm {

struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16 *A;  // op(A) is M x K
  int lda, transA;
  const __nv_bfloat16 *B;  // op(B) is K x N
  int ldb, transB;
  const float *bias;       // [N] or null
  int relu;
  const float *mask_z;     // [M, ldc]: zero the output where mask_z <= 0 (ReLU derivative), or null
  float *C;                // fp32 out [M, ldc] or null
  __nv_bfloat16 *Cb;       // bf16 out [M, ldc] or null
  int ldc;
  int *err;                // set to 1 if a bounded wait for the tensor cores gave up (or null)
};

void launch_gemm(const GemmArgs &g, cudaStream_t st);
// the same product for M = 1, op(A) = A, op(B) = B (a row vector times a
// K x N matrix): a thread per output, FP32 accumulation in k order
void launch_gemv(const GemmArgs &g, cudaStream_t st);
void launch_bce_grad(const float *logit, const float *target, const float *mask, int64_t n, float inv_n, float *dy,
                     __nv_bfloat16 *dyb, float *loss, cudaStream_t st);
void launch_colsum(const float *x, int rows, int cols, float *out, cudaStream_t st);
void launch_adam(float *w, const float *grad, float *m, float *v, __nv_bfloat16 *wb, int64_t n, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t st);
void launch_to_bf16(const float *x, __nv_bfloat16 *y, int64_t n, cudaStream_t st);

}  // namespace vm
