// Learned page prefetcher: a 3-layer MLP (inputs -> ReLU hidden -> ReLU hidden
// -> one logit per page of a page window) trained and evaluated on the GPU.
// The paper has no learned part; its limitations (Sec. 4.3) ask for earlier,
// prioritised and asynchronous copies, which the prefetcher provides.
//
// GEMM: C[M,N] = op(A)[M,K] * op(B)[K,N], A and B bf16 in row-major memory
// (op = optional transpose), FP32 accumulation on the tensor cores with
// mma.sync m16n8k16 (bf16 x bf16 -> f32).  Block tile 64 x 64 x 32, 4 warps
// of 32 x 32.  Epilogue: + bias[n], optional ReLU, optional multiply by
// (mask_z[m,n] > 0) (the ReLU derivative), stores fp32 and/or bf16.
#include <cuda_bf16.h>

#include "mlp.cuh"

namespace vm {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_kernel(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];   // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];   // [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    // A tile: element (m, k) of op(A)
    for (int e = tid; e < BM * BK; e += 128) {
      const int r = e / BK, c = e % BK;
      const int m = m0 + r, k = k0 + c;
      __nv_bfloat16 v = zero;
      if (m < g.M && k < g.K) v = g.transA ? g.A[(int64_t)k * g.lda + m] : g.A[(int64_t)m * g.lda + k];
      As[r][c] = v;
    }
    // B tile: element (k, n) of op(B), stored [n][k]
    for (int e = tid; e < BN * BK; e += 128) {
      const int r = e / BK, c = e % BK;   // r = n offset, c = k offset
      const int n = n0 + r, k = k0 + c;
      __nv_bfloat16 v = zero;
      if (n < g.N && k < g.K) v = g.transB ? g.B[(int64_t)n * g.ldb + k] : g.B[(int64_t)k * g.ldb + n];
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gq;
        af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * tq]);
        af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * tq]);
        af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * tq + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * tq + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + gq;
        bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * tq]);
        bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * tq + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
  // epilogue: accumulator element (row gq or gq+8, col 2tq or 2tq+1) of each 16x8 tile
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int m = m0 + wm + i * 16 + gq + (h >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tq + (h & 1);
        if (m >= g.M || n >= g.N) continue;
        float v = acc[i][j][h];
        if (g.bias) v += g.bias[n];
        if (g.relu) v = v > 0.0f ? v : 0.0f;
        const int64_t o = (int64_t)m * g.ldc + n;
        if (g.mask_z && !(g.mask_z[o] > 0.0f)) v = 0.0f;
        if (g.C) g.C[o] = v;
        if (g.Cb) g.Cb[o] = __float2bfloat16(v);
      }
}

// Batch-1 inference: y[n] = x . B[:, n] (+ bias, ReLU), a thread per output
// column n (coalesced rows of B), the input row staged in shared memory.
constexpr int kGemvThreads = 256, kGemvMaxK = 1024;
__global__ void __launch_bounds__(kGemvThreads) gemv_kernel(GemmArgs g) {
  __shared__ float xs[kGemvMaxK];
  for (int k = threadIdx.x; k < g.K; k += kGemvThreads) xs[k] = __bfloat162float(g.A[k]);
  __syncthreads();
  const int n = blockIdx.x * kGemvThreads + threadIdx.x;
  if (n >= g.N) return;
  const __nv_bfloat16 *b = g.B + n;
  float acc = 0.0f;
#pragma unroll 8
  for (int k = 0; k < g.K; ++k) acc += xs[k] * __bfloat162float(b[(int64_t)k * g.ldb]);
  float v = acc;
  if (g.bias) v += g.bias[n];
  if (g.relu) v = v > 0.0f ? v : 0.0f;
  if (g.C) g.C[n] = v;
  if (g.Cb) g.Cb[n] = __float2bfloat16(v);
}

// dY = (sigmoid(logit) - target) * mask / max(sum(mask), 1); loss (mean BCE) into *loss
__global__ void bce_grad_kernel(const float *logit, const float *target, const float *mask, int64_t n, float inv_n,
                                float *dy, __nv_bfloat16 *dyb, float *loss) {
  __shared__ float red[256];
  float acc = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float x = logit[i], t = target[i], m = mask[i];
    const float s = 1.0f / (1.0f + __expf(-x));
    const float d = (s - t) * m * inv_n;
    dy[i] = d;
    dyb[i] = __float2bfloat16(d);
    acc += m * (fmaxf(x, 0.0f) - x * t + log1pf(__expf(-fabsf(x))));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0] * inv_n);
}

// column sums of a [rows, cols] fp32 matrix (bias gradients)
__global__ void colsum_kernel(const float *x, int rows, int cols, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += x[(int64_t)r * cols + c];
  out[c] = s;
}

// one Adam step on fp32 master weights, bf16 copy refreshed
__global__ void adam_kernel(float *w, const float *grad, float *m, float *v, __nv_bfloat16 *wb, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
  }
}

__global__ void to_bf16_kernel(const float *x, __nv_bfloat16 *y, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = __float2bfloat16(x[i]);
}

unsigned blocks_for(int64_t n, int per = 256) {
  int64_t b = (n + per - 1) / per;
  if (b > 148 * 8) b = 148 * 8;
  return (unsigned)(b > 0 ? b : 1);
}

}  // namespace

void launch_gemm(const GemmArgs &g, cudaStream_t st) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  gemm_kernel<<<grid, 128, 0, st>>>(g);
}

void launch_gemv(const GemmArgs &g, cudaStream_t st) {
  if (g.M != 1 || g.transA || g.transB || g.mask_z || g.K > kGemvMaxK) {
    launch_gemm(g, st);
    return;
  }
  gemv_kernel<<<(g.N + kGemvThreads - 1) / kGemvThreads, kGemvThreads, 0, st>>>(g);
}

void launch_bce_grad(const float *logit, const float *target, const float *mask, int64_t n, float inv_n, float *dy,
                     __nv_bfloat16 *dyb, float *loss, cudaStream_t st) {
  bce_grad_kernel<<<blocks_for(n), 256, 0, st>>>(logit, target, mask, n, inv_n, dy, dyb, loss);
}

void launch_colsum(const float *x, int rows, int cols, float *out, cudaStream_t st) {
  colsum_kernel<<<(cols + 255) / 256, 256, 0, st>>>(x, rows, cols, out);
}

void launch_adam(float *w, const float *grad, float *m, float *v, __nv_bfloat16 *wb, int64_t n, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t st) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  adam_kernel<<<blocks_for(n), 256, 0, st>>>(w, grad, m, v, wb, n, lr, b1, b2, eps, c1, c2);
}

void launch_to_bf16(const float *x, __nv_bfloat16 *y, int64_t n, cudaStream_t st) {
  to_bf16_kernel<<<blocks_for(n), 256, 0, st>>>(x, y, n);
}

}  // namespace vm
