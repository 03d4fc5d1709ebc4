// Learned page prefetcher: a 3-layer MLP (inputs -> ReLU hidden -> ReLU hidden
// -> one logit per page of a page window) trained and evaluated on the GPU.
// The paper has no learned part; its limitations (Sec. 4.3) ask for earlier,
// prioritised and asynchronous copies, which the prefetcher provides.
//
// GEMM: C[M,N] = op(A)[M,K] * op(B)[K,N], A and B bf16 in row-major memory
// (op = optional transpose), FP32 accumulation on the tensor cores
// (tcgen05.mma, accumulator in tensor memory; batch-1 inference instead
// takes a GEMV on the CUDA cores).  Epilogue: + bias[n], optional ReLU,
// optional multiply by (mask_z[m,n] > 0) (the ReLU derivative), stores fp32
// and/or bf16.
#include <cuda_bf16.h>

#include "mlp.cuh"

namespace vm {
namespace {

// GEMM on the 5th-generation tensor cores: a CTA of 4 warps computes a
// 128 x 64 tile of C with tcgen05.mma (kind::f16, bf16 x bf16 -> f32, M = 128,
// N = 64, K = 16 per instruction) into a 64-column accumulator in tensor
// memory.  Per K-step of 64 the threads stage op(A) and op(B) tiles (zero
// padded) in shared memory in the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, adjacent along K 128 B apart (leading byte
// offset), adjacent 8-row groups 1024 B apart (stride byte offset).  One
// thread issues the four MMAs and commits them to an mbarrier the CTA waits
// on (bounded); the epilogue reads the accumulator rows of each warp's lane
// quarter with tcgen05.ld.
constexpr int TM = 128, TN = 64, TK = 64;
constexpr uint32_t kLbo = 128, kSbo = (TK / 8) * 128;

__device__ __forceinline__ uint32_t core_off(int r, int k) {  // byte offset of (r, k) in a staged tile
  return (uint32_t)((r >> 3) * kSbo + (k >> 3) * kLbo + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kSbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // no swizzle, base offset 0
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__global__ void __launch_bounds__(128) gemm_tc_kernel(GemmArgs g) {
  __shared__ __align__(1024) uint8_t As[TM * TK * 2];
  __shared__ __align__(1024) uint8_t Bs[TN * TK * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"((uint32_t)TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar)), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < g.K; k0 += TK) {
    for (int e = tid; e < TM * TK; e += 128) {
      const int r = e / TK, c = e % TK, m = m0 + r, k = k0 + c;
      __nv_bfloat16 v = zero;
      if (m < g.M && k < g.K) v = g.transA ? g.A[(int64_t)k * g.lda + m] : g.A[(int64_t)m * g.lda + k];
      *reinterpret_cast<__nv_bfloat16 *>(As + core_off(r, c)) = v;
    }
    for (int e = tid; e < TN * TK; e += 128) {
      const int r = e / TK, c = e % TK, n = n0 + r, k = k0 + c;
      __nv_bfloat16 v = zero;
      if (n < g.N && k < g.K) v = g.transB ? g.B[(int64_t)n * g.ldb + k] : g.B[(int64_t)k * g.ldb + n];
      *reinterpret_cast<__nv_bfloat16 *>(Bs + core_off(r, c)) = v;
    }
    // the staged tiles become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int s = 0; s < TK / 16; ++s) {
        const uint64_t ad = smem_desc(smem_addr(As) + s * 2 * kLbo), bd = smem_desc(smem_addr(Bs) + s * 2 * kLbo);
        const uint32_t acc = (k0 > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(&bar))
                   : "memory");
    }
    // wait (bounded) for the MMAs: they read the staged tiles
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it)
      asm volatile(
          "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
          : "=r"(done)
          : "r"(smem_addr(&bar)), "r"(phase)
          : "memory");
    ok = ok && done;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok && tid == 0 && g.err) atomicExch(g.err, 1);
  // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile in its lane quarter
  const int m = m0 + 32 * warp + lane;
#pragma unroll
  for (int c = 0; c < TN / 16; ++c) {
    uint32_t v[16];
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * c);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (m < g.M && g.K > 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + 16 * c + j;
        if (n >= g.N) continue;
        float x = __uint_as_float(v[j]);
        if (g.bias) x += g.bias[n];
        if (g.relu) x = x > 0.0f ? x : 0.0f;
        const int64_t o = (int64_t)m * g.ldc + n;
        if (g.mask_z && !(g.mask_z[o] > 0.0f)) x = 0.0f;
        if (g.C) g.C[o] = x;
        if (g.Cb) g.Cb[o] = __float2bfloat16(x);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TN) : "memory");
  }
}

// Batch-1 inference: y[n] = x . B[:, n] (+ bias, ReLU).  A CTA takes 32
// output columns (a warp reads 32 consecutive weights of a row) and splits
// the K rows over its 8 warps (warp w: rows w, w + 8, ...); the 8 partial
// sums are added in warp order from shared memory.  The input row is staged
// in shared memory.
constexpr int kGemvThreads = 256, kGemvMaxK = 1024, kGemvCols = 32, kGemvSplit = kGemvThreads / kGemvCols;
__global__ void __launch_bounds__(kGemvThreads) gemv_kernel(GemmArgs g) {
  __shared__ float xs[kGemvMaxK];
  __shared__ float part[kGemvSplit][kGemvCols];
  for (int k = threadIdx.x; k < g.K; k += kGemvThreads) xs[k] = __bfloat162float(g.A[k]);
  __syncthreads();
  const int c = threadIdx.x % kGemvCols, w = threadIdx.x / kGemvCols;
  const int n = blockIdx.x * kGemvCols + c;
  float acc = 0.0f;
  if (n < g.N) {
    const __nv_bfloat16 *b = g.B + n;
#pragma unroll 8
    for (int k = w; k < g.K; k += kGemvSplit) acc += xs[k] * __bfloat162float(b[(int64_t)k * g.ldb]);
  }
  part[w][c] = acc;
  __syncthreads();
  if (w != 0 || n >= g.N) return;
  float v = 0.0f;
#pragma unroll
  for (int j = 0; j < kGemvSplit; ++j) v += part[j][c];
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
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM);
  gemm_tc_kernel<<<grid, 128, 0, st>>>(g);
}

void launch_gemv(const GemmArgs &g, cudaStream_t st) {
  if (g.M != 1 || g.transA || g.transB || g.mask_z || g.K > kGemvMaxK) {
    launch_gemm(g, st);
    return;
  }
  gemv_kernel<<<(g.N + kGemvCols - 1) / kGemvCols, kGemvThreads, 0, st>>>(g);
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
