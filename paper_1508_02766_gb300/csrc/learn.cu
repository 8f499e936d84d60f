// Learned bandwidth proposal.  The paper points to fast bandwidth selection
// with the same FFT machinery (Sec. 1, Sec. 5); the network is not from the
// paper.  This file holds its GPU side:
//   - sample standardisation and features (moments, and a 32 x 32 block
//     downsampling of the binned grid of the standardised samples);
//   - a three-layer MLP (ReLU) with BF16 operands and FP32 accumulation,
//     trained with Adam on FP32 master weights.  Every matrix product runs on
//     the 5th-generation tensor cores: tcgen05.mma issued by one thread per
//     CTA, operands staged in shared memory by cp.async, accumulators in
//     tensor memory read back with tcgen05.ld for fused epilogues (bias,
//     ReLU, ReLU gradient, BF16 and transposed BF16 copies).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>

#include "kde_internal.h"
#include "tc_wait.cuh"

namespace kde {
namespace {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// Tensor-core GEMM: D[M x N] = A[M x K] B[N x K]^T, A and B K-major BF16,
// FP32 accumulation.  CTA tile 128 x BN, K in steps of 64 (four MMAs of
// K = 16).  Tiles sit in shared memory in the no-swizzle canonical layout:
// core matrices of 8 rows x 16 bytes, element (r, k) at byte
// (r/8) 1024 + (k/8) 128 + (r%8) 16 + (k%8) 2, i.e. 128 bytes between
// K-adjacent core matrices (leading byte offset) and 1024 bytes between
// 8-row groups (stride byte offset).  Sizes: M % 128 == 0, N % BN == 0,
// K % 64 == 0, row strides multiples of 8 elements, 16-byte aligned bases.
// ---------------------------------------------------------------------------
enum Epi { EPI_STORE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_RELU_GRAD = 3 };

struct GemmArgs {
  const bf16* A;
  int lda;
  const bf16* B;
  int ldb;
  int M, N, K;
  float* C;            // FP32 result after the epilogue (pre-activation for BIAS_RELU)
  int ldc;
  const float* bias;   // BIAS_RELU, BIAS: per column
  const float* Z;      // RELU_GRAD: D is multiplied by (Z > 0)
  int ldz;
  bf16* Cb;            // optional BF16 copy of the activation / gradient, row-major
  int ldcb;
  bf16* Ct;            // optional BF16 transposed copy: Ct[n ldct + m]
  int ldct;
  int* status;         // set to 1 if a wait for the tensor cores gave up
};


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor version
// 1 (bit 46), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(1024u >> 4) << 32) | (1ull << 46);
}

// Stage the 64-wide K slice k0 of A's rows m0.. and B's rows n0.. into one
// shared-memory stage with 16-byte cp.async copies (one commit group).
template <int BN>
__device__ __forceinline__ void stage_tiles(const GemmArgs& g, uint8_t* sA, uint8_t* sB, int m0,
                                            int n0, int k0) {
  const int tid = threadIdx.x;
  for (int i = tid; i < 128 * 8; i += 128) {
    const int r = i >> 3, c = i & 7;
    const size_t src = __cvta_generic_to_global(g.A + (size_t)(m0 + r) * g.lda + k0 + 8 * c);
    const uint32_t dst = smem_u32(sA + (r >> 3) * 1024 + c * 128 + (r & 7) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  }
  for (int i = tid; i < BN * 8; i += 128) {
    const int r = i >> 3, c = i & 7;
    const size_t src = __cvta_generic_to_global(g.B + (size_t)(n0 + r) * g.ldb + k0 + 8 * c);
    const uint32_t dst = smem_u32(sB + (r >> 3) * 1024 + c * 128 + (r & 7) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Two shared-memory stages: the copies of K slice k+1 are in flight while
// the tensor cores work on slice k; a stage is refilled only after the MMAs
// that read it have completed (its mbarrier).
template <int BN, int EPI>
__global__ void __launch_bounds__(128) kde_gemm_tc_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int kStageBytes = 16384 + BN * 128;  // A 128 x 64 + B BN x 64, BF16
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  constexpr uint32_t kCols = BN < 32 ? 32 : BN;  // TMEM columns: a power of two >= 32
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16
  // (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  uint32_t phase = 0u, used = 0u;  // bit b: stage b's barrier phase / MMAs pending
  bool ok = true;
  const int nk = g.K / 64;
  stage_tiles<BN>(g, smem, smem + 16384, m0, n0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1, nx = st ^ 1;
    if (kt + 1 < nk) {
      // the other stage was read by the MMAs of slice kt - 1: wait for them
      if ((used >> nx) & 1u) {
        const bool done = mbar_wait(smem_u32(&mbar[nx]), (phase >> nx) & 1u);
        if (!__syncthreads_and(done)) {
          ok = false;
          break;
        }
        phase ^= 1u << nx;
        used &= ~(1u << nx);
      }
      stage_tiles<BN>(g, smem + nx * kStageBytes, smem + nx * kStageBytes + 16384, m0, n0,
                      (kt + 1) * 64);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    // the tensor cores read shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + st * kStageBytes), b0 = a0 + 16384u;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint64_t da = umma_desc(a0 + 256u * s);
        const uint64_t db = umma_desc(b0 + 256u * s);
        const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[st]))
          : "memory");
    }
    used |= 1u << st;
  }
  // every MMA has been committed; the last commit tracks them all
  if (ok) {
    const int last = (nk - 1) & 1;
    const bool done = mbar_wait(smem_u32(&mbar[last]), (phase >> last) & 1u);
    ok = __syncthreads_and(done);
  }
  if (!ok) {
    if (tid == 0) atomicExch(g.status, 1);
    // one more bounded chance for the MMAs in flight before TMEM is freed
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    for (int b = 0; b < 2; ++b)
      if ((used >> b) & 1u) mbar_wait(smem_u32(&mbar[b]), (phase >> b) & 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
          "[%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + c0 + j;
        float x = __uint_as_float(v[j]);
        float a = x;
        if (EPI == EPI_BIAS_RELU || EPI == EPI_BIAS) x += g.bias[n];
        if (EPI == EPI_BIAS_RELU) a = fmaxf(x, 0.f);
        if (EPI == EPI_RELU_GRAD) {
          x = g.Z[(size_t)row * g.ldz + n] > 0.f ? x : 0.f;
          a = x;
        }
        g.C[(size_t)row * g.ldc + n] = x;
        if (EPI == EPI_BIAS_RELU || EPI == EPI_RELU_GRAD) {
          const bf16 b = __float2bfloat16_rn(a);
          if (g.Cb) g.Cb[(size_t)row * g.ldcb + n] = b;
          if (g.Ct) g.Ct[(size_t)n * g.ldct + row] = b;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
}

template <int BN, int EPI>
cudaError_t launch_gemm_bn(const GemmArgs& g, cudaStream_t st) {
  // Two stages of A (16 KB) and B (BN x 128 bytes); 56 KB of dynamic shared
  // memory caps the CTAs per SM at 4, so the tensor memory they hold
  // (4 x 64 columns) stays within the SM's 512 columns.
  const int smem = 56 * 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kde_gemm_tc_kernel<BN, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  LaunchScope ls("kde_gemm_tc_kernel", st);
  kde_gemm_tc_kernel<BN, EPI><<<dim3(g.M / 128, g.N / BN), 128, smem, st>>>(g);
  return cudaGetLastError();
}

kde_status launch_gemm(const GemmArgs& g, int epi, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.M % 128 || g.N % 16 || g.K % 64 || g.lda % 8 ||
      g.ldb % 8 || ((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15) || !g.C || !g.status)
    return fail(KDE_ERR_INVALID_ARG,
                "tensor-core GEMM: need M % 128 == 0, N % 16 == 0, K % 64 == 0, row strides "
                "multiples of 8 elements and 16-byte aligned operands");
  cudaError_t e;
  const bool wide = g.N % 64 == 0;
  switch (epi) {
    case EPI_STORE: e = wide ? launch_gemm_bn<64, EPI_STORE>(g, st) : launch_gemm_bn<16, EPI_STORE>(g, st); break;
    case EPI_BIAS_RELU: e = wide ? launch_gemm_bn<64, EPI_BIAS_RELU>(g, st) : launch_gemm_bn<16, EPI_BIAS_RELU>(g, st); break;
    case EPI_BIAS: e = wide ? launch_gemm_bn<64, EPI_BIAS>(g, st) : launch_gemm_bn<16, EPI_BIAS>(g, st); break;
    default: e = wide ? launch_gemm_bn<64, EPI_RELU_GRAD>(g, st) : launch_gemm_bn<16, EPI_RELU_GRAD>(g, st); break;
  }
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_gemm_tc_kernel");
}

// ---------------------------------------------------------------------------
// Element-wise and reduction kernels of the MLP.
// ---------------------------------------------------------------------------
// X (B x in, FP32) -> Xb (Bp x in, BF16) and its transpose Xt (in x Bp);
// rows B .. Bp-1 are zero.
__global__ void __launch_bounds__(256) kde_mlp_cast_kernel(const float* __restrict__ X, int B,
                                                           int Bp, int in, bf16* __restrict__ Xb,
                                                           bf16* __restrict__ Xt) {
  const int64_t total = (int64_t)Bp * in;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / in), k = (int)(i - (int64_t)b * in);
    const bf16 v = __float2bfloat16_rn(b < B ? X[i] : 0.f);
    Xb[i] = v;
    if (Xt) Xt[(int64_t)k * Bp + b] = v;
  }
}

// Loss = (1/B) sum_{b < B, j < out} (Y - T)^2 and its gradient
// dY = (2/B)(Y - T): BF16 copies dYb (Bp x 64, zero beyond out) and
// dYt (outp x Bp), and db3 = sum_b dY (FP32, fixed order).  One block.
__global__ void __launch_bounds__(256) kde_mlp_loss_kernel(const float* __restrict__ Y, int ldy,
                                                           const float* __restrict__ T, int B,
                                                           int Bp, int out, int outp,
                                                           bf16* __restrict__ dYb,
                                                           bf16* __restrict__ dYt,
                                                           float* __restrict__ db3,
                                                           float* __restrict__ loss) {
  __shared__ double part[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < Bp * 64; i += blockDim.x) {
    const int b = i / 64, j = i % 64;
    float g = 0.f;
    if (b < B && j < out) {
      const float r = Y[(size_t)b * ldy + j] - T[(size_t)b * out + j];
      acc += (double)r * r;
      g = 2.f * r / (float)B;
    }
    const bf16 gb = __float2bfloat16_rn(g);
    dYb[i] = gb;
    if (j < outp) dYt[(size_t)j * Bp + b] = gb;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = (float)(part[0] / B);
  for (int j = threadIdx.x; j < out; j += blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += 2.f * (Y[(size_t)b * ldy + j] - T[(size_t)b * out + j]) / (float)B;
    db3[j] = s;
  }
}

// db[n] = sum_{b < B} dZ[b n] (one thread per column, fixed order).
__global__ void __launch_bounds__(256) kde_mlp_colsum_kernel(const float* __restrict__ dZ, int ld,
                                                             int B, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(size_t)b * ld + n];
  db[n] = s;
}

// G_W3[j h] = dW3t[h j] for j < out.
__global__ void __launch_bounds__(256) kde_mlp_w3grad_kernel(const float* __restrict__ dW3t, int hid,
                                                             int outp, int out,
                                                             float* __restrict__ gW3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= out * hid) return;
  const int j = i / hid, h = i % hid;
  gW3[i] = dW3t[(size_t)h * outp + j];
}

// Adam on the flat FP32 parameters.
__global__ void __launch_bounds__(256) kde_mlp_adam_kernel(float* __restrict__ P,
                                                           const float* __restrict__ G,
                                                           float* __restrict__ Mo,
                                                           float* __restrict__ Vo, int64_t n,
                                                           float lr, float b1, float b2, float eps,
                                                           float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * Mo[i] + (1.f - b1) * g;
    const float v = b2 * Vo[i] + (1.f - b2) * g * g;
    Mo[i] = m;
    Vo[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// BF16 working copies of the weights: W1b (hid x in), W2b (hid x hid),
// W2t (hid x hid, transposed), W3b (outp x hid, zero rows beyond out),
// W3t (hid x 64: W3t[h j] = W3[j h] for j < out, else 0), b3p (outp).
__global__ void __launch_bounds__(256) kde_mlp_refresh_kernel(
    const float* __restrict__ W1, const float* __restrict__ W2, const float* __restrict__ W3,
    const float* __restrict__ b3, int in, int hid, int out, int outp, bf16* __restrict__ W1b,
    bf16* __restrict__ W2b, bf16* __restrict__ W2t, bf16* __restrict__ W3b,
    bf16* __restrict__ W3t, float* __restrict__ b3p) {
  const int64_t n1 = (int64_t)hid * in, n2 = (int64_t)hid * hid, n3 = (int64_t)outp * hid,
                n4 = (int64_t)hid * 64;
  const int64_t total = n1 + n2 + n3 + n4 + outp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n1) {
      W1b[i] = __float2bfloat16_rn(W1[i]);
    } else if (i < n1 + n2) {
      const int64_t t = i - n1;
      const int r = (int)(t / hid), c = (int)(t % hid);
      const bf16 v = __float2bfloat16_rn(W2[t]);
      W2b[t] = v;
      W2t[(int64_t)c * hid + r] = v;
    } else if (i < n1 + n2 + n3) {
      const int64_t t = i - n1 - n2;
      const int j = (int)(t / hid);
      W3b[t] = __float2bfloat16_rn(j < out ? W3[t] : 0.f);
    } else if (i < n1 + n2 + n3 + n4) {
      const int64_t t = i - n1 - n2 - n3;
      const int h = (int)(t / 64), j = (int)(t % 64);
      W3t[t] = __float2bfloat16_rn(j < out ? W3[(int64_t)j * hid + h] : 0.f);
    } else {
      const int j = (int)(i - n1 - n2 - n3 - n4);
      b3p[j] = j < out ? b3[j] : 0.f;
    }
  }
}

// Y[b j] (b < B, j < out) from the padded output.
__global__ void __launch_bounds__(256) kde_mlp_take_kernel(const float* __restrict__ Yp, int ldy,
                                                           int B, int out, float* __restrict__ Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * out) return;
  Y[i] = Yp[(size_t)(i / out) * ldy + (i % out)];
}

// ---------------------------------------------------------------------------
// Standardisation and features (d = 2).  FP64 arithmetic runs at a small
// fraction of FP32's rate on this GPU, so the sums are FP32 trees (each
// thread about ten samples, then warp shuffles and one warp over the warp
// partials); only thread 0 forms the FP64 outputs.
// ---------------------------------------------------------------------------
__device__ float block_sum_f(float v, float* wbuf) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) wbuf[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float w = threadIdx.x < (blockDim.x >> 5) ? wbuf[threadIdx.x] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w += __shfl_down_sync(0xffffffffu, w, off);
    if (threadIdx.x == 0) wbuf[32] = w;
  }
  __syncthreads();
  const float r = wbuf[32];
  __syncthreads();
  return r;
}

// One block of 1024 threads.  moments = {mean0, mean1, sd0, sd1, corr,
// skew0, skew1, (kurt0 + kurt1)/2 - 3} (population moments); Z = (X - mean)
// / sd in FP32.
__device__ __forceinline__ void standardize2_body(const float* __restrict__ X, int64_t n,
                                                  float* __restrict__ Z, double* __restrict__ mom) {
  __shared__ float wbuf[33];
  const float inv_n = 1.0f / (float)n;
  float s0 = 0.f, s1 = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    s0 += X[2 * i];
    s1 += X[2 * i + 1];
  }
  const float m0 = block_sum_f(s0, wbuf) * inv_n, m1 = block_sum_f(s1, wbuf) * inv_n;
  float q00 = 0.f, q11 = 0.f, q01 = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float a = X[2 * i] - m0, b = X[2 * i + 1] - m1;
    q00 = fmaf(a, a, q00);
    q11 = fmaf(b, b, q11);
    q01 = fmaf(a, b, q01);
  }
  const float v0 = block_sum_f(q00, wbuf) * inv_n, v1 = block_sum_f(q11, wbuf) * inv_n;
  const float c01 = block_sum_f(q01, wbuf) * inv_n;
  const float sd0 = sqrtf(v0), sd1 = sqrtf(v1);
  const float r0 = 1.0f / sd0, r1 = 1.0f / sd1;
  float t3a = 0.f, t3b = 0.f, t4a = 0.f, t4b = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float a = (X[2 * i] - m0) * r0, b = (X[2 * i + 1] - m1) * r1;
    Z[2 * i] = a;
    Z[2 * i + 1] = b;
    const float a2 = a * a, b2 = b * b;
    t3a = fmaf(a2, a, t3a);
    t3b = fmaf(b2, b, t3b);
    t4a = fmaf(a2, a2, t4a);
    t4b = fmaf(b2, b2, t4b);
  }
  const float sk0 = block_sum_f(t3a, wbuf) * inv_n, sk1 = block_sum_f(t3b, wbuf) * inv_n;
  const float k0 = block_sum_f(t4a, wbuf), k1 = block_sum_f(t4b, wbuf);
  if (threadIdx.x == 0) {
    mom[0] = m0;
    mom[1] = m1;
    mom[2] = sd0;
    mom[3] = sd1;
    mom[4] = (double)c01 / ((double)sd0 * sd1);
    mom[5] = sk0;
    mom[6] = sk1;
    mom[7] = 0.5 * ((double)k0 + k1) / (double)n - 3.0;
  }
}

__global__ void __launch_bounds__(1024) kde_standardize2_kernel(const float* __restrict__ X,
                                                                int64_t n, float* __restrict__ Z,
                                                                double* __restrict__ mom) {
  standardize2_body(X, n, Z, mom);
}

// One block per dataset of a batch: rows [off[b], off[b + 1]) of X and Z,
// moments at 8 b.
__global__ void __launch_bounds__(1024) kde_standardize2_sets_kernel(
    const float* __restrict__ X, const int64_t* __restrict__ off, float* __restrict__ Z,
    double* __restrict__ mom) {
  const int64_t a = off[blockIdx.x], b = off[blockIdx.x + 1];
  standardize2_body(X + 2 * a, b - a, Z + 2 * a, mom + 8 * (int64_t)blockIdx.x);
}

// 32 blocks of 256 threads, block `by` for the 32 block-features of one
// block row of the M x M grid (w = M/32 cells a side): thread (y0, bx) sums
// rows y0, y0 + 8, ... of block (by, bx); the rows are then added in shared
// memory.  feat[32 by + bx] = 8 sqrt(mass / n) with mass the block's counts
// times 2^-32; block 0 also writes feat[1024..] = corr, skew0, skew1, excess
// kurtosis, log10(n)/4, 1, then zeros.
__device__ __forceinline__ void features2_body(int by, const long long* __restrict__ counts,
                                               int M, int64_t n, const double* __restrict__ mom,
                                               float* __restrict__ feat) {
  __shared__ unsigned long long part[8][32];
  const int t = threadIdx.x, bx = t & 31, y0 = t >> 5, w = M / 32;
  unsigned long long s = 0;
  for (int y = y0; y < w; y += 8) {
    const long long* row = counts + (size_t)(by * w + y) * M + bx * w;
    for (int x = 0; x < w; ++x) s += (unsigned long long)row[x];
  }
  part[y0][bx] = s;
  __syncthreads();
  if (t < 32) {
    unsigned long long tot = 0;
    for (int k = 0; k < 8; ++k) tot += part[k][t];
    // tot 2^-32 from its two 32-bit halves (no 64-bit integer conversion)
    const float mass =
        fmaf((float)(unsigned)(tot >> 32), 1.0f, (float)(unsigned)tot * 2.3283064365386963e-10f) /
        (float)n;
    feat[by * 32 + t] = 8.0f * sqrtf(mass);
  }
  if (by == 0 && t < 64) {
    float v = 0.f;
    if (t == 0) v = (float)mom[4];
    if (t == 1) v = (float)mom[5];
    if (t == 2) v = (float)mom[6];
    if (t == 3) v = (float)mom[7];
    if (t == 4) v = (float)(log10((double)n) / 4.0);
    if (t == 5) v = 1.f;
    feat[1024 + t] = v;
  }
}

__global__ void __launch_bounds__(256) kde_features2_kernel(const long long* __restrict__ counts,
                                                            int M, int64_t n,
                                                            const double* __restrict__ mom,
                                                            float* __restrict__ feat) {
  features2_body(blockIdx.x, counts, M, n, mom, feat);
}

// Grid (32, nsets): block row blockIdx.x of dataset blockIdx.y, whose
// counts start at y M^2, moments at 8 y and features at y KDE_FEAT_DIM.
__global__ void __launch_bounds__(256) kde_features2_sets_kernel(
    const long long* __restrict__ counts, int M, const int64_t* __restrict__ off,
    const double* __restrict__ mom, float* __restrict__ feat) {
  const int64_t y = blockIdx.y;
  features2_body(blockIdx.x, counts + y * M * M, M, off[y + 1] - off[y], mom + 8 * y,
                 feat + y * KDE_FEAT_DIM);
}

}  // namespace
}  // namespace kde

namespace kde {

kde_status standardize2_sets(const float* X, const int64_t* off_dev, int nsets, float* Z,
                             double* moments, cudaStream_t st) {
  LaunchScope ls("kde_standardize2_sets_kernel", st);
  kde_standardize2_sets_kernel<<<nsets, 1024, 0, st>>>(X, off_dev, Z, moments);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_standardize2_sets_kernel");
}

kde_status features2_sets(const int64_t* counts, int M, int nsets, const int64_t* off_dev,
                          const double* moments, float* feat, cudaStream_t st) {
  LaunchScope ls("kde_features2_sets_kernel", st);
  kde_features2_sets_kernel<<<dim3(32, (unsigned)nsets), 256, 0, st>>>(
      (const long long*)counts, M, off_dev, moments, feat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_features2_sets_kernel");
}

}  // namespace kde

using namespace kde;

struct kde_mlp_s {
  int in, hid, out, outp, maxB;
  int64_t nparam, oW1, ob1, oW2, ob2, oW3, ob3;
  float *P, *G, *Mo, *Vo;
  bf16 *W1b, *W2b, *W2t, *W3b, *W3t;
  bf16 *Xb, *Xt, *A1b, *A1t, *A2b, *A2t, *dYb, *dYt, *dZ2b, *dZ2t, *dZ1t;
  float *Z1, *Z2, *Y, *dZ1, *dZ2, *dW3t, *b3p, *loss;
  int* status;
  int64_t step;
  std::vector<void*> allocs;
};

namespace {

template <typename T>
cudaError_t mlp_alloc(kde_mlp_s* m, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(16, count * sizeof(T)));
  if (e != cudaSuccess) return e;
  e = cudaMemset(q, 0, std::max<size_t>(16, count * sizeof(T)));
  m->allocs.push_back(q);
  *p = (T*)q;
  return e;
}

kde_status mlp_refresh(kde_mlp_s* m, cudaStream_t st) {
  LaunchScope ls("kde_mlp_refresh_kernel", st);
  kde_mlp_refresh_kernel<<<1024, 256, 0, st>>>(m->P + m->oW1, m->P + m->oW2, m->P + m->oW3,
                                                m->P + m->ob3, m->in, m->hid, m->out, m->outp,
                                                m->W1b, m->W2b, m->W2t, m->W3b, m->W3t, m->b3p);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_mlp_refresh_kernel");
}

GemmArgs gemm_args(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, float* C,
                   int ldc, int* status) {
  GemmArgs g{};
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.C = C;
  g.ldc = ldc;
  g.status = status;
  return g;
}

// Forward pass on the first B rows of X (B <= maxB), padded to Bp rows.
kde_status mlp_forward(kde_mlp_s* m, const float* X, int B, int Bp, bool keep_t, cudaStream_t st) {
  {
    LaunchScope ls("kde_mlp_cast_kernel", st);
    kde_mlp_cast_kernel<<<512, 256, 0, st>>>(X, B, Bp, m->in, m->Xb, keep_t ? m->Xt : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kde_mlp_cast_kernel");
  }
  GemmArgs g1 = gemm_args(m->Xb, m->in, m->W1b, m->in, Bp, m->hid, m->in, m->Z1, m->hid, m->status);
  g1.bias = m->P + m->ob1;
  g1.Cb = m->A1b;
  g1.ldcb = m->hid;
  g1.Ct = keep_t ? m->A1t : nullptr;
  g1.ldct = Bp;
  kde_status s = launch_gemm(g1, EPI_BIAS_RELU, st);
  if (s != KDE_OK) return s;
  GemmArgs g2 = gemm_args(m->A1b, m->hid, m->W2b, m->hid, Bp, m->hid, m->hid, m->Z2, m->hid, m->status);
  g2.bias = m->P + m->ob2;
  g2.Cb = m->A2b;
  g2.ldcb = m->hid;
  g2.Ct = keep_t ? m->A2t : nullptr;
  g2.ldct = Bp;
  if ((s = launch_gemm(g2, EPI_BIAS_RELU, st)) != KDE_OK) return s;
  GemmArgs g3 = gemm_args(m->A2b, m->hid, m->W3b, m->hid, Bp, m->outp, m->hid, m->Y, m->outp, m->status);
  g3.bias = m->b3p;
  return launch_gemm(g3, EPI_BIAS, st);
}

// Loss and gradients into m->G (layout of m->P) for the first B rows.
kde_status mlp_backward(kde_mlp_s* m, const float* T, int B, int Bp, float* loss_out,
                        cudaStream_t st) {
  cudaError_t e;
  {
    LaunchScope ls("kde_mlp_loss_kernel", st);
    kde_mlp_loss_kernel<<<1, 256, 0, st>>>(m->Y, m->outp, T, B, Bp, m->out, m->outp, m->dYb, m->dYt,
                                           m->G + m->ob3, loss_out ? loss_out : m->loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_mlp_loss_kernel");
  }
  // dW3^T = A2^T dY  (M = hid, N = outp, K = Bp)
  kde_status s = launch_gemm(gemm_args(m->A2t, Bp, m->dYt, Bp, m->hid, m->outp, Bp, m->dW3t,
                                       m->outp, m->status),
                             EPI_STORE, st);
  if (s != KDE_OK) return s;
  {
    LaunchScope ls("kde_mlp_w3grad_kernel", st);
    kde_mlp_w3grad_kernel<<<(m->out * m->hid + 255) / 256, 256, 0, st>>>(m->dW3t, m->hid, m->outp,
                                                                         m->out, m->G + m->oW3);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_mlp_w3grad_kernel");
  }
  // dZ2 = (dY W3) * (Z2 > 0)  (M = Bp, N = hid, K = 64)
  GemmArgs g5 = gemm_args(m->dYb, 64, m->W3t, 64, Bp, m->hid, 64, m->dZ2, m->hid, m->status);
  g5.Z = m->Z2;
  g5.ldz = m->hid;
  g5.Cb = m->dZ2b;
  g5.ldcb = m->hid;
  g5.Ct = m->dZ2t;
  g5.ldct = Bp;
  if ((s = launch_gemm(g5, EPI_RELU_GRAD, st)) != KDE_OK) return s;
  {
    LaunchScope ls("kde_mlp_colsum_kernel", st);
    kde_mlp_colsum_kernel<<<(m->hid + 255) / 256, 256, 0, st>>>(m->dZ2, m->hid, B, m->hid,
                                                                m->G + m->ob2);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_mlp_colsum_kernel");
  }
  // dW2 = dZ2^T A1  (M = hid, N = hid, K = Bp)
  if ((s = launch_gemm(gemm_args(m->dZ2t, Bp, m->A1t, Bp, m->hid, m->hid, Bp, m->G + m->oW2,
                                 m->hid, m->status),
                       EPI_STORE, st)) != KDE_OK)
    return s;
  // dZ1 = (dZ2 W2) * (Z1 > 0)  (M = Bp, N = hid, K = hid)
  GemmArgs g7 = gemm_args(m->dZ2b, m->hid, m->W2t, m->hid, Bp, m->hid, m->hid, m->dZ1, m->hid,
                          m->status);
  g7.Z = m->Z1;
  g7.ldz = m->hid;
  g7.Ct = m->dZ1t;
  g7.ldct = Bp;
  if ((s = launch_gemm(g7, EPI_RELU_GRAD, st)) != KDE_OK) return s;
  {
    LaunchScope ls("kde_mlp_colsum_kernel", st);
    kde_mlp_colsum_kernel<<<(m->hid + 255) / 256, 256, 0, st>>>(m->dZ1, m->hid, B, m->hid,
                                                                m->G + m->ob1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_mlp_colsum_kernel");
  }
  // dW1 = dZ1^T X  (M = hid, N = in, K = Bp)
  return launch_gemm(gemm_args(m->dZ1t, Bp, m->Xt, Bp, m->hid, m->in, Bp, m->G + m->oW1, m->in,
                               m->status),
                     EPI_STORE, st);
}

kde_status mlp_check_batch(const kde_mlp_s* m, int B, int* Bp) {
  if (!m || B <= 0 || B > m->maxB) return fail(KDE_ERR_INVALID_ARG, "batch size out of range");
  *Bp = (B + 127) / 128 * 128;
  return KDE_OK;
}

}  // namespace

extern "C" {

kde_status kde_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                         float* C, int ldc, int* status, kde_stream_t stream) {
  if (!A || !B || !C || !status) return fail(KDE_ERR_INVALID_ARG, "NULL pointer");
  return launch_gemm(gemm_args((const bf16*)A, lda, (const bf16*)B, ldb, M, N, K, C, ldc, status),
                     EPI_STORE, (cudaStream_t)stream);
}

kde_status kde_mlp_create(int in_dim, int hidden, int out_dim, int max_batch, uint64_t seed,
                          kde_mlp* out) {
  if (!out) return fail(KDE_ERR_INVALID_ARG, "NULL output");
  *out = nullptr;
  if (in_dim <= 0 || in_dim % 64 || hidden <= 0 || hidden % 128 || out_dim <= 0 || out_dim > 16 ||
      max_batch <= 0)
    return fail(KDE_ERR_INVALID_ARG,
                "MLP sizes: in_dim % 64 == 0, hidden % 128 == 0, 1 <= out_dim <= 16");
  kde_mlp_s* m = new kde_mlp_s();
  m->in = in_dim;
  m->hid = hidden;
  m->out = out_dim;
  m->outp = 16;
  m->maxB = max_batch;
  const int Bp = (max_batch + 127) / 128 * 128;
  m->oW1 = 0;
  m->ob1 = m->oW1 + (int64_t)hidden * in_dim;
  m->oW2 = m->ob1 + hidden;
  m->ob2 = m->oW2 + (int64_t)hidden * hidden;
  m->oW3 = m->ob2 + hidden;
  m->ob3 = m->oW3 + (int64_t)out_dim * hidden;
  m->nparam = m->ob3 + out_dim;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t count) {
    if (e == cudaSuccess) e = mlp_alloc(m, p, count);
  };
  A(&m->P, m->nparam);
  A(&m->G, m->nparam);
  A(&m->Mo, m->nparam);
  A(&m->Vo, m->nparam);
  A(&m->W1b, (size_t)hidden * in_dim);
  A(&m->W2b, (size_t)hidden * hidden);
  A(&m->W2t, (size_t)hidden * hidden);
  A(&m->W3b, (size_t)m->outp * hidden);
  A(&m->W3t, (size_t)hidden * 64);
  A(&m->Xb, (size_t)Bp * in_dim);
  A(&m->Xt, (size_t)Bp * in_dim);
  A(&m->A1b, (size_t)Bp * hidden);
  A(&m->A1t, (size_t)Bp * hidden);
  A(&m->A2b, (size_t)Bp * hidden);
  A(&m->A2t, (size_t)Bp * hidden);
  A(&m->dYb, (size_t)Bp * 64);
  A(&m->dYt, (size_t)m->outp * Bp);
  A(&m->dZ2b, (size_t)Bp * hidden);
  A(&m->dZ2t, (size_t)Bp * hidden);
  A(&m->dZ1t, (size_t)Bp * hidden);
  A(&m->Z1, (size_t)Bp * hidden);
  A(&m->Z2, (size_t)Bp * hidden);
  A(&m->Y, (size_t)Bp * m->outp);
  A(&m->dZ1, (size_t)Bp * hidden);
  A(&m->dZ2, (size_t)Bp * hidden);
  A(&m->dW3t, (size_t)hidden * m->outp);
  A(&m->b3p, (size_t)m->outp);
  A(&m->loss, 4);
  A(&m->status, 4);
  if (e != cudaSuccess) {
    kde_mlp_destroy(m);
    return cuda_fail(e, "cudaMalloc(MLP)");
  }
  // He-normal weights, zero biases, from a seeded host generator.
  std::vector<float> h(m->nparam, 0.f);
  std::mt19937_64 rng(seed);
  auto fill = [&](int64_t off, int rows, int cols) {
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / cols));
    for (int64_t i = 0; i < (int64_t)rows * cols; ++i) h[off + i] = (float)nd(rng);
  };
  fill(m->oW1, hidden, in_dim);
  fill(m->oW2, hidden, hidden);
  fill(m->oW3, out_dim, hidden);
  kde_status s = kde_mlp_set_params(m, h.data(), m->nparam);
  if (s != KDE_OK) {
    kde_mlp_destroy(m);
    return s;
  }
  *out = m;
  return KDE_OK;
}

kde_status kde_mlp_destroy(kde_mlp m) {
  if (!m) return KDE_OK;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return KDE_OK;
}

kde_status kde_mlp_param_count(kde_mlp m, int64_t* count) {
  if (!m || !count) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  *count = m->nparam;
  return KDE_OK;
}

kde_status kde_mlp_get_params(kde_mlp m, float* host, int64_t count) {
  if (!m || !host || count != m->nparam) return fail(KDE_ERR_INVALID_ARG, "bad parameter buffer");
  cudaError_t e = cudaMemcpy(host, m->P, sizeof(float) * count, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaMemcpy(params)");
}

kde_status kde_mlp_set_params(kde_mlp m, const float* host, int64_t count) {
  if (!m || !host || count != m->nparam) return fail(KDE_ERR_INVALID_ARG, "bad parameter buffer");
  cudaError_t e = cudaMemcpy(m->P, host, sizeof(float) * count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(params)");
  kde_status s = mlp_refresh(m, 0);
  if (s != KDE_OK) return s;
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_mlp_set_params");
}

kde_status kde_mlp_get_state(kde_mlp m, float* adam_m, float* adam_v, int64_t* step) {
  if (!m || !adam_m || !adam_v || !step) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaMemcpy(adam_m, m->Mo, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(adam_v, m->Vo, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
  *step = m->step;
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaMemcpy(optimizer state)");
}

kde_status kde_mlp_set_state(kde_mlp m, const float* adam_m, const float* adam_v, int64_t step) {
  if (!m || !adam_m || !adam_v || step < 0) return fail(KDE_ERR_INVALID_ARG, "bad optimizer state");
  cudaError_t e = cudaMemcpy(m->Mo, adam_m, sizeof(float) * m->nparam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->Vo, adam_v, sizeof(float) * m->nparam, cudaMemcpyHostToDevice);
  m->step = step;
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaMemcpy(optimizer state)");
}

kde_status kde_mlp_forward(kde_mlp m, const float* X, int B, float* Y, kde_stream_t stream) {
  int Bp;
  kde_status s = mlp_check_batch(m, B, &Bp);
  if (s != KDE_OK) return s;
  if (!X || !Y) return fail(KDE_ERR_INVALID_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = mlp_forward(m, X, B, Bp, false, st)) != KDE_OK) return s;
  LaunchScope ls("kde_mlp_take_kernel", st);
  kde_mlp_take_kernel<<<(B * m->out + 255) / 256, 256, 0, st>>>(m->Y, m->outp, B, m->out, Y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_mlp_take_kernel");
}

kde_status kde_mlp_loss_grad(kde_mlp m, const float* X, const float* T, int B, float* loss,
                             float* grads, kde_stream_t stream) {
  int Bp;
  kde_status s = mlp_check_batch(m, B, &Bp);
  if (s != KDE_OK) return s;
  if (!X || !T) return fail(KDE_ERR_INVALID_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = mlp_forward(m, X, B, Bp, true, st)) != KDE_OK) return s;
  if ((s = mlp_backward(m, T, B, Bp, loss, st)) != KDE_OK) return s;
  if (grads) {
    cudaError_t e = cudaMemcpyAsync(grads, m->G, sizeof(float) * m->nparam,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(grads)");
  }
  return KDE_OK;
}

kde_status kde_mlp_train_step(kde_mlp m, const float* X, const float* T, int B, float lr,
                              float* loss, kde_stream_t stream) {
  kde_status s = kde_mlp_loss_grad(m, X, T, B, loss, nullptr, stream);
  if (s != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow((double)b1, (double)m->step);
  const float c2 = 1.f - (float)std::pow((double)b2, (double)m->step);
  {
    LaunchScope ls("kde_mlp_adam_kernel", st);
    kde_mlp_adam_kernel<<<512, 256, 0, st>>>(m->P, m->G, m->Mo, m->Vo, m->nparam, lr, b1, b2,
                                             1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kde_mlp_adam_kernel");
  }
  return mlp_refresh(m, st);
}

kde_status kde_mlp_status(kde_mlp m, int* flag) {
  if (!m || !flag) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(flag, m->status, sizeof(int), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_mlp_status");
}

kde_status kde_mlp_status_copy(kde_mlp m, int* dst, kde_stream_t stream) {
  if (!m || !dst) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(dst, m->status, sizeof(int), cudaMemcpyDefault,
                                  (cudaStream_t)stream);
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_mlp_status_copy");
}

kde_status kde_standardize2(const float* X, int64_t n, float* Z, double* moments,
                            kde_stream_t stream) {
  if (!X || !Z || !moments || n < 2) return fail(KDE_ERR_INVALID_ARG, "bad standardisation input");
  cudaStream_t st = (cudaStream_t)stream;
  LaunchScope ls("kde_standardize2_kernel", st);
  kde_standardize2_kernel<<<1, 1024, 0, st>>>(X, n, Z, moments);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_standardize2_kernel");
}

kde_status kde_features2(const int64_t* counts, int M, int64_t n, const double* moments,
                         float* feat, kde_stream_t stream) {
  if (!counts || !moments || !feat || M < 32 || M % 32 || n < 1)
    return fail(KDE_ERR_INVALID_ARG, "features: M must be a multiple of 32");
  cudaStream_t st = (cudaStream_t)stream;
  LaunchScope ls("kde_features2_kernel", st);
  kde_features2_kernel<<<32, 256, 0, st>>>((const long long*)counts, M, n, moments, feat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_features2_kernel");
}

}  // extern "C"
