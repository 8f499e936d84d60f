// First pass of the evaluation (Eq. 10 along the last axis) as a dense
// DFT-matrix product on the tensor cores, in split TF32.
//
// Each zero-padded row of counts (M_last data points of a length-P row) has
// the half spectrum X_q = sum_{x < M_last} c_x e^{-2 pi i q x / P},
// q < Q = P/2 + 1.  With F the real 2Q x M_last matrix of rows
// (cos, -sin)(2 pi q x / P), all rows at once are D = C F^T: a GEMM with
// M = the number of rows, N = 2Q, K = M_last, whose output columns 2q, 2q+1
// are Re, Im of X_q (the half-spectrum layout of the FFT path).  Zero
// padding costs nothing: F simply stops at M_last.
//
// Precision: the tensor cores read FP32 operands as TF32 (10 explicit
// significand bits).  Both operands are split, x = x_hi + x_lo with x_hi
// rounded to TF32 and x_lo = x - x_hi exact in FP32, and three products are
// accumulated in FP32: hi*hi + hi*lo + lo*hi (the lo*lo term is below
// 2^-20 relative).  The counts are converted from int64 to FP32 first.
//
// Kernel: CTA tile 128 rows x 64 columns, K in slices of 32 (four MMAs of
// K = 8 per split pair); tiles in shared memory in the no-swizzle canonical
// layout (8-row x 16-byte core matrices, 128 bytes between K-adjacent core
// matrices, 1024 between 8-row groups), two stages: while the tensor cores
// run on one slice the threads fill the other.  tcgen05.mma is issued by
// one thread, accumulators live in tensor memory and are read back with
// tcgen05.ld; every wait is bounded and reports through a status word.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "kde_internal.h"
#include "tc_wait.cuh"

namespace kde {
namespace {

constexpr int kSlice = 32;  // K elements per shared-memory stage

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t desc_nosw(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(1024u >> 4) << 32) | (1ull << 46);
}

// x rounded to TF32 (10 significand bits, ties away from zero in magnitude).
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

struct TcArgs {
  const long long* counts;  // rows x M1 int64
  int64_t rows;
  int M1;                   // data points per row (K before padding)
  int K;                    // padded to a multiple of kSlice
  int Q;
  const float* Fhi;         // N x K
  const float* Flo;
  float2* out;              // rows x Q
  int* status;
};

// One thread's share of an A slice (128 rows x 32 counts): 8 groups of 4
// consecutive counts of one row, group i = tid + 128 j.
struct ASlice {
  long long v[32];
};

__device__ __forceinline__ void load_a(const TcArgs& a, ASlice& r, int64_t m0, int k0) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int i = threadIdx.x + 128 * j, row_in = i >> 3, c = i & 7;
    const int64_t row = m0 + row_in;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int x = k0 + 4 * c + u;
      r.v[4 * j + u] = (row < a.rows && x < a.M1) ? __ldg(a.counts + row * a.M1 + x) : 0ll;
    }
  }
}

// Counts -> FP32 -> TF32 high part and exact remainder, into the stage.
__device__ __forceinline__ void store_a(const ASlice& r, uint8_t* Ahi, uint8_t* Alo) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int i = threadIdx.x + 128 * j, row_in = i >> 3, c = i & 7;
    float hv[4], lv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long q = r.v[4 * j + u];
      const float v = fmaf((float)(int)(q >> 32), 4294967296.0f, (float)(unsigned)(unsigned long long)q);
      hv[u] = tf32_hi(v);
      lv[u] = v - hv[u];
    }
    const int off = (row_in >> 3) * 1024 + c * 128 + (row_in & 7) * 16;
    *reinterpret_cast<float4*>(Ahi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4*>(Alo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
}

// B (BN rows of F hi and lo x 32) with cp.async, one commit group.
template <int BN>
__device__ __forceinline__ void copy_b(const TcArgs& a, uint8_t* Bhi, uint8_t* Blo, int n0, int k0) {
  for (int i = threadIdx.x; i < BN * 8 * 2; i += 128) {
    const int h = i / (BN * 8), j = i % (BN * 8);
    const int r = j >> 3, c = j & 7;
    const float* F = h ? a.Flo : a.Fhi;
    const size_t src = __cvta_generic_to_global(F + (size_t)(n0 + r) * a.K + k0 + 4 * c);
    const uint32_t dst = su32((h ? Blo : Bhi) + (r >> 3) * 1024 + c * 128 + (r & 7) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Two stages; the counts of slice k+2 are loaded into registers while the
// tensor cores run slice k and slice k+1 is written to the free stage.
template <int BN>
__global__ void __launch_bounds__(128) kde_rows_r2c_tc_kernel(TcArgs a) {
  constexpr int kStage = 2 * 16384 + 2 * BN * 128;  // A hi, A lo (16 KB each), B hi, B lo
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  const int n0 = blockIdx.y * BN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // kind::tf32 instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32
  // (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  const int nk = a.K / kSlice;
  uint32_t phase = 0u, used = 0u;
  bool ok = true;
  ASlice reg;
  // prologue: slice 0 into stage 0, slice 1 into registers
  copy_b<BN>(a, smem + 32768, smem + 32768 + BN * 128, n0, 0);
  load_a(a, reg, m0, 0);
  store_a(reg, smem, smem + 16384);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (nk > 1) load_a(a, reg, m0, kSlice);
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1, nx = st ^ 1;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ahi = su32(smem + st * kStage), alo = ahi + 16384u, bhi = ahi + 32768u,
                     blo = bhi + BN * 128u;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint64_t dah = desc_nosw(ahi + 256u * s), dal = desc_nosw(alo + 256u * s);
        const uint64_t dbh = desc_nosw(bhi + 256u * s), dbl = desc_nosw(blo + 256u * s);
        const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p, t;\n setp.ne.b32 p, %4, 0;\n setp.eq.b32 t, %4, %4;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %5, %3, t;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %6, %2, %3, t;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbh), "r"(idesc), "r"(acc), "l"(dbl), "l"(dal)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(&mbar[st]))
          : "memory");
    }
    used |= 1u << st;
    if (kt + 1 < nk) {
      // the other stage was read by the MMAs of slice kt - 1
      if ((used >> nx) & 1u) {
        const bool done = mbar_wait(su32(&mbar[nx]), (phase >> nx) & 1u);
        if (!__syncthreads_and(done)) {
          ok = false;
          break;
        }
        phase ^= 1u << nx;
        used &= ~(1u << nx);
      }
      uint8_t* sg = smem + nx * kStage;
      copy_b<BN>(a, sg + 32768, sg + 32768 + BN * 128, n0, (kt + 1) * kSlice);
      store_a(reg, sg, sg + 16384);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (kt + 2 < nk) load_a(a, reg, m0, (kt + 2) * kSlice);
    }
  }
  if (ok) {
    const int last = (nk - 1) & 1;
    const bool done = mbar_wait(su32(&mbar[last]), (phase >> last) & 1u);
    ok = __syncthreads_and(done);
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.status, 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    for (int b = 0; b < 2; ++b)
      if ((used >> b) & 1u) mbar_wait(su32(&mbar[b]), (phase >> b) & 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int64_t row = m0 + warp * 32 + lane;
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
      if (row < a.rows) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int q = (n0 + c0 + j) >> 1;
          if (q < a.Q)
            a.out[row * a.Q + q] = make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)BN)
                 : "memory");
}

template <int BN>
cudaError_t launch_tc(const TcArgs& a, int N, cudaStream_t st) {
  const int smem = 2 * (2 * 16384 + 2 * BN * 128);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kde_rows_r2c_tc_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  LaunchScope ls("kde_rows_r2c_tc_kernel", st);
  kde_rows_r2c_tc_kernel<BN><<<dim3((unsigned)((a.rows + 127) / 128), N / BN), 128, smem, st>>>(a);
  return cudaGetLastError();
}

int num_sms_dev() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

// TF32 rounding of the table entries on the host (same rule as tf32_hi).
float tf32_round_host(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

}  // namespace

kde_status dft_tc_setup(kde_plan_s* p) {
  const kde_plan_info& I = p->info;
  const int dl = I.d - 1;
  const int P = (int)I.P[dl], M1 = (int)I.M[dl], Q = (int)I.Q;
  // Tile width: the least padding of the 2Q output columns among widths
  // that still give about one CTA per SM (wider tiles re-read the counts
  // fewer times), else 64.
  int64_t rows = 1;
  for (int k = 0; k < dl; ++k) rows *= I.M[k];
  const int64_t mt = (rows + 127) / 128;
  int BN = 64;
  int64_t best = -1;
  for (int bn : {256, 128, 64}) {
    const int64_t np = (2 * Q + bn - 1) / bn * bn;
    if (mt * (np / bn) < num_sms_dev() && bn != 64) continue;
    if (best < 0 || np < best) {
      best = np;
      BN = bn;
    }
  }
  const int K = (M1 + kSlice - 1) / kSlice * kSlice, N = (2 * Q + BN - 1) / BN * BN;
  std::vector<float> tab((size_t)2 * N * K, 0.f);
  const double two_pi = 6.283185307179586476925286766559;
  for (int q = 0; q < Q; ++q)
    for (int x = 0; x < M1; ++x) {
      const int64_t m = ((int64_t)q * x) % P;  // exact angle reduction
      const double ang = two_pi * (double)m / (double)P;
      const double vals[2] = {std::cos(ang), -std::sin(ang)};
      for (int h = 0; h < 2; ++h) {
        const float v = (float)vals[h];
        const float hi = tf32_round_host(v);
        const float lo = (float)(vals[h] - (double)hi);
        tab[(size_t)(2 * q + h) * K + x] = hi;
        tab[(size_t)N * K + (size_t)(2 * q + h) * K + x] = lo;
      }
    }
  // the table (the kernel's wait status goes to the plan's status word)
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, tab.size() * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(DFT matrix)");
  e = cudaMemcpy(d, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "cudaMemcpy(DFT matrix)");
  }
  p->dft_tab = (float*)d;
  p->dft_N = N;
  p->dft_K = K;
  p->dft_BN = BN;
  return KDE_OK;
}

kde_status dft_tc_rows(const kde_plan_s* p, const long long* counts, int64_t rows, void* out,
                       cudaStream_t st) {
  TcArgs a;
  a.counts = counts;
  a.rows = rows;
  a.M1 = (int)p->info.M[p->info.d - 1];
  a.K = p->dft_K;
  a.Q = (int)p->info.Q;
  a.Fhi = p->dft_tab;
  a.Flo = p->dft_tab + (size_t)p->dft_N * p->dft_K;
  a.out = (float2*)out;
  a.status = p->status_dev;
  cudaError_t e;
  switch (p->dft_BN) {
    case 256: e = launch_tc<256>(a, p->dft_N, st); break;
    case 128: e = launch_tc<128>(a, p->dft_N, st); break;
    default: e = launch_tc<64>(a, p->dft_N, st); break;
  }
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_rows_r2c_tc_kernel");
}

}  // namespace kde
