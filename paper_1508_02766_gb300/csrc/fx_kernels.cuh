// Two-phase FFT passes (FP32) for kde_kernel_grid and kde_fft_eval, device
// side: the
// convolution of Eq. 10 in the wrapped, zero-padded form, with every line of
// padded length P = N1 N2 transformed as
//   phase A: thread n2 (0 <= n2 < N2) holds x[n2 + N2 n1], n1 < N1, takes
//            their N1-point DFT in registers, multiplies entry k1 by
//            e^{-2 pi i n2 k1 / P} and writes it to shared memory;
//   phase B: thread k1 (0 <= k1 < N1) reads those N2 values and takes their
//            N2-point DFT in registers, which gives X[k1 + N1 k2], k2 < N2.
// The inverse runs the same steps backwards (B then A, conjugate twiddles),
// so a forward transform, a pointwise product and the inverse need two
// exchanges through shared memory.  Input positions n2 + N2 n1 and output
// positions k1 + N1 k2 are contiguous across neighbouring threads, so lines
// are read from and written to global memory directly.
//
// Passes (row-major, last axis contiguous, Q = P_last/2 + 1):
//   rows:  two real rows ride in one complex line (x + i y), split into their
//          half spectra after phase B (counts, or the kernel grid generated
//          on the fly); the inverse rebuilds the pair from Hermitian symmetry
//          and writes the rows cropped;
//   cols:  B adjacent columns per block (column index fastest across
//          threads); modes forward, forward to the real kernel spectrum (two
//          Hermitian columns per line), forward * K * inverse with crop (the
//          leading axis), inverse with crop.
// Only lines that hold data are transformed and only lines that survive the
// crop are inverse-transformed; positions beyond the data are zero padding.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <set>
#include <type_traits>

#include "fx_dft.cuh"
#include "fx_pairs.h"
#include "kde_debug.cuh"
#include "kde_internal.h"
#include "kgen.cuh"
#include "pdl.cuh"

namespace kde {
namespace fx {


inline constexpr int kThreadsSmall = 512;  // block limit, factors <= 20
inline constexpr int kThreadsLarge = 384;  // block limit, factors <= KDE_TWO_PHASE_MAX
inline constexpr int kSmallMax = 20;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Calls f(std::integral_constant<int, n>) for the factor sizes of a class:
// CLS 0 the factors up to 20, CLS 1 every 7-smooth factor up to 40.
template <int CLS, typename F>
__device__ __forceinline__ void with_size(int n, F&& f) {
#define KDE_FX_CASE(v) \
  case v:              \
    f(std::integral_constant<int, v>{}); \
    break;
  if constexpr (CLS == 0) {
    switch (n) {
      KDE_FX_CASE(2) KDE_FX_CASE(3) KDE_FX_CASE(4) KDE_FX_CASE(5) KDE_FX_CASE(6)
      KDE_FX_CASE(7) KDE_FX_CASE(8) KDE_FX_CASE(9) KDE_FX_CASE(10) KDE_FX_CASE(12)
      KDE_FX_CASE(14) KDE_FX_CASE(15) KDE_FX_CASE(16) KDE_FX_CASE(18) KDE_FX_CASE(20)
      default: break;
    }
  } else {
    switch (n) {
      KDE_FX_CASE(2) KDE_FX_CASE(3) KDE_FX_CASE(4) KDE_FX_CASE(5) KDE_FX_CASE(6)
      KDE_FX_CASE(7) KDE_FX_CASE(8) KDE_FX_CASE(9) KDE_FX_CASE(10) KDE_FX_CASE(12)
      KDE_FX_CASE(14) KDE_FX_CASE(15) KDE_FX_CASE(16) KDE_FX_CASE(18) KDE_FX_CASE(20)
      KDE_FX_CASE(21) KDE_FX_CASE(24) KDE_FX_CASE(25) KDE_FX_CASE(27) KDE_FX_CASE(28)
      KDE_FX_CASE(30) KDE_FX_CASE(32) KDE_FX_CASE(35) KDE_FX_CASE(36) KDE_FX_CASE(40)
      default: break;
    }
  }
#undef KDE_FX_CASE
}

// A kernel compiled for one split calls f with its fixed size NT; a generic
// kernel (NT = 0) dispatches on the runtime size.
template <int NT, int CLS, typename F>
__device__ __forceinline__ void size_call(int n, F&& f) {
  if constexpr (NT > 0)
    f(std::integral_constant<int, NT>{});
  else
    with_size<CLS>(n, f);
}

template <int N1T, int N2T>
constexpr int block_limit() {
  return (N1T > 0 && N1T <= kSmallMax && N2T <= kSmallMax) || N1T == 0 ? kThreadsSmall : kThreadsLarge;
}

// A factor of the line split: the compile-time one where the kernel was
// compiled for its split (NT > 0), else the runtime one.
template <int NT>
__device__ __forceinline__ int factor(int runtime) {
  return NT > 0 ? NT : runtime;
}

// Runtime split of a line: P = N1 N2; k / N1 = umulhi(k, magic1) for the
// k < 2^13 that occur (magic1 = floor(2^32 / N1) + 1).
struct Line {
  int P, N1, N2, N3;  // N3 = 0: two factors
  unsigned magic1;
};

// Phase A forward tail: x holds the N1 inputs of thread n2; DFT, twiddle by
// e^{-2 pi i n2 k1 / P} (table tw[m] = e^{-2 pi i m / P}, m = n2 k1 < P),
// store entry k1 at dst[k1 * SK].
template <int N1>
__device__ __forceinline__ void a_fwd_store(float2 (&x)[N1], int n2, const float2* __restrict__ tw,
                                            float2* dst, int SK) {
  dft<N1>(x);
  dst[0] = x[0];
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) dst[k1 * SK] = cmul(x[k1], __ldg(tw + n2 * k1));
}

// Phase B inverse tail: y holds X[k1 + N1 k2], k2 < N2, of thread k1;
// inverse DFT, twiddle by e^{+2 pi i n2 k1 / P}, store entry n2 at dst[n2 * SN].
template <int N2>
__device__ __forceinline__ void b_inv_store(float2 (&y)[N2], int k1, const float2* __restrict__ tw,
                                            float2* dst, int SN) {
  idft<N2>(y);
  dst[0] = y[0];
#pragma unroll
  for (int n2 = 1; n2 < N2; ++n2) dst[n2 * SN] = cmulc(y[n2], __ldg(tw + n2 * k1));
}

// ---------------------------------------------------------------------------
// Row passes.  Line b of the block is the row pair (r0, r0 + 1), r0 =
// 2 (blockIdx.x B + b).  Exchange buffer per line: entry (k1, n2) at
// k1 SK + n2 (SK odd), lines N1 SK apart.
// ---------------------------------------------------------------------------
struct RowsArgs {
  int64_t nrows;      // real rows
  int Min;            // data length of an input row (counts); zero beyond
  int64_t in_stride;  // elements between input rows
  int Q;
  int Mout;           // c2r: output row length (crop)
  Line ln;
  int B;              // row pairs per block
  int SK;
  float2* out;        // forward: half spectra [nrows][Q]
  const float2* in;   // c2r: half spectra [nrows][Q]
  float* out_real;    // c2r: rows [nrows][Mout]
  const float2* tw;
  // Batched bandwidths (grid.y = bandwidth h): the kernel grid of h from
  // gens[h] (nullptr: the kernel argument), and element offsets between
  // consecutive h of out, in and out_real.
  const KGen<float>* gens;
  int64_t slab_out, slab_in, slab_real;
};

// Per-bandwidth view of the arguments (h = blockIdx.y).
__device__ __forceinline__ void rows_slab(RowsArgs& a, KGen<float>& g) {
  const int64_t h = blockIdx.y;
  if (a.gens) {
    g = a.gens[h];
    a.nrows = g.d == 2 ? 2 * g.L[0] + 1 : (int64_t)(2 * g.L[0] + 1) * (2 * g.L[1] + 1);
  }
  if (h) {
    a.out += h * a.slab_out;
    a.in += h * a.slab_in;
    a.out_real += h * a.slab_real;
  }
}

enum { SRC_COUNTS = 0, SRC_KGEN = 1 };

template <int N1, int SRC, int N2T = 0>
__device__ __forceinline__ void rows_a_fwd(const RowsArgs& a, const long long* __restrict__ counts,
                                           const KGen<float>& g, float2* sm) {
  const int N2 = factor<N2T>(a.ln.N2);
  const int t = threadIdx.x;
  if (t >= a.B * N2) return;
  const int b = t / N2, n2 = t - b * N2;
  const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
  float2 x[N1];
  if (r0 >= a.nrows) return;
  const bool two = r0 + 1 < a.nrows;
  if constexpr (SRC == SRC_COUNTS) {
    // every load issued before any value is converted (all in flight together)
    const long long* c0 = counts + r0 * a.in_stride;
    const long long* c1 = two ? c0 + a.in_stride : c0;
    long long v0[N1], v1[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int pos = n2 + N2 * n1;
      v0[n1] = pos < a.Min ? __ldg(c0 + pos) : 0;
      v1[n1] = (pos < a.Min && two) ? __ldg(c1 + pos) : 0;
    }
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1)
      x[n1] = make_float2(count_value<float>(v0[n1]), count_value<float>(v1[n1]));
  } else {
    // kernel values staged in shared memory beyond the exchange buffers
    const float2* stage = sm + a.B * N1 * a.SK + (size_t)b * a.ln.P;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) x[n1] = stage[n2 + N2 * n1];
  }
  a_fwd_store<N1>(x, n2, a.tw, sm + b * (N1 * a.SK) + n2, a.SK);
}

// Phase B of the forward row pass: Z[k1 + N1 k2] written back to the slots
// (k1, k2) the thread read from.
template <int N2, int N1T = 0>
__device__ __forceinline__ void rows_b_fwd(const RowsArgs& a, float2* sm) {
  const int N1 = factor<N1T>(a.ln.N1);
  const int t = threadIdx.x;
  if (t >= a.B * N1) return;
  const int b = t / N1, k1 = t - b * N1;
  float2* src = sm + b * (N1 * a.SK) + k1 * a.SK;
  float2 y[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) y[n2] = src[n2];
  dft<N2>(y);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) src[k2] = y[k2];
}

// X = F(x), Y = F(y) from Z = F(x + i y) on [0, Q), stored to both rows.
template <int N1T = 0, int N2T = 0>
__device__ __forceinline__ void rows_split_store(const RowsArgs& a, const float2* sm) {
  const int N1 = factor<N1T>(a.ln.N1), P = N1T > 0 && N2T > 0 ? N1T * N2T : a.ln.P;
  for (int b = 0; b < a.B; ++b) {
    const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
    if (r0 >= a.nrows) break;
    const bool two = r0 + 1 < a.nrows;
    const float2* z = sm + b * (N1 * a.SK);
    float2* o0 = a.out + r0 * a.Q;
    for (int k = threadIdx.x; k < a.Q; k += blockDim.x) {
      const int km = k == 0 ? 0 : P - k;
      const int q = N1T > 0 ? k / N1T : (int)__umulhi((unsigned)k, a.ln.magic1);
      const int qm = N1T > 0 ? km / N1T : (int)__umulhi((unsigned)km, a.ln.magic1);
      const float2 zk = z[(k - q * N1) * a.SK + q];
      const float2 zm = z[(km - qm * N1) * a.SK + qm];
      if (!KDE_DCHECK(k < a.Q && km < P, KDE_DBG_ROWS_STORE)) continue;
      o0[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      if (two) o0[a.Q + k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
  }
}

// Kernel-grid rows: k at every position of the block's row pairs into the
// staging area (zero where the wrapped lag is beyond the support).  Row r
// enumerates the leading lags (l_0[, l_1]) with |l_k| <= L_k.
__device__ __forceinline__ void rows_stage_kgen(const RowsArgs& a, const KGen<float>& g,
                                                float2* stage) {
  const int P = a.ln.P;
  const int Llast = g.d == 2 ? g.L[1] : g.L[2];
  for (int i = threadIdx.x; i < a.B * P; i += blockDim.x) {
    const int b = i / P, pos = i - b * P;
    const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
    const int ll = wrapped_lag(pos, P, Llast);
    float v[2] = {0.f, 0.f};
    if (ll <= Llast) {
      for (int h = 0; h < 2; ++h) {
        const int64_t r = r0 + h;
        if (r >= a.nrows) break;
        int l[KDE_MAX_D] = {0, 0, 0};
        if (g.d == 2) {
          l[0] = (int)r - g.L[0];
          l[1] = ll;
        } else {
          const int w1 = 2 * g.L[1] + 1;
          l[0] = (int)(r / w1) - g.L[0];
          l[1] = (int)(r % w1) - g.L[1];
          l[2] = ll;
        }
        v[h] = kernel_value<float>(g, l);
      }
    }
    stage[i] = make_float2(v[0], v[1]);
  }
}

template <int CLS, int N1T, int N2T, int SRC>
__global__ void __launch_bounds__(block_limit<N1T, N2T>())
kde_fx_rows_fwd_kernel(RowsArgs a, const long long* __restrict__ counts, KGen<float> g) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ float2 fx_sm[];
  rows_slab(a, g);
  if constexpr (SRC == SRC_KGEN) {
    rows_stage_kgen(a, g, fx_sm + a.B * a.ln.N1 * a.SK);
    __syncthreads();
  }
  size_call<N1T, CLS>(a.ln.N1,
                      [&](auto N) { rows_a_fwd<decltype(N)::value, SRC, N2T>(a, counts, g, fx_sm); });
  __syncthreads();
  size_call<N2T, CLS>(a.ln.N2, [&](auto N) { rows_b_fwd<decltype(N)::value, N1T>(a, fx_sm); });
  __syncthreads();
  rows_split_store<N1T, N2T>(a, fx_sm);
}

// Inverse row pass, phase B: the full line Z_k = X_k + i Y_k rebuilt from
// the two half spectra (Hermitian symmetry above Q), inverse N2-point DFT.
template <int N2, int N1T = 0>
__device__ __forceinline__ void rows_b_inv(const RowsArgs& a, float2* sm) {
  const int N1 = factor<N1T>(a.ln.N1), P = N1T > 0 ? N1T * N2 : a.ln.P;
  const int t = threadIdx.x;
  if (t >= a.B * N1) return;
  const int b = t / N1, k1 = t - b * N1;
  const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
  if (r0 >= a.nrows) return;
  const bool two = r0 + 1 < a.nrows;
  const float2* x0 = a.in + r0 * a.Q;
  const float2* x1 = two ? x0 + a.Q : x0;
  float2 y[N2];
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const int k = k1 + N1 * k2;
    const bool lo = k < a.Q;
    const int kk = lo ? k : P - k;
    const float2 X = __ldg(x0 + kk);
    const float2 Y = two ? __ldg(x1 + kk) : make_float2(0.f, 0.f);
    y[k2] = lo ? make_float2(X.x - Y.y, X.y + Y.x) : make_float2(X.x + Y.y, Y.x - X.y);
  }
  b_inv_store<N2>(y, k1, a.tw, sm + b * (N1 * a.SK) + k1 * a.SK, 1);
}

// Inverse row pass, phase A: inverse N1-point DFT, rows cropped to Mout.
template <int N1, int N2T = 0>
__device__ __forceinline__ void rows_a_inv(const RowsArgs& a, const float2* sm) {
  const int N2 = factor<N2T>(a.ln.N2);
  const int t = threadIdx.x;
  if (t >= a.B * N2) return;
  const int b = t / N2, n2 = t - b * N2;
  const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
  if (r0 >= a.nrows) return;
  const bool two = r0 + 1 < a.nrows;
  const float2* src = sm + b * (N1 * a.SK) + n2;
  float2 x[N1];
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) x[k1] = src[k1 * a.SK];
  idft<N1>(x);
  float* o0 = a.out_real + r0 * a.Mout;
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    const int pos = n2 + N2 * n1;
    if (pos < a.Mout && KDE_DCHECK(r0 < a.nrows, KDE_DBG_ROWS_STORE)) {
      o0[pos] = x[n1].x;
      if (two) o0[a.Mout + pos] = x[n1].y;
    }
  }
}

template <int CLS, int N1T, int N2T>
__global__ void __launch_bounds__(block_limit<N1T, N2T>())
kde_fx_rows_c2r_kernel(RowsArgs a) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ float2 fx_sm[];
  KGen<float> g_unused;
  rows_slab(a, g_unused);
  size_call<N2T, CLS>(a.ln.N2, [&](auto N) { rows_b_inv<decltype(N)::value, N1T>(a, fx_sm); });
  __syncthreads();
  size_call<N1T, CLS>(a.ln.N1, [&](auto N) { rows_a_inv<decltype(N)::value, N2T>(a, fx_sm); });
}

// ---------------------------------------------------------------------------
// Column passes: B (a power of two) adjacent columns per block, column index
// fastest across threads.  Input [O][Nin][S], output [O][Nout][S] complex
// (or [P][S] real).  Exchange buffer: entry (column b, k1, n2) at
// b + n2 B + k1 SK with SK = B (mod 16) for B < 16 (conflict-free phase-B
// reads) and B N2 otherwise.
// ---------------------------------------------------------------------------
// COL_AUTO: COL_MID with z <- |s_pre z|^2 s_post in place of the product
// with K (the counts' power spectrum, for their autocorrelation).
enum { COL_FWD = 0, COL_FWD_REAL = 1, COL_MID = 2, COL_INV = 3, COL_AUTO = 4 };

struct ColsArgs {
  const float2* in;
  float2* out;
  float* out_real;   // COL_FWD_REAL: [P][S]
  const float* K;    // COL_MID: real spectrum [P][S]
  int64_t S;         // columns
  int Nin;           // input rows holding data (COL_INV: P)
  int Nout;          // output rows kept (crop); COL_FWD: P
  int Lw;            // >= 0: input row j holds lag j - Lw at position (j - Lw) mod P
  Line ln;
  int B, lgB, SK;
  const float2* tw;
  // Element offsets between consecutive slabs (grid.y): outer slabs of a
  // 3-D pass, or batched bandwidths (in 0 when they share the input); with
  // h_L0 (batched kernel spectra) the input of slab h holds 2 L0 + 1 wrapped
  // rows with L0 = h_L0[h].
  int64_t slab_in, slab_out, slab_real, slab_K;
  const int* h_L0;
  float s_pre, s_post;  // COL_AUTO scales
  // Optional: counts (clear_n words) that the pass before this one has
  // consumed, set to zero by this pass's threads once their work is done.
  unsigned long long* clear;
  int64_t clear_n;
};

// Zeroes words [0, n) of c with every thread of the grid (16-byte stores
// where c is aligned).  Called where every thread of the kernel arrives.
__device__ __forceinline__ void clear_words(unsigned long long* c, int64_t n) {
  const int64_t nthr = (int64_t)gridDim.x * gridDim.y * blockDim.x;
  const int64_t tid = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
  if (((uintptr_t)c & 15) == 0) {
    ulonglong2* c2 = reinterpret_cast<ulonglong2*>(c);
    for (int64_t i = tid; i < n / 2; i += nthr) c2[i] = make_ulonglong2(0ull, 0ull);
    if (tid == 0 && (n & 1)) c[n - 1] = 0ull;
  } else {
    for (int64_t i = tid; i < n; i += nthr) c[i] = 0ull;
  }
}

// Per-slab view of the arguments (slab = blockIdx.y).
__device__ __forceinline__ void cols_slab(ColsArgs& a) {
  const int64_t h = blockIdx.y;
  if (a.h_L0) {
    a.Lw = a.h_L0[h];
    a.Nin = 2 * a.Lw + 1;
  }
  if (h) {
    a.in += h * a.slab_in;
    a.out += h * a.slab_out;
    a.out_real += h * a.slab_real;
    a.K += h * a.slab_K;
  }
}

// Input row feeding transform position pos, or -1 for zero padding.
__device__ __forceinline__ int col_source(int pos, int P, int Lw, int Nin) {
  if (Lw < 0) return pos < Nin ? pos : -1;
  const int l = wrapped_lag(pos, P, Lw);
  return l <= Lw ? l + Lw : -1;
}

template <int MODE>
__device__ __forceinline__ int64_t col_first(const ColsArgs& a) {
  return (int64_t)blockIdx.x * a.B * (MODE == COL_FWD_REAL ? 2 : 1);
}

template <int N1, int MODE, int N2T = 0>
__device__ __forceinline__ void cols_a_fwd(const ColsArgs& a, float2* sm) {
  const int N2 = factor<N2T>(a.ln.N2);
  const int t = threadIdx.x;
  if (t >= (a.B << 0) * N2) return;
  const int b = t & (a.B - 1), n2 = t >> a.lgB;
  const float2* in = a.in;
  float2 x[N1];
  if constexpr (MODE == COL_FWD_REAL) {
    const int64_t s = col_first<MODE>(a) + 2 * b;
    const bool v0 = s < a.S, v1 = s + 1 < a.S;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int j = col_source(n2 + N2 * n1, a.ln.P, a.Lw, a.Nin);
      float2 p = make_float2(0.f, 0.f), q = make_float2(0.f, 0.f);
      if (j >= 0) {
        if (v0) p = __ldg(in + (int64_t)j * a.S + s);
        if (v1) q = __ldg(in + (int64_t)j * a.S + s + 1);
      }
      x[n1] = make_float2(p.x - q.y, p.y + q.x);  // p + i q
    }
  } else {
    const int64_t s = col_first<MODE>(a) + b;
    const bool v = s < a.S;
    if (a.Lw < 0) {
      // plain rows: position pos reads row pos < Nin; the row pointer steps
      // by N2 rows per value
      const float2* p = in + s + (int64_t)n2 * a.S;
      const int64_t step = (int64_t)N2 * a.S;
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) {
        const int pos = n2 + N2 * n1;
        x[n1] = (pos < a.Nin && v) ? __ldg(p) : make_float2(0.f, 0.f);
        p += step;
      }
    } else {
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) {
        const int j = col_source(n2 + N2 * n1, a.ln.P, a.Lw, a.Nin);
        x[n1] = (j >= 0 && v && KDE_DCHECK(j < a.Nin, KDE_DBG_COLS_LOAD))
                    ? __ldg(in + (int64_t)j * a.S + s)
                    : make_float2(0.f, 0.f);
      }
    }
  }
  a_fwd_store<N1>(x, n2, a.tw, sm + b + n2 * a.B, a.SK);
}

template <int N2, int MODE, int N1T = 0>
__device__ __forceinline__ void cols_b_fwd(const ColsArgs& a, float2* sm) {
  const int N1 = factor<N1T>(a.ln.N1);
  const int t = threadIdx.x;
  if (t >= a.B * N1) return;
  const int b = t & (a.B - 1), k1 = t >> a.lgB;
  float2* src = sm + b + k1 * a.SK;
  float2 y[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) y[n2] = src[n2 * a.B];
  dft<N2>(y);
  if constexpr (MODE == COL_FWD) {
    const int64_t s = col_first<MODE>(a) + b;
    if (s >= a.S) return;
    float2* out = a.out + s + (int64_t)k1 * a.S;
    const int64_t step = (int64_t)N1 * a.S;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      if (KDE_DCHECK(k1 + N1 * k2 < a.ln.P, KDE_DBG_COLS_STORE)) *out = y[k2];
      out += step;
    }
  } else if constexpr (MODE == COL_FWD_REAL) {
    const int64_t s = col_first<MODE>(a) + 2 * b;
    if (s >= a.S) return;
    const bool v1 = s + 1 < a.S;
    float* out = a.out_real + s;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int64_t k = k1 + N1 * k2;
      out[k * a.S] = y[k2].x;
      if (v1) out[k * a.S + 1] = y[k2].y;
    }
  } else if constexpr (MODE == COL_AUTO) {  // power spectrum, inverse, back to the slots
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const float re = y[k2].x * a.s_pre, im = y[k2].y * a.s_pre;
      y[k2] = make_float2((re * re + im * im) * a.s_post, 0.f);
    }
    b_inv_store<N2>(y, k1, a.tw, src, a.B);
  } else {  // COL_MID: times K, inverse, back to the same slots
    const int64_t s = col_first<MODE>(a) + b;
    const bool v = s < a.S;
    const float* pk = a.K + s + (int64_t)k1 * a.S;
    const int64_t step = (int64_t)N1 * a.S;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const float kv = v ? __ldg(pk) : 0.f;
      pk += step;
      y[k2].x *= kv;
      y[k2].y *= kv;
    }
    b_inv_store<N2>(y, k1, a.tw, src, a.B);
  }
}

// COL_INV phase B: X[k1 + N1 k2] from the input rows, inverse N2-point DFT.
template <int N2, int N1T = 0>
__device__ __forceinline__ void cols_b_inv(const ColsArgs& a, float2* sm) {
  const int N1 = factor<N1T>(a.ln.N1);
  const int t = threadIdx.x;
  if (t >= a.B * N1) return;
  const int b = t & (a.B - 1), k1 = t >> a.lgB;
  const int64_t s = col_first<COL_INV>(a) + b;
  const bool v = s < a.S;
  const float2* in = a.in + s + (int64_t)k1 * a.S;
  const int64_t step = (int64_t)N1 * a.S;
  float2 y[N2];
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    y[k2] = v ? __ldg(in) : make_float2(0.f, 0.f);
    in += step;
  }
  b_inv_store<N2>(y, k1, a.tw, sm + b + k1 * a.SK, a.B);
}

// Inverse phase A: inverse N1-point DFT, rows cropped to Nout.
template <int N1, int MODE, int N2T = 0>
__device__ __forceinline__ void cols_a_inv(const ColsArgs& a, const float2* sm) {
  const int N2 = factor<N2T>(a.ln.N2);
  const int t = threadIdx.x;
  if (t >= a.B * N2) return;
  const int b = t & (a.B - 1), n2 = t >> a.lgB;
  const int64_t s = col_first<MODE>(a) + b;
  if (s >= a.S) return;
  const float2* src = sm + b + n2 * a.B;
  float2 x[N1];
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) x[k1] = src[k1 * a.SK];
  idft<N1>(x);
  float2* out = a.out + s + (int64_t)n2 * a.S;
  const int64_t step = (int64_t)N2 * a.S;
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    const int pos = n2 + N2 * n1;
    if (pos < a.Nout && KDE_DCHECK(s < a.S, KDE_DBG_COLS_STORE)) *out = x[n1];
    out += step;
  }
}

template <int CLS, int N1T, int N2T, int MODE>
__global__ void __launch_bounds__(block_limit<N1T, N2T>())
kde_fx_cols_kernel(ColsArgs a) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ float2 fx_sm[];
  cols_slab(a);
  if constexpr (MODE == COL_INV) {
    size_call<N2T, CLS>(a.ln.N2, [&](auto N) { cols_b_inv<decltype(N)::value, N1T>(a, fx_sm); });
    __syncthreads();
    size_call<N1T, CLS>(a.ln.N1, [&](auto N) { cols_a_inv<decltype(N)::value, MODE, N2T>(a, fx_sm); });
  } else {
    size_call<N1T, CLS>(a.ln.N1, [&](auto N) { cols_a_fwd<decltype(N)::value, MODE, N2T>(a, fx_sm); });
    __syncthreads();
    size_call<N2T, CLS>(a.ln.N2, [&](auto N) { cols_b_fwd<decltype(N)::value, MODE, N1T>(a, fx_sm); });
    if constexpr (MODE == COL_MID || MODE == COL_AUTO) {
      __syncthreads();
      size_call<N1T, CLS>(a.ln.N1, [&](auto N) { cols_a_inv<decltype(N)::value, MODE, N2T>(a, fx_sm); });
    }
  }
  if (a.clear) clear_words(a.clear, a.clear_n);
}

// Launch of the kernel for the split (N1, N2): the one compiled for it if it
// is in the list, else the generic kernel for factors up to 20.
#define KDE_FX_DISPATCH(KERNEL_T, ...)                                                   \
  if (l.n3) {                                                                          \
    switch (l.n1 * 4096 + l.n2 * 64 + l.n3) {                                          \
      KDE_FX_TRIPLES(KDE_FX_CASE_TRIPLE)                                               \
      default:                                                                         \
        return cudaErrorInvalidConfiguration;                                          \
    }                                                                                  \
  }                                                                                    \
  switch (l.n1 * 64 + l.n2) {                                                          \
    KDE_FX_PAIRS(KDE_FX_CASE_PAIR)                                                     \
    default:                                                                           \
      if (l.n1 > kSmallMax || l.n2 > kSmallMax) return cudaErrorInvalidConfiguration;  \
      return launch_kernel(KERNEL_T(0, 0), l.grid, l.threads, l.smem, l.st, __VA_ARGS__); \
  }

// ---------------------------------------------------------------------------
// Launchers, one translation unit each (fx_launch_*.cu, compiled in
// parallel): kernel of size class cls (0: factors <= 20) on the stream.
// ---------------------------------------------------------------------------
constexpr size_t kSmemMax = 227 * 1024;

template <typename F>
cudaError_t allow_smem(F* fn) {
  static std::mutex mu;
  static std::set<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count((const void*)fn)) return cudaSuccess;
  cudaFuncAttributes attr{};
  cudaError_t e = cudaFuncGetAttributes(&attr, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemMax - attr.sharedSizeBytes));
  if (e == cudaSuccess) done.insert((const void*)fn);
  return e;
}

// Every pass kernel starts with pdl_trigger(); pdl_wait(); so it may be
// launched as a programmatic dependent of the kernel before it.
template <typename Kern, typename... Args>
cudaError_t launch_kernel(Kern* fn, dim3 grid, int threads, size_t smem, cudaStream_t st,
                          Args... args) {
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return e;
  e = launch_pdl(fn, grid, dim3(threads), smem, st, args...);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

struct Launch {
  int n1, n2, n3;  // the line split (n3 = 0: two factors)
  dim3 grid;
  int threads;
  size_t smem;
  cudaStream_t st;
};

cudaError_t launch_rows_counts(const Launch& l, const RowsArgs& a, const long long* counts);
cudaError_t launch_rows_kgen(const Launch& l, const RowsArgs& a, const KGen<float>& g);
cudaError_t launch_rows_c2r(const Launch& l, const RowsArgs& a);
cudaError_t launch_cols_fwd(const Launch& l, const ColsArgs& a);
cudaError_t launch_cols_real(const Launch& l, const ColsArgs& a);
cudaError_t launch_cols_mid(const Launch& l, const ColsArgs& a);
cudaError_t launch_cols_auto(const Launch& l, const ColsArgs& a);
cudaError_t launch_cols_inv(const Launch& l, const ColsArgs& a);

}  // namespace fx
}  // namespace kde
