// The convolution step (Eq. 10) in wrapped, zero-padded form:
//   kde_kernel_grid: k_l on |l_k| <= L_k at index l mod P_k (Eq. 6, Eq. 12
//                    without the shift), transformed to its real spectrum K;
//   kde_fft_eval:    C = F(c) of the zero-padded counts, S = C K,
//                    s = F^{-1}(S), cropped to [0, M_k) (Eq. 14 shifted).
// Passes (row-major, last axis contiguous, Q = P_last/2 + 1); every line is
// transformed by a group of tpl threads (line_fft), tpl chosen per launch:
//   rows_r2c  real rows -> half spectra; two real rows ride in one complex
//             FFT (x + i y) and are separated afterwards;
//   cols      FFT along a strided axis: a block stages W adjacent columns in
//             shared memory with coalesced loads, each thread group
//             transforms one, and the block stores them back coalesced.  Modes: forward,
//             forward-to-real (the kernel spectrum, written with the
//             transformed axis contiguous), forward * K * inverse with crop
//             (the leading axis), inverse with crop;
//   rows_c2r  half spectra -> real rows, cropped (two rows per complex FFT);
//   line1d    d = 1: forward, * K, inverse and crop.
// Only lines that hold data are transformed and only lines that survive the
// crop are inverse-transformed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include "fft_engine.cuh"
#include "kde_internal.h"
#include "kde_debug.cuh"
#include "kgen.cuh"

namespace kde {
namespace {


// Global loads issued back to back by one thread before their values are
// stored to shared memory (memory-level parallelism of the load phases).
// Loads of arrays that other blocks produce (counts, spectra) take the
// L2-only path (__ldcg): the persistent batch kernel reads, within one
// launch, data that other blocks wrote after a completion counter said so.
constexpr int kLoadBatch = 8;

// Twiddle table -> shared memory by asynchronous copies (cp.async): they
// hold no registers and are in flight together with a pass's own data
// loads; twiddles_wait() completes this thread's copies, and the block
// barrier after it publishes the table.  Every thread of the block calls
// both.  Tables start on 256-byte boundaries; one whose size is an odd
// multiple of 8 bytes ends with an 8-byte copy.
template <typename V>
__device__ __forceinline__ void twiddles_async(V* tw_s, const V* tw, int P) {
  const int bytes = P * (int)sizeof(V);
  const int n16 = bytes >> 4;
  const size_t src = __cvta_generic_to_global(tw);
  const unsigned dst = (unsigned)__cvta_generic_to_shared(tw_s);
  for (int i = threadIdx.x; i < n16; i += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * i),
                 "l"(src + 16ull * i)
                 : "memory");
  if ((bytes & 15) && threadIdx.x == 0)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst + 16u * n16),
                 "l"(src + 16ull * n16)
                 : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void twiddles_wait() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
struct RowsParams {
  using V = typename Cplx<T>::type;
  int64_t nrows;      // real rows
  int Min;            // data length of a row (zero-padded to P)
  int64_t in_stride;  // elements between input rows
  int Q;
  V* out;             // complex half spectra, row stride Q
  T* out_real;        // real part only (d = 1 kernel spectrum)
  int tpl;           // threads per line
  LinePlan lp;
  const V* tw;
};

// Split Z = F(x + i y) into X = F(x), Y = F(y) for k in [0, Q) and store.
template <typename T>
__device__ __forceinline__ void store_r2c(const RowsParams<T>& p, const typename Cplx<T>::type* z,
                                          int64_t r0, const LineGroup& g) {
  using V = typename Cplx<T>::type;
  const int P = p.lp.N;
  for (int k = g.lt; k < p.Q; k += g.tpl) {
    V zk = z[k];
    V zm = z[k == 0 ? 0 : P - k];
    V X = mk<V>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
    V Y = mk<V>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
    if (!KDE_DCHECK(r0 < p.nrows, KDE_DBG_STOCKHAM)) continue;
    if (p.out_real) {
      p.out_real[r0 * p.Q + k] = X.x;
    } else {
      p.out[r0 * p.Q + k] = X;
      if (r0 + 1 < p.nrows) p.out[(r0 + 1) * p.Q + k] = Y;
    }
  }
}

// The line group of this thread (line li of the block).
__device__ __forceinline__ LineGroup line_group(int tpl, int& li) {
  li = threadIdx.x / tpl;
  return LineGroup{(int)threadIdx.x - li * tpl, tpl, 1 + li};
}

// Counts rows -> half spectra, one row pair per line group.  Counts are int64
// in units of 2^-32; the unit is folded into the kernel spectrum.
template <typename T>
__device__ __forceinline__ void rows_counts_body(const long long* __restrict__ counts,
                                                 const RowsParams<T>& p, int64_t vb) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = p.lp.N;
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  int li;
  const LineGroup g = line_group(p.tpl, li);
  V* a = tw_s + P + 2 * li * P;
  V* b = a + P;
  twiddles_async(tw_s, p.tw, P);
  const int64_t r0 = 2 * (vb * (blockDim.x / p.tpl) + li);
  const bool act = r0 < p.nrows;
  const long long* c0 = counts + r0 * p.in_stride;
  const long long* c1 = c0 + p.in_stride;
  const bool two = r0 + 1 < p.nrows;
  for (int x0 = g.lt; act && x0 < P; x0 += kLoadBatch * g.tpl) {
    long long u0[kLoadBatch], u1[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int x = x0 + u * g.tpl;
      u0[u] = x < p.Min ? __ldcg(c0 + x) : 0;
      u1[u] = (x < p.Min && two) ? __ldcg(c1 + x) : 0;
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int x = x0 + u * g.tpl;
      if (x < P) a[x] = mk<V>(count_value<T>(u0[u]), count_value<T>(u1[u]));
    }
  }
  twiddles_wait();
  __syncthreads();
  if (!act) return;
  V* z = line_fft<V, false>(a, b, p.lp, tw_s, g);
  store_r2c<T>(p, z, r0, g);
}

template <typename T>
__global__ void __launch_bounds__(256)
kde_rows_r2c_counts_kernel(const long long* __restrict__ counts, RowsParams<T> p) {
  rows_counts_body<T>(counts, p, blockIdx.x);
}

// Kernel-grid rows -> half spectra (or real spectrum for d = 1).  Row r
// enumerates the leading lags (l_0, ..., l_{d-2}) with |l_k| <= L_k; the last
// axis holds lag l at position l mod P.
template <typename T>
__device__ __forceinline__ void rows_kgen_body(const KGen<T>& gen, const RowsParams<T>& p,
                                               int64_t vb) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = p.lp.N;
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  int li;
  const LineGroup g = line_group(p.tpl, li);
  V* a = tw_s + P + 2 * li * P;
  V* b = a + P;
  twiddles_async(tw_s, p.tw, P);
  const int64_t r0 = 2 * (vb * (blockDim.x / p.tpl) + li);
  const bool act = r0 < p.nrows;
  const int Llast = gen.d == 1 ? gen.L[0] : (gen.d == 2 ? gen.L[1] : gen.L[2]);
  for (int x = g.lt; act && x < P; x += g.tpl) {
    T val[2] = {0, 0};
    const int ll = wrapped_lag(x, P, Llast);
    if (ll <= Llast) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t r = r0 + h;
        if (r >= p.nrows) break;
        // lags of this row and position, indexed statically (a runtime
        // index would put the array in local memory)
        int l[KDE_MAX_D] = {ll, 0, 0};
        if (gen.d == 2) {
          l[0] = (int)r - gen.L[0];
          l[1] = ll;
        } else if (gen.d == 3) {
          const int w1 = 2 * gen.L[1] + 1;
          l[0] = (int)(r / w1) - gen.L[0];
          l[1] = (int)(r % w1) - gen.L[1];
          l[2] = ll;
        }
        val[h] = kernel_value<T>(gen, l);
      }
    }
    a[x] = mk<V>(val[0], val[1]);
  }
  twiddles_wait();
  __syncthreads();
  if (!act) return;
  V* z = line_fft<V, false>(a, b, p.lp, tw_s, g);
  store_r2c<T>(p, z, r0, g);
}

template <typename T>
__global__ void __launch_bounds__(256)
kde_rows_r2c_kgen_kernel(KGen<T> gen, RowsParams<T> p) {
  rows_kgen_body<T>(gen, p, blockIdx.x);
}

template <typename T>
struct C2RParams {
  using V = typename Cplx<T>::type;
  const V* in;        // half spectra, row stride Q
  T* out;             // real rows, row stride Mout
  int64_t nrows;
  int Mout;
  int Q;
  int tpl;
  LinePlan lp;
  const V* tw;
};

// Half spectra -> real rows cropped to [0, Mout).  Z = X + i Y is rebuilt on
// the full length from Hermitian symmetry: Z_k = conj(X_{P-k}) + i conj(Y_{P-k})
// for k >= Q; then x + i y = F^{-1}(Z).
template <typename T>
__device__ __forceinline__ void rows_c2r_body(const C2RParams<T>& p, int64_t vb) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = p.lp.N;
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  int li;
  const LineGroup g = line_group(p.tpl, li);
  V* a = tw_s + P + 2 * li * P;
  V* b = a + P;
  twiddles_async(tw_s, p.tw, P);
  const int64_t r0 = 2 * (vb * (blockDim.x / p.tpl) + li);
  const bool act = r0 < p.nrows;
  const bool two = r0 + 1 < p.nrows;
  const V* x0 = p.in + r0 * p.Q;
  const V* x1 = x0 + p.Q;
  for (int k0 = g.lt; act && k0 < p.Q; k0 += kLoadBatch * g.tpl) {
    V X[kLoadBatch], Y[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int k = k0 + u * g.tpl;
      X[u] = k < p.Q ? __ldcg(x0 + k) : mk<V>(0, 0);
      Y[u] = (k < p.Q && two) ? __ldcg(x1 + k) : mk<V>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int k = k0 + u * g.tpl;
      if (k >= p.Q) continue;
      a[k] = mk<V>(X[u].x - Y[u].y, X[u].y + Y[u].x);
      if (k > 0 && P - k >= p.Q) a[P - k] = mk<V>(X[u].x + Y[u].y, Y[u].x - X[u].y);
    }
  }
  twiddles_wait();
  __syncthreads();
  if (!act) return;
  V* z = line_fft<V, true>(a, b, p.lp, tw_s, g);
  T* o0 = p.out + r0 * p.Mout;
  T* o1 = o0 + p.Mout;
  for (int m = g.lt; m < p.Mout; m += g.tpl) {
    V v = z[m];
    o0[m] = v.x;
    if (two) o1[m] = v.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) kde_rows_c2r_kernel(C2RParams<T> p) {
  rows_c2r_body<T>(p, blockIdx.x);
}

// d = 1: counts -> F -> * K (real, even: K_k = K_{P-k}) -> F^{-1} -> crop.
template <typename T>
__global__ void __launch_bounds__(256)
kde_line1d_kernel(const long long* __restrict__ counts, const T* __restrict__ K, T* out, int M,
                  int Q, LinePlan lp, const typename Cplx<T>::type* tw) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = lp.N;
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + P;
  V* b = a + P;
  const LineGroup g{(int)threadIdx.x, (int)blockDim.x, 1};
  twiddles_async(tw_s, tw, P);
  for (int x = g.lt; x < P; x += g.tpl) a[x] = mk<V>(x < M ? count_value<T>(counts[x]) : T(0), 0);
  twiddles_wait();
  __syncthreads();
  V* z = line_fft<V, false>(a, b, lp, tw_s, g);
  for (int k = g.lt; k < P; k += g.tpl) {
    T kv = K[k < Q ? k : P - k];
    z[k] = mk<V>(z[k].x * kv, z[k].y * kv);
  }
  g.sync();
  V* other = (z == a) ? b : a;
  V* y = line_fft<V, true>(z, other, lp, tw_s, g);
  for (int m = g.lt; m < M; m += g.tpl) out[m] = y[m].x;
}

enum ColMode { COL_FWD = 0, COL_FWD_REAL = 1, COL_MID = 2, COL_INV = 3, COL_FWD_POWER = 4,
               COL_FWD_DOT = 5, COL_AUTO = 6 };

template <typename T>
struct ColsParams {
  using V = typename Cplx<T>::type;
  const V* in;     // [O][Nin][S]
  V* out;          // [O][Nout][S]
  T* out_real;     // COL_FWD_REAL: [O][S][P] (transformed axis contiguous)
  const T* K;      // COL_MID: [S][P] real spectrum, transformed axis contiguous
  int64_t S;
  int Nin, Nout;
  int Lw;          // >= 0: input row n holds lag n - Lw (wrapped); < 0: row n at position n
  int tpl;         // threads per column
  LinePlan lp;
  const V* tw;
  // COL_FWD_POWER: out_real = w(k) |2^-32 z|^2 with k = s mod Qw the
  // last-axis frequency and w = 1 at k = 0 and k = Plw/2, else 2.
  // COL_FWD_DOT: partial[blockIdx.x] += sum over the block of W * Re z.
  int Qw, Plw;
  const T* W;
  double* partial;
  // COL_AUTO: z <- |s_pre z|^2 s_post between the forward and inverse
  // transforms (the counts' power spectrum, for their autocorrelation).
  T s_pre, s_post;
};

__device__ __forceinline__ int half_weight(int64_t s, int Q, int Plast) {
  const int k = (int)(s % Q);
  return (k == 0 || 2 * k == Plast) ? 1 : 2;
}

// Block-wide sum of one double per thread, written by thread 0.
__device__ __forceinline__ void block_sum_to(double v, double* out) {
  __shared__ double warp_part[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_part[w];
    *out = t;
  }
}

// W adjacent columns (s0 .. s0+W-1) of outer slab o, one line group each.
template <typename T, int MODE>
__device__ __forceinline__ void cols_body_slab(const ColsParams<T>& p, int64_t slab,
                                               int64_t vbx) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = p.lp.N;
  // Passes whose columns are Hermitian (the kernel spectrum's last pass: k is
  // real and even, so every column transforms to a real line) transform two
  // columns per FFT: F(x1 + i x2) = F(x1) + i F(x2) with both real.
  constexpr bool PAIRED = MODE == COL_FWD_REAL || MODE == COL_FWD_DOT;
  const int W = (PAIRED ? 2 : 1) * (blockDim.x / p.tpl);
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  // Line t owns lines[t LS ..): its buffer, then its scratch.  LS = 2P + 1
  // puts the lines of one position in different banks.
  const int LS = 2 * P + 1;
  V* lines = tw_s + P;
  int li;
  const LineGroup g = line_group(p.tpl, li);
  twiddles_async(tw_s, p.tw, P);
  const int64_t o = slab;
  const int64_t s0 = vbx * W;
  const V* in = p.in + o * (int64_t)p.Nin * p.S;
  if constexpr (PAIRED) {
    // line t holds columns s0 + 2t (real part) and s0 + 2t + 1 (imaginary)
    const int npair = W / 2;
    for (int idx0 = threadIdx.x; idx0 < P * npair; idx0 += kLoadBatch * blockDim.x) {
      V v1[kLoadBatch], v2[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = idx0 + u * blockDim.x;
        const int pos = idx / npair, t = idx - pos * npair;
        const int n = source_row(pos, P, p.Lw, p.Nin);
        const int64_t s = s0 + 2 * t;
        const bool ok = idx < P * npair && n < p.Nin;
        v1[u] = (ok && s < p.S) ? __ldcg(in + (int64_t)n * p.S + s) : mk<V>(0, 0);
        v2[u] = (ok && s + 1 < p.S) ? __ldcg(in + (int64_t)n * p.S + s + 1) : mk<V>(0, 0);
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = idx0 + u * blockDim.x;
        const int pos = idx / npair, t = idx - pos * npair;
        if (idx < P * npair) lines[t * LS + pos] = mk<V>(v1[u].x - v2[u].y, v1[u].y + v2[u].x);
      }
    }
    twiddles_wait();
    __syncthreads();
    const int64_t s1 = s0 + 2 * li;
    V* a = lines + li * LS;
    double acc = 0.0;
    if (s1 < p.S) {
      const V* z = line_fft<V, false>(a, a + P, p.lp, tw_s, g);
      const bool two = s1 + 1 < p.S;
      if (MODE == COL_FWD_REAL) {
        T* d1 = p.out_real + (o * p.S + s1) * P;
        for (int k = g.lt; k < P; k += g.tpl) {
          d1[k] = z[k].x;
          if (two) d1[P + k] = z[k].y;
        }
      } else {
        const T* W1 = p.W + s1 * P;
        T part = 0;
        for (int k0 = g.lt; k0 < P; k0 += kLoadBatch * g.tpl) {
          T w1[kLoadBatch], w2[kLoadBatch];
#pragma unroll
          for (int u = 0; u < kLoadBatch; ++u) {
            const int k = k0 + u * g.tpl;
            w1[u] = k < P ? __ldg(W1 + k) : T(0);
            w2[u] = (k < P && two) ? __ldg(W1 + P + k) : T(0);
          }
#pragma unroll
          for (int u = 0; u < kLoadBatch; ++u) {
            const int k = k0 + u * g.tpl;
            if (k < P) part += w1[u] * z[k].x + w2[u] * z[k].y;
          }
        }
        acc = (double)part;
      }
    }
    if (MODE == COL_FWD_DOT) block_sum_to(acc, p.partial + blockIdx.x);
    return;
  }
  for (int idx0 = threadIdx.x; idx0 < P * W; idx0 += kLoadBatch * blockDim.x) {
    V v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int idx = idx0 + u * blockDim.x;
      const int pos = idx / W, t = idx - pos * W;
      const int n = source_row(pos, P, p.Lw, p.Nin);
      const int64_t s = s0 + t;
      v[u] = (idx < P * W && n < p.Nin && s < p.S) ? __ldcg(in + (int64_t)n * p.S + s) : mk<V>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int idx = idx0 + u * blockDim.x;
      const int pos = idx / W, t = idx - pos * W;
      if (idx < P * W) lines[t * LS + pos] = v[u];
    }
  }
  twiddles_wait();
  __syncthreads();
  const int64_t s = s0 + li;
  V* a = lines + li * LS;
  V* b = a + P;
  V* z = a;
  if (s < p.S) {
    // COL_MID: the first kLoadBatch values of the column's K per thread are
    // loaded before the forward transform, which hides their latency.
    T kpre[kLoadBatch];
    const T* Kc = p.K + s * P;
    if (MODE == COL_MID) {
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int k = g.lt + u * g.tpl;
        kpre[u] = k < P ? __ldcg(Kc + k) : T(0);
      }
    }
    if (MODE == COL_INV)
      z = line_fft<V, true>(a, b, p.lp, tw_s, g);
    else
      z = line_fft<V, false>(a, b, p.lp, tw_s, g);
    if (MODE == COL_MID) {
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int k = g.lt + u * g.tpl;
        if (k < P) z[k] = mk<V>(z[k].x * kpre[u], z[k].y * kpre[u]);
      }
      for (int k0 = g.lt + kLoadBatch * g.tpl; k0 < P; k0 += kLoadBatch * g.tpl) {
        T kv[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int k = k0 + u * g.tpl;
          kv[u] = k < P ? __ldcg(Kc + k) : T(0);
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int k = k0 + u * g.tpl;
          if (k < P) z[k] = mk<V>(z[k].x * kv[u], z[k].y * kv[u]);
        }
      }
      g.sync();
      V* other = (z == a) ? b : a;
      z = line_fft<V, true>(z, other, p.lp, tw_s, g);
    }
    if (MODE == COL_AUTO) {
      for (int k = g.lt; k < P; k += g.tpl) {
        const T re = z[k].x * p.s_pre, im = z[k].y * p.s_pre;
        z[k] = mk<V>((re * re + im * im) * p.s_post, T(0));
      }
      g.sync();
      V* other = (z == a) ? b : a;
      z = line_fft<V, true>(z, other, p.lp, tw_s, g);
    }
    if (MODE == COL_FWD_POWER) {
      T* dst = p.out_real + (o * p.S + s) * P;
      const T w = (T)half_weight(s, p.Qw, p.Plw);
      const T sc = (T)2.3283064365386963e-10;  // 2^-32
      for (int k = g.lt; k < P; k += g.tpl) {
        const T re = z[k].x * sc, im = z[k].y * sc;
        dst[k] = w * (re * re + im * im);
      }
    }
  }
  if (MODE == COL_FWD_POWER) return;
  // Every warp's result sits in the same buffer of its pair (same plan).
  const int zoff = (z == a) ? 0 : P;
  __syncthreads();
  const int nout = (MODE == COL_FWD) ? P : p.Nout;
  for (int idx = threadIdx.x; idx < nout * W; idx += blockDim.x) {
    const int pos = idx / W, t = idx - pos * W;
    const int64_t ss = s0 + t;
    if (ss >= p.S) continue;
    p.out[(o * nout + pos) * p.S + ss] = lines[t * LS + zoff + pos];
  }
}

template <typename T, int MODE>
__device__ __forceinline__ void cols_body(const ColsParams<T>& p) {
  cols_body_slab<T, MODE>(p, blockIdx.y, blockIdx.x);
}

// Column passes with many columns: a block holds kSimdW adjacent columns
// position-major in shared memory (element (pos, c) at pos kSimdW + c).
// Thread t works on column t mod kSimdW; the kSimdW threads of a group run
// the same butterfly on every column, so index arithmetic and twiddles are
// uniform and each group's shared and global accesses are one contiguous
// row segment of kSimdW elements.  The kernel spectrum of such a pass is
// stored [P][S] (columns contiguous).
constexpr int kSimdW = 16;
// Column kernels launch with up to this many threads (SIMD blocks: kSimdW
// lanes per butterfly group times 16 to 32 groups).
constexpr int kColsMaxThreads = 512;

template <typename V, int R, bool INV>
__device__ __forceinline__ void simd_stage(const V* __restrict__ in, V* __restrict__ out,
                                           const Stage& s, const V* __restrict__ tw, int c, int g,
                                           int ng) {
  for (int j = g; j < s.nb; j += ng) {
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = in[(j + r * s.nb) * kSimdW + c];
    int base;
    if (s.Ns > 1) {
      const unsigned q = __umulhi((unsigned)j, s.magic);
      const int k = j - (int)q * s.Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = tw[r * k * s.twstep];
        if (INV) w = cconj(w);
        x[r] = cmul(x[r], w);
      }
      base = (int)q * s.Ns * R + k;
    } else {
      base = j * R;
    }
    SmallDFT<V, R, INV>::run(x);
#pragma unroll
    for (int r = 0; r < R; ++r) out[(base + r * s.Ns) * kSimdW + c] = x[r];
  }
}

template <typename V, bool INV>
__device__ V* simd_fft(V* a, V* b, const LinePlan& lp, const V* __restrict__ tw, int c, int g,
                       int ng) {
  for (int s = 0; s < lp.nst; ++s) {
    const Stage& st = lp.st[s];
    switch (st.R) {
      case 2: simd_stage<V, 2, INV>(a, b, st, tw, c, g, ng); break;
      case 3: simd_stage<V, 3, INV>(a, b, st, tw, c, g, ng); break;
      case 4: simd_stage<V, 4, INV>(a, b, st, tw, c, g, ng); break;
      case 5: simd_stage<V, 5, INV>(a, b, st, tw, c, g, ng); break;
      case 7: simd_stage<V, 7, INV>(a, b, st, tw, c, g, ng); break;
      default: simd_stage<V, 8, INV>(a, b, st, tw, c, g, ng); break;
    }
    __syncthreads();
    V* t = a;
    a = b;
    b = t;
  }
  return a;
}

template <typename T, int MODE>
__device__ __forceinline__ void cols_simd_body_slab(const ColsParams<T>& p, int64_t slab) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = p.lp.N;
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* bufA = tw_s + P;
  V* bufB = bufA + P * kSimdW;
  const int c = threadIdx.x % kSimdW, g = threadIdx.x / kSimdW, ng = blockDim.x / kSimdW;
  twiddles_async(tw_s, p.tw, P);
  const int64_t o = slab;
  const V* in = p.in + o * (int64_t)p.Nin * p.S;
  // Hermitian columns (see cols_body_slab): a block takes 2 kSimdW columns,
  // column c and c + kSimdW share one FFT as real and imaginary parts.
  constexpr bool PAIRED = MODE == COL_FWD_REAL || MODE == COL_FWD_DOT;
  if constexpr (PAIRED) {
    const int64_t sA = (int64_t)blockIdx.x * 2 * kSimdW + c, sB = sA + kSimdW;
    for (int pos0 = g; pos0 < P; pos0 += kLoadBatch * ng) {
      V va[kLoadBatch], vb[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int pos = pos0 + u * ng;
        const int n = source_row(pos, P, p.Lw, p.Nin);
        const bool ok = pos < P && n < p.Nin;
        va[u] = (ok && sA < p.S) ? in[(int64_t)n * p.S + sA] : mk<V>(0, 0);
        vb[u] = (ok && sB < p.S) ? in[(int64_t)n * p.S + sB] : mk<V>(0, 0);
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int pos = pos0 + u * ng;
        if (pos < P) bufA[pos * kSimdW + c] = mk<V>(va[u].x - vb[u].y, va[u].y + vb[u].x);
      }
    }
    twiddles_wait();
    __syncthreads();
    const V* z = simd_fft<V, false>(bufA, bufB, p.lp, tw_s, c, g, ng);
    if (MODE == COL_FWD_DOT) {
      T part = 0;
      for (int pos0 = g; pos0 < P; pos0 += kLoadBatch * ng) {
        T wa[kLoadBatch], wb[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int pos = pos0 + u * ng;
          wa[u] = (pos < P && sA < p.S) ? __ldg(p.W + (int64_t)pos * p.S + sA) : T(0);
          wb[u] = (pos < P && sB < p.S) ? __ldg(p.W + (int64_t)pos * p.S + sB) : T(0);
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int pos = pos0 + u * ng;
          if (pos < P) {
            const V v = z[pos * kSimdW + c];
            part += wa[u] * v.x + wb[u] * v.y;
          }
        }
      }
      block_sum_to((double)part, p.partial + blockIdx.x);
    } else {
      for (int pos = g; pos < P; pos += ng) {
        const V v = z[pos * kSimdW + c];
        if (sA < p.S) p.out_real[(o * P + pos) * p.S + sA] = v.x;
        if (sB < p.S) p.out_real[(o * P + pos) * p.S + sB] = v.y;
      }
    }
    return;
  }
  const int64_t s = (int64_t)blockIdx.x * kSimdW + c;
  const bool col_ok = s < p.S;
  // kLoadBatch independent loads in flight per thread before any is stored
  for (int pos0 = g; pos0 < P; pos0 += kLoadBatch * ng) {
    V v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int pos = pos0 + u * ng;
      const int n = source_row(pos, P, p.Lw, p.Nin);
      v[u] = (pos < P && n < p.Nin && col_ok) ? in[(int64_t)n * p.S + s] : mk<V>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int pos = pos0 + u * ng;
      if (pos < P) bufA[pos * kSimdW + c] = v[u];
    }
  }
  twiddles_wait();
  __syncthreads();
  // COL_MID: this thread's first kLoadBatch values of K, loaded before the
  // forward transform.
  T kpre[kLoadBatch];
  if (MODE == COL_MID) {
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int pos = g + u * ng;
      kpre[u] = (pos < P && col_ok) ? __ldg(p.K + (int64_t)pos * p.S + s) : T(0);
    }
  }
  V* z = (MODE == COL_INV) ? simd_fft<V, true>(bufA, bufB, p.lp, tw_s, c, g, ng)
                           : simd_fft<V, false>(bufA, bufB, p.lp, tw_s, c, g, ng);
  if (MODE == COL_MID) {
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int pos = g + u * ng;
      if (pos < P) {
        V v = z[pos * kSimdW + c];
        z[pos * kSimdW + c] = mk<V>(v.x * kpre[u], v.y * kpre[u]);
      }
    }
    for (int pos0 = g + kLoadBatch * ng; pos0 < P; pos0 += kLoadBatch * ng) {
      T kv[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int pos = pos0 + u * ng;
        kv[u] = (pos < P && col_ok) ? __ldg(p.K + (int64_t)pos * p.S + s) : T(0);
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int pos = pos0 + u * ng;
        if (pos < P) {
          V v = z[pos * kSimdW + c];
          z[pos * kSimdW + c] = mk<V>(v.x * kv[u], v.y * kv[u]);
        }
      }
    }
    __syncthreads();
    V* other = (z == bufA) ? bufB : bufA;
    z = simd_fft<V, true>(z, other, p.lp, tw_s, c, g, ng);
  }
  if (MODE == COL_AUTO) {
    for (int pos = g; pos < P; pos += ng) {
      const V v = z[pos * kSimdW + c];
      const T re = v.x * p.s_pre, im = v.y * p.s_pre;
      z[pos * kSimdW + c] = mk<V>((re * re + im * im) * p.s_post, T(0));
    }
    __syncthreads();
    V* other = (z == bufA) ? bufB : bufA;
    z = simd_fft<V, true>(z, other, p.lp, tw_s, c, g, ng);
  }
  if (!col_ok) return;
  if (MODE == COL_FWD_POWER) {
    const T w = (T)half_weight(s, p.Qw, p.Plw);
    const T sc = (T)2.3283064365386963e-10;  // 2^-32
    for (int pos = g; pos < P; pos += ng) {
      const V v = z[pos * kSimdW + c];
      const T re = v.x * sc, im = v.y * sc;
      p.out_real[(o * P + pos) * p.S + s] = w * (re * re + im * im);
    }
    return;
  }
  const int nout = (MODE == COL_FWD) ? P : p.Nout;
  for (int pos = g; pos < nout; pos += ng) p.out[(o * nout + pos) * p.S + s] = z[pos * kSimdW + c];
}

template <typename T, int MODE>
__device__ __forceinline__ void cols_simd_body(const ColsParams<T>& p) {
  cols_simd_body_slab<T, MODE>(p, blockIdx.y);
}

template <typename T, bool SIMD>
__global__ void __launch_bounds__(kColsMaxThreads) kde_cols_fwd_kernel(ColsParams<T> p) {
  if (SIMD)
    cols_simd_body<T, COL_FWD>(p);
  else
    cols_body<T, COL_FWD>(p);
}
template <typename T, bool SIMD>
__global__ void __launch_bounds__(kColsMaxThreads) kde_cols_kgen_kernel(ColsParams<T> p) {
  if (SIMD)
    cols_simd_body<T, COL_FWD>(p);
  else
    cols_body<T, COL_FWD>(p);
}
template <typename T, bool SIMD>
__global__ void __launch_bounds__(kColsMaxThreads) kde_cols_kgen_real_kernel(ColsParams<T> p) {
  if (SIMD)
    cols_simd_body<T, COL_FWD_REAL>(p);
  else
    cols_body<T, COL_FWD_REAL>(p);
}
template <typename T, bool SIMD>
__global__ void __launch_bounds__(kColsMaxThreads) kde_cols_mid_kernel(ColsParams<T> p) {
  if (SIMD)
    cols_simd_body<T, COL_MID>(p);
  else
    cols_body<T, COL_MID>(p);
}
template <typename T, bool SIMD>
__global__ void __launch_bounds__(kColsMaxThreads) kde_cols_power_kernel(ColsParams<T> p) {
  if (SIMD)
    cols_simd_body<T, COL_FWD_POWER>(p);
  else
    cols_body<T, COL_FWD_POWER>(p);
}
template <typename T, bool SIMD>
__global__ void __launch_bounds__(kColsMaxThreads) kde_cols_auto_kernel(ColsParams<T> p) {
  if (SIMD)
    cols_simd_body<T, COL_AUTO>(p);
  else
    cols_body<T, COL_AUTO>(p);
}



// Batched kernel spectra (Eq. 6 and Eq. 10 for many matrices at once): one
// chunk holds up to kBatch matrices; blockIdx.y picks the matrix.
constexpr int kBatch = 64;

template <typename T>
struct BatchKGen {
  int nb;
  KGen<T> gen[kBatch];
  int rows[kBatch];       // rows of the matrix's lag grid (2 L_0 + 1; 1 for d = 1)
  int64_t off[kBatch];    // its first row in the chunk's scratch (complex elements)
};

template <typename T>
__global__ void __launch_bounds__(256) kde_rows_kgen_batch_kernel(BatchKGen<T> bk, RowsParams<T> p) {
  const int b = blockIdx.y;
  if (b >= bk.nb) return;
  // this matrix's parameters in shared memory (a per-thread copy indexed at
  // run time would live in local memory)
  __shared__ RowsParams<T> q;
  __shared__ KGen<T> gen;
  if (threadIdx.x == 0) {
    q = p;
    q.nrows = bk.rows[b];
    if (p.out_real)
      q.out_real = p.out_real + (int64_t)b * p.Q;
    else
      q.out = p.out + bk.off[b];
    gen = bk.gen[b];
  }
  __syncthreads();
  rows_kgen_body<T>(gen, q, blockIdx.x);
}

// Axis-0 pass of the batched spectra, fused with the dot product against the
// count spectrum W: no kernel spectrum is written.  Partials are laid out
// [matrix][column block].
template <typename T, bool SIMD>
__global__ void __launch_bounds__(256) kde_cols_kgen_dot_kernel(BatchKGen<T> bk, ColsParams<T> p) {
  const int b = blockIdx.y;
  if (b >= bk.nb) return;
  __shared__ ColsParams<T> q;
  if (threadIdx.x == 0) {
    q = p;
    q.in = p.in + bk.off[b];
    q.Nin = bk.rows[b];
    q.Lw = bk.gen[b].L[0];
    q.partial = p.partial + (int64_t)b * gridDim.x;
  }
  __syncthreads();
  // the bodies index the outer slab by blockIdx.y; here there is one slab
  if (SIMD)
    cols_simd_body_slab<T, COL_FWD_DOT>(q, 0);
  else
    cols_body_slab<T, COL_FWD_DOT>(q, 0, blockIdx.x);
}

// d = 1: dot of the real spectrum of matrix b with W.
template <typename T>
__global__ void __launch_bounds__(256) kde_dot1d_kernel(int nb, const T* __restrict__ K, int Q,
                                                        const T* __restrict__ W,
                                                        double* __restrict__ partial) {
  const int b = blockIdx.x;
  if (b >= nb) return;
  T part = 0;
  for (int k = threadIdx.x; k < Q; k += blockDim.x) part += W[k] * K[(int64_t)b * Q + k];
  block_sum_to((double)part, partial + b);
}

// Pair sums S_b = scale * sum of the matrix's partials (fixed order, FP64),
// then LSCV_i = S(2H_i) / n^2 - 2 (S(H_i) - n K_{H_i}(0)) / (n (n - 1)) for
// matrices ordered H_0, 2H_0, H_1, 2H_1, ...
struct LscvReduce {
  int nb, nparts;
  double scale, n;
  double K0[kBatch / 2];
};

__global__ void __launch_bounds__(32) kde_lscv_reduce_kernel(LscvReduce r, const double* __restrict__ partial,
                                                             double* __restrict__ S_out,
                                                             double* __restrict__ lscv_out) {
  const int i = blockIdx.x;  // candidate within the chunk
  if (2 * i + 1 >= r.nb) return;
  double s[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double* pp = partial + (int64_t)(2 * i + h) * r.nparts;
    double v = 0.0;
    for (int j = threadIdx.x; j < r.nparts; j += 32) v += pp[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    s[h] = __shfl_sync(0xffffffffu, v, 0) * r.scale;
  }
  if (threadIdx.x == 0) {
    if (S_out) {
      S_out[2 * i] = s[0];
      S_out[2 * i + 1] = s[1];
    }
    lscv_out[i] = s[1] / (r.n * r.n) - 2.0 * (s[0] - r.n * r.K0[i]) / (r.n * (r.n - 1.0));
  }
}

// Binned pair sums from the counts' autocorrelation R (P_0 x P_1, lag
// (l_0, l_1) at (l_0 mod P_0, l_1 mod P_1)):
//   S(A) = sum_{|l_k| <= L_k} K_A(delta o l) R(l).
// K_A and R are even, so the sum runs over the half plane l_0 > 0, or
// l_0 = 0 and l_1 > 0, twice, plus the lag 0 once.
//
// Along lag row l_0 >= 0 the Gaussian is C exp(e) in the completed squares
// of KGen (d = 2, column lag m = l_1, or |l_1| in Wand's layout):
//   e = D_0 l_0^2 + D_1 (m + b l_0)^2,  b = B_10 = b_hi + b_lo,
// so per row e_0 = D_0 l_0^2 and b l_0 are formed once.  D_0 and D_1 are
// stored times log2(e) (scaled in FP64 on the host), so each term is one
// exp2 of the exponent in base-2 units.
template <typename T>
struct AcGen {
  int L0, L1, wand;
  int rpu;     // lag rows per work unit
  int u0, nu;  // this matrix's work units [u0, u0 + nu)
  int set;     // whose autocorrelation: R + set * (P_0 P_1)
  T D0, D1, b_hi, b_lo, C;
};

// Up to kAcChunk candidates (2 kAcChunk matrices) per launch; their
// parameters and work units are uploaded to the workspace.  A work unit is
// kAcRows or more lag rows of one matrix, about kAcTerms lag terms.
constexpr int kAcChunk = 1024;
constexpr int kAcRows = 8;
constexpr int kAcTerms = 4096;

// Block u takes work unit units[u] = (matrix, first row), one warp per lag
// row, and writes one FP64 partial.  blockIdx.y > 0 scores the same units
// against autocorrelation g.set + blockIdx.y, partials at y gridDim.x.
template <typename T>
__global__ void __launch_bounds__(256) kde_lscv_ac_kernel(const AcGen<T>* __restrict__ gens,
                                                          const int2* __restrict__ units,
                                                          const T* __restrict__ Rall, int P1,
                                                          int64_t set_stride,
                                                          double* __restrict__ partial) {
  const int2 u = units[blockIdx.x];
  const AcGen<T> g = gens[u.x];
  const T* __restrict__ R = Rall + (int64_t)(g.set + blockIdx.y) * set_stride;
  partial += (int64_t)blockIdx.y * gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int r1 = min(g.L0, u.y + g.rpu - 1);
  T acc = 0;
  for (int l0 = u.y + warp; l0 <= r1; l0 += nw) {
    const T tl = (T)l0;
    const T t_hi = g.b_hi * tl;
    const T t_lo = prod_lo(g.b_hi, g.b_lo, tl, t_hi);
    const T e0 = g.D0 * tl * tl;
    const T* Rrow = R + (size_t)l0 * P1;
    T racc = 0;
    for (int l1 = (l0 == 0 ? 0 : -g.L1) + lane; l1 <= g.L1; l1 += 32) {
      const T v = ((T)(g.wand ? abs(l1) : l1) + t_hi) + t_lo;
      racc += ex2(fma(g.D1 * v, v, e0)) * __ldg(Rrow + (l1 < 0 ? l1 + P1 : l1));
    }
    // every lag of the half plane counts twice, the lag 0 (K = C) once
    if (l0 == 0 && lane == 0) racc -= T(0.5) * __ldg(Rrow);
    acc += T(2) * racc;
  }
  block_sum_to((double)(g.C * acc), partial + blockIdx.x);
}

// As kde_lscv_reduce_kernel with K_{H_i}(0) and n read from memory (kn[2i],
// kn[2i + 1]; n_all > 0 replaces every n) and scale 1; matrix 2i + h sums
// the partials of its work units.
template <typename T>
__global__ void __launch_bounds__(32) kde_lscv_ac_reduce_kernel(const AcGen<T>* __restrict__ gens,
                                                                const double* __restrict__ kn,
                                                                double n_all,
                                                                const double* __restrict__ partial,
                                                                double* __restrict__ S_out,
                                                                double* __restrict__ lscv_out) {
  const int i = blockIdx.x;
  double s[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int u0 = gens[2 * i + h].u0, nu = gens[2 * i + h].nu;
    double v = 0.0;
    for (int j = threadIdx.x; j < nu; j += 32) v += partial[u0 + j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    s[h] = __shfl_sync(0xffffffffu, v, 0);
  }
  if (threadIdx.x == 0) {
    if (S_out) {
      S_out[2 * i] = s[0];
      S_out[2 * i + 1] = s[1];
    }
    const double K0 = kn[2 * i], n = n_all > 0.0 ? n_all : kn[2 * i + 1];
    lscv_out[i] = s[1] / (n * n) - 2.0 * (s[0] - n * K0) / (n * (n - 1.0));
  }
}

// kde_lscv_ac_reduce_kernel for a prepared candidate set scored against
// many autocorrelations: blockIdx.y is the dataset (its n in nset[y], its
// partials at y nunits), outputs at y nH_all + i.
template <typename T>
__global__ void __launch_bounds__(256) kde_lscv_ac_reduce_sets_kernel(
    const AcGen<T>* __restrict__ gens, const double* __restrict__ kn,
    const double* __restrict__ nset, const double* __restrict__ partial, int nunits, int nh,
    int64_t nH_all, double* __restrict__ S_out, double* __restrict__ lscv_out) {
  // one warp per candidate, eight per block
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nh) return;
  const int lane = threadIdx.x & 31;
  const int64_t y = blockIdx.y;
  partial += y * nunits;
  double s[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int u0 = gens[2 * i + h].u0, nu = gens[2 * i + h].nu;
    double v = 0.0;
    for (int j = lane; j < nu; j += 32) v += partial[u0 + j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    s[h] = __shfl_sync(0xffffffffu, v, 0);
  }
  if (lane == 0) {
    if (S_out) {
      S_out[2 * (y * nH_all + i)] = s[0];
      S_out[2 * (y * nH_all + i) + 1] = s[1];
    }
    const double K0 = kn[2 * i], n = nset[y];
    lscv_out[y * nH_all + i] = s[1] / (n * n) - 2.0 * (s[0] - n * K0) / (n * (n - 1.0));
  }
}

// ---------------------------------------------------------------------------
// Candidates of the learned proposal built and scored on the device: for
// dataset s, candidate j < J is the network's theta_s clipped to a box plus
// offset j, candidate J the reference theta_s; theta = (a, beta, c) stands
// for H = R R^T with R = [[e^a, 0], [beta e^c, e^c]].  Each candidate gives
// the two matrices A = H and A = 2H of the LSCV criterion.
// ---------------------------------------------------------------------------
struct ThetaArgs {
  int nsets, J;
  const float* theta;     // nsets x 3 (device)
  const double* n;        // nsets
  const double* ref;      // nsets x 3
  const double* off;      // J x 3
  double box_lo[3], box_hi[3];
  double tau, delta[2];
  int M[2], P[2];
  int wand, per_axis;
  AcGen<float>* gens;     // [nsets][J + 1][2]; L0 < 0 marks a candidate that does not fit
  double* K0;             // [nsets][J + 1]: K_H(0)
};

// One thread per matrix: the same FP64 steps as the host path (H from
// theta, support by Eq. 15, Cholesky factor, completed-square constants),
// rounded to the lag sums' FP32 parameters.
__global__ void __launch_bounds__(128) kde_theta_gen_kernel(ThetaArgs t) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = 2 * (int64_t)(t.J + 1);
  if (m >= (int64_t)t.nsets * per) return;
  const int s = (int)(m / per), r = (int)(m % per), j = r >> 1, h = r & 1;
  double th[3];
  for (int k = 0; k < 3; ++k) {
    if (j < t.J) {
      const double v = (double)t.theta[3 * s + k];
      th[k] = fmin(fmax(v, t.box_lo[k]), t.box_hi[k]) + t.off[3 * j + k];
    } else {
      th[k] = t.ref[3 * s + k];
    }
  }
  const double ea = exp(th[0]), ec = exp(th[2]), b = th[1] * ec, sc = h ? 2.0 : 1.0;
  const double A00 = sc * (ea * ea), A01 = sc * (ea * b), A11 = sc * (b * b + ec * ec);
  const double mid = 0.5 * (A00 + A11), hd = 0.5 * (A00 - A11);
  const double lam = mid + sqrt(hd * hd + A01 * A01);
  int L[2];
  bool ok = isfinite(lam) && A00 > 0.0;
  const double Akk[2] = {A00, A11};
  for (int k = 0; k < 2; ++k) {
    const double half = t.per_axis ? t.tau * sqrt(Akk[k]) : t.tau * sqrt(fabs(lam));
    const double c = ceil(half / t.delta[k]);
    L[k] = c >= (double)(t.M[k] - 1) ? t.M[k] - 1 : (int)c;
    ok = ok && t.M[k] + L[k] <= t.P[k];
  }
  const double r00 = sqrt(A00), r10 = A01 / r00, r11 = sqrt(A11 - r10 * r10);
  ok = ok && r11 > 0.0;
  const double i00 = 1.0 / r00, i11 = 1.0 / r11, i10 = -(r10 * i00) / r11;
  const double D0 = -0.5 * t.delta[0] * t.delta[0] * i00 * i00;
  const double D1 = -0.5 * t.delta[1] * t.delta[1] * i11 * i11;
  const double B = i10 * t.delta[0] / (i11 * t.delta[1]);
  const double det = (r00 * r11) * (r00 * r11);
  const double C = (1.0 / 6.283185307179586476925287) / sqrt(det);
  const double log2e = 1.4426950408889634073599246810;
  AcGen<float> g{};
  g.L0 = ok ? L[0] : -1;
  g.L1 = L[1];
  g.wand = t.wand;
  g.set = s;
  g.D0 = (float)(D0 * log2e);
  g.D1 = (float)(D1 * log2e);
  g.b_hi = (float)B;
  g.b_lo = (float)(B - (double)g.b_hi);
  g.C = (float)C;
  t.gens[m] = g;
  if (h == 0) t.K0[m >> 1] = C;
}

// One block per matrix: S(A) = sum over the support of K_A(delta o l) R(l)
// with the lag-row arithmetic of kde_lscv_ac_kernel (one warp per lag row,
// FP32 terms and row sums, FP64 across warps); NaN for a candidate that
// does not fit the plan.
__global__ void __launch_bounds__(256) kde_lscv_theta_sums_kernel(const AcGen<float>* __restrict__ gens,
                                                                  const float* __restrict__ Rall,
                                                                  int P1, int64_t set_stride,
                                                                  double* __restrict__ S) {
  const AcGen<float> g = gens[blockIdx.x];
  if (g.L0 < 0) {
    if (threadIdx.x == 0) S[blockIdx.x] = nan("");
    return;
  }
  const float* __restrict__ R = Rall + (int64_t)g.set * set_stride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float acc = 0.f;
  for (int l0 = warp; l0 <= g.L0; l0 += nw) {
    const float tl = (float)l0;
    const float t_hi = g.b_hi * tl;
    const float t_lo = prod_lo(g.b_hi, g.b_lo, tl, t_hi);
    const float e0 = g.D0 * tl * tl;
    const float* Rrow = R + (size_t)l0 * P1;
    float racc = 0.f;
    for (int l1 = (l0 == 0 ? 0 : -g.L1) + lane; l1 <= g.L1; l1 += 32) {
      const float v = ((float)(g.wand ? abs(l1) : l1) + t_hi) + t_lo;
      racc += ex2(fmaf(g.D1 * v, v, e0)) * __ldg(Rrow + (l1 < 0 ? l1 + P1 : l1));
    }
    if (l0 == 0 && lane == 0) racc -= 0.5f * __ldg(Rrow);
    acc += 2.f * racc;
  }
  block_sum_to((double)(g.C * acc), S + blockIdx.x);
}

// One warp per dataset: LSCV of its J + 1 candidates (optionally stored),
// the first index of the smallest among the first J (a candidate that does
// not fit counts as +inf) and out[s] = {that index, its LSCV, the reference
// candidate's LSCV, that candidate's theta}.
__global__ void __launch_bounds__(32) kde_lscv_theta_pick_kernel(ThetaArgs t,
                                                                 const double* __restrict__ S,
                                                                 double* __restrict__ lscv,
                                                                 double* __restrict__ out) {
  const int J = t.J;
  const double* __restrict__ n_all = t.n;
  const double* __restrict__ K0 = t.K0;
  const int s = blockIdx.x;
  const double n = n_all[s];
  double best = HUGE_VAL;
  int bi = J;   // no candidate fits
  double ref = HUGE_VAL;
  for (int j = threadIdx.x; j <= J; j += 32) {
    const int64_t c = (int64_t)s * (J + 1) + j;
    const double s1 = S[2 * c], s2 = S[2 * c + 1];
    double v = s2 / (n * n) - 2.0 * (s1 - n * K0[c]) / (n * (n - 1.0));
    if (isnan(v)) v = HUGE_VAL;
    if (lscv) lscv[c] = v;
    if (j == J) ref = v;
    else if (v < best) {   // j increases per lane, so the first smallest is kept
      best = v;
      bi = j;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov < best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
    ref = fmin(ref, __shfl_down_sync(0xffffffffu, ref, off));
  }
  if (threadIdx.x == 0) {
    double th[3] = {0.0, 0.0, 0.0};
    if (bi < J)
      for (int k = 0; k < 3; ++k) {
        const double v = (double)t.theta[3 * s + k];
        th[k] = fmin(fmax(v, t.box_lo[k]), t.box_hi[k]) + t.off[3 * bi + k];
      }
    double* o = out + 6 * (int64_t)s;
    o[0] = (double)bi;
    o[1] = best;
    o[2] = ref;
    o[3] = th[0];
    o[4] = th[1];
    o[5] = th[2];
  }
}

template <typename T, bool SIMD>
__global__ void __launch_bounds__(kColsMaxThreads) kde_cols_inv_kernel(ColsParams<T> p) {
  if (SIMD)
    cols_simd_body<T, COL_INV>(p);
  else
    cols_body<T, COL_INV>(p);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
constexpr size_t kSmemMax = 227 * 1024;

template <typename F>
cudaError_t allow_smem(F* fn) {
  static std::mutex mu;
  static std::set<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count((const void*)fn)) return cudaSuccess;
  // the opt-in limit covers static and dynamic shared memory together
  cudaFuncAttributes attr{};
  cudaError_t e = cudaFuncGetAttributes(&attr, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemMax - attr.sharedSizeBytes));
  if (e == cudaSuccess) done.insert((const void*)fn);
  return e;
}

LinePlan line_plan(const kde_plan_info& info, int k) {
  LinePlan lp{};
  lp.N = (int)info.P[k];
  lp.nst = info.nstages[k];
  int Ns = 1;
  for (int s = 0; s < lp.nst; ++s) {
    Stage& st = lp.st[s];
    st.R = info.radix[k][s];
    st.Ns = Ns;
    st.nb = lp.N / st.R;
    st.twstep = lp.N / (Ns * st.R);
    st.magic = (unsigned)((1ull << 32) / (unsigned)Ns + 1ull);
    Ns *= st.R;
  }
  return lp;
}

template <typename T>
const typename Cplx<T>::type* twiddles(const kde_plan_s* plan, int k) {
  return reinterpret_cast<const typename Cplx<T>::type*>((const char*)plan->tw_dev + plan->tw_offset[k]);
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

// Launch shape for `lines` lines of length P: threads per line (tpl) grows
// with the work per line and shrinks as lines multiply, aiming at about 16
// resident warps per SM; blocks hold up to 256 threads (lines * tpl) within
// shared memory (twiddles plus two buffers per line).
struct LineShape {
  int tpl, lpb;
};

template <typename T>
LineShape line_shape(int64_t lines, int P, int lpb_min) {
  const size_t cb = sizeof(typename Cplx<T>::type);
  const int64_t target_warps = 16LL * num_sms();
  int64_t per_line = (target_warps + lines - 1) / std::max<int64_t>(1, lines);
  int tpl = 32;
  // about one radix-8 butterfly (P/8 per stage) per thread at most, and
  // room for lpb_min lines in a 256-thread block
  const int tpl_max = std::max(32, std::min(256 / lpb_min, ((P / 8 + 31) / 32) * 32));
  while (tpl * 2 <= tpl_max && tpl / 32 < per_line) tpl *= 2;
  int lpb = std::max(1, 256 / tpl);
  const int lpb_smem = (int)((kSmemMax / cb - P) / (2 * (size_t)P + 1));
  lpb = std::max(1, std::min(lpb, lpb_smem));
  // keep at least two blocks per SM where the line count allows
  while (lpb > lpb_min && (lines + lpb - 1) / lpb < 2 * num_sms()) lpb /= 2;
  lpb = std::max(lpb, std::min(lpb_min, lpb_smem));
  return {tpl, lpb};
}

template <typename T>
size_t line_smem(int P, int W) {
  return ((size_t)(1 + 2 * W) * P + W) * sizeof(typename Cplx<T>::type);
}

// Row kernels take the launch shape in their parameters (p.tpl).
template <typename T, typename Kern, typename Params, typename... Args>
kde_status launch_rows(Kern* fn, const char* name, int64_t nrows, Params& p, cudaStream_t st,
                       Args... args) {
  const int P = p.lp.N;
  const int64_t pairs = (nrows + 1) / 2;
  const LineShape sh = line_shape<T>(pairs, P, 1);
  p.tpl = sh.tpl;
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  LaunchScope ls(name, st);
  fn<<<(unsigned)((pairs + sh.lpb - 1) / sh.lpb), sh.tpl * sh.lpb, line_smem<T>(P, sh.lpb), st>>>(
      args..., p);
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, name);
}

// Column passes with at least this many 16-column tiles per SM, and whose
// tiles fit twice per SM, use the SIMD-across-columns body.
template <typename T>
bool simd_cols(int variant, int64_t columns, int P) {
  const size_t smem = (size_t)(1 + 2 * kSimdW) * P * sizeof(typename Cplx<T>::type);
  if (variant == KDE_COLS_LINES || smem > 100 * 1024) return false;
  return variant == KDE_COLS_SIMD || columns >= (int64_t)4 * kSimdW * num_sms();
}

// Threads of a SIMD column block: kSimdW lanes per butterfly group and the
// number of groups ng in 16..32 that leaves the fewest idle lanes over the
// plan's stages (a stage of nb butterflies takes ceil(nb / ng) rounds; for
// P = 280 = 8 7 5 the stages hold 35, 40, 56 butterflies: 82% of the lanes
// busy with 16 groups, 94% with 20), the larger ng on a tie.
static int simd_threads(const LinePlan& lp) {
  int best_ng = 16;
  double best = -1.0;
  for (int ng = 16; ng <= kColsMaxThreads / kSimdW; ng += 4) {
    int64_t work = 0, slots = 0;
    for (int s = 0; s < lp.nst; ++s) {
      const int nb = lp.st[s].nb;
      work += nb;
      slots += (int64_t)((nb + ng - 1) / ng) * ng;
    }
    const double u = (double)work / (double)slots;
    if (u > best + 1e-12 || (u > best - 1e-12 && ng > best_ng)) {
      best = u;
      best_ng = ng;
    }
  }
  return best_ng * kSimdW;
}

template <typename T>
using ColsKernel = void (*)(ColsParams<T>);

template <typename T>
kde_status launch_cols(ColsKernel<T> fn_lines, ColsKernel<T> fn_simd, ColsParams<T> p, int64_t O,
                       int variant, cudaStream_t st, const char* name, bool paired = false) {
  const int P = p.lp.N;
  const int per = paired ? 2 : 1;  // columns per transformed line
  cudaError_t e;
  if (simd_cols<T>(variant, p.S * O, P)) {
    if ((e = allow_smem(fn_simd)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    const size_t smem = (size_t)(1 + 2 * kSimdW) * P * sizeof(typename Cplx<T>::type);
    dim3 grid((unsigned)((p.S + per * kSimdW - 1) / (per * kSimdW)), (unsigned)O);
    LaunchScope ls(name, st);
    fn_simd<<<grid, simd_threads(p.lp), smem, st>>>(p);
  } else {
    const LineShape sh = line_shape<T>((p.S + per - 1) / per * O, P, 2);
    p.tpl = sh.tpl;
    const int W = sh.lpb * per;  // columns per block
    if ((e = allow_smem(fn_lines)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    dim3 grid((unsigned)((p.S + W - 1) / W), (unsigned)O);
    LaunchScope ls(name, st);
    fn_lines<<<grid, sh.tpl * sh.lpb, line_smem<T>(P, sh.lpb), st>>>(p);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, name);
}

#define KDE_COLS(kern) kern<T, false>, kern<T, true>

// Kernel-grid parameters of K_A (no 1/n, 2^-32 or 1/prod P folded in).
template <typename T>
kde_status kgen_for(const kde_plan_info& I, const double* A, double detA, const int64_t* L,
                    int wand, KGen<T>* g) {
  double D[3], B[3];
  kde_status st = gauss_factor(I.d, A, I.delta, D, B);
  if (st != KDE_OK) return st;
  *g = KGen<T>{};
  g->d = I.d;
  g->wand = wand;
  for (int k = 0; k < I.d; ++k) {
    g->L[k] = (int)L[k];
    g->D[k] = (T)D[k];
  }
  for (int e = 0; e < 3; ++e) {
    g->Bh[e] = (T)B[e];
    g->Bl[e] = (T)(B[e] - (double)g->Bh[e]);
  }
  g->C = (T)(std::pow(6.283185307179586476925287, -0.5 * I.d) / std::sqrt(detA));
  return KDE_OK;
}

template <typename T>
kde_status kernel_grid_impl(kde_plan_s* plan, int64_t n, void* Kspec, void* ws, cudaStream_t st) {
  using V = typename Cplx<T>::type;
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  KGen<T> gen;
  kde_status st0 = kgen_for<T>(I, plan->H, I.det_H, I.L, plan->layout_mode == KDE_LAYOUT_WAND, &gen);
  if (st0 != KDE_OK) return st0;
  double prodP = 1.0;
  for (int k = 0; k < d; ++k) prodP *= (double)I.P[k];
  const double two_pi = 6.283185307179586476925287;
  double C = std::pow(two_pi, -0.5 * d) / std::sqrt(I.det_H) / ((double)n * 4294967296.0 * prodP);
  gen.C = (T)C;
  if constexpr (std::is_same<T, float>::value) {
    if (I.engine == KDE_ENGINE_TWO_PHASE) return fx_kernel_grid(plan, gen, Kspec, ws, st);
  }
  const int dl = d - 1;
  RowsParams<T> rp{};
  rp.Q = (int)I.Q;
  rp.Min = 0;
  rp.lp = line_plan(I, dl);
  rp.tw = twiddles<T>(plan, dl);
  if (d == 1) {
    rp.nrows = 1;
    rp.out_real = (T*)Kspec;
    return launch_rows<T>(kde_rows_r2c_kgen_kernel<T>, "kde_rows_r2c_kgen_kernel", 1, rp, st, gen);
  }
  V* t1 = (V*)ws;
  int64_t rows = 1;
  for (int k = 0; k < d - 1; ++k) rows *= 2 * I.L[k] + 1;
  rp.nrows = rows;
  rp.out = t1;
  kde_status s = launch_rows<T>(kde_rows_r2c_kgen_kernel<T>, "kde_rows_r2c_kgen_kernel", rows, rp,
                                st, gen);
  if (s != KDE_OK) return s;
  if (d == 2) {
    ColsParams<T> cp{};
    cp.in = t1;
    cp.out_real = (T*)Kspec;
    cp.S = I.Q;
    cp.Nin = (int)(2 * I.L[0] + 1);
    cp.Lw = (int)I.L[0];
    cp.lp = line_plan(I, 0);
    cp.tw = twiddles<T>(plan, 0);
    return launch_cols<T>(KDE_COLS(kde_cols_kgen_real_kernel), cp, 1, plan->cols_variant, st,
                          "kde_cols_kgen_real_kernel", true);
  }
  // d == 3: axis 1 (wrapped) into t2, then axis 0 (wrapped) to the real spectrum.
  V* t2 = t1 + rows * I.Q;
  ColsParams<T> c1{};
  c1.in = t1;
  c1.out = t2;
  c1.S = I.Q;
  c1.Nin = (int)(2 * I.L[1] + 1);
  c1.Lw = (int)I.L[1];
  c1.lp = line_plan(I, 1);
  c1.tw = twiddles<T>(plan, 1);
  s = launch_cols<T>(KDE_COLS(kde_cols_kgen_kernel), c1, 2 * I.L[0] + 1, plan->cols_variant, st, "kde_cols_kgen_kernel");
  if (s != KDE_OK) return s;
  ColsParams<T> c0{};
  c0.in = t2;
  c0.out_real = (T*)Kspec;
  c0.S = I.P[1] * I.Q;
  c0.Nin = (int)(2 * I.L[0] + 1);
  c0.Lw = (int)I.L[0];
  c0.lp = line_plan(I, 0);
  c0.tw = twiddles<T>(plan, 0);
  return launch_cols<T>(KDE_COLS(kde_cols_kgen_real_kernel), c0, 1, plan->cols_variant, st,
                        "kde_cols_kgen_real_kernel", true);
}

// First pass: counts rows -> half spectra, by the FFT engine or (plans
// with dft_tc) by the tensor-core DFT-matrix product.
template <typename T>
kde_status counts_rows(kde_plan_s* plan, const long long* cnt, int64_t rows, RowsParams<T>& rp,
                       cudaStream_t st) {
  if (plan->dft_tc && sizeof(T) == sizeof(float)) return dft_tc_rows(plan, cnt, rows, rp.out, st);
  return launch_rows<T>(kde_rows_r2c_counts_kernel<T>, "kde_rows_r2c_counts_kernel", rows, rp, st,
                        cnt);
}

template <typename T>
kde_status fft_eval_impl(kde_plan_s* plan, const int64_t* counts, const void* Kspec, void* density,
                         void* ws, cudaStream_t st) {
  using V = typename Cplx<T>::type;
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  const int dl = d - 1;
  const long long* cnt = reinterpret_cast<const long long*>(counts);
  if constexpr (std::is_same<T, float>::value) {
    if (I.engine == KDE_ENGINE_TWO_PHASE)
      return fx_fft_eval(plan, cnt, (const float*)Kspec, (float*)density, ws, st);
  }
  if (d == 1) {
    const int P = (int)I.P[0];
    auto* fn = kde_line1d_kernel<T>;
    cudaError_t e = allow_smem(fn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    LaunchScope ls("kde_line1d_kernel", st);
    fn<<<1, 256, line_smem<T>(P, 1), st>>>(cnt, (const T*)Kspec, (T*)density, (int)I.M[0], (int)I.Q,
                                          line_plan(I, 0), twiddles<T>(plan, 0));
    e = cudaGetLastError();
    return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_line1d_kernel");
  }
  V* A = (V*)ws;  // [M_0 .. M_{d-2}][Q]
  int64_t rows = 1;
  for (int k = 0; k < d - 1; ++k) rows *= I.M[k];
  RowsParams<T> rp{};
  rp.nrows = rows;
  rp.Min = (int)I.M[dl];
  rp.in_stride = I.M[dl];
  rp.Q = (int)I.Q;
  rp.out = A;
  rp.lp = line_plan(I, dl);
  rp.tw = twiddles<T>(plan, dl);
  kde_status s = counts_rows<T>(plan, cnt, rows, rp, st);
  if (s != KDE_OK) return s;
  if (d == 2) {
    ColsParams<T> cp{};
    cp.in = A;
    cp.out = A;
    cp.K = (const T*)Kspec;
    cp.S = I.Q;
    cp.Nin = (int)I.M[0];
    cp.Nout = (int)I.M[0];
    cp.Lw = -1;
    cp.lp = line_plan(I, 0);
    cp.tw = twiddles<T>(plan, 0);
    s = launch_cols<T>(KDE_COLS(kde_cols_mid_kernel), cp, 1, plan->cols_variant, st, "kde_cols_mid_kernel");
    if (s != KDE_OK) return s;
  } else {
    V* B = A + rows * I.Q;  // [M_0][P_1][Q]
    ColsParams<T> c1{};
    c1.in = A;
    c1.out = B;
    c1.S = I.Q;
    c1.Nin = (int)I.M[1];
    c1.Lw = -1;
    c1.lp = line_plan(I, 1);
    c1.tw = twiddles<T>(plan, 1);
    s = launch_cols<T>(KDE_COLS(kde_cols_fwd_kernel), c1, I.M[0], plan->cols_variant, st, "kde_cols_fwd_kernel");
    if (s != KDE_OK) return s;
    ColsParams<T> c0{};
    c0.in = B;
    c0.out = B;
    c0.K = (const T*)Kspec;
    c0.S = I.P[1] * I.Q;
    c0.Nin = (int)I.M[0];
    c0.Nout = (int)I.M[0];
    c0.Lw = -1;
    c0.lp = line_plan(I, 0);
    c0.tw = twiddles<T>(plan, 0);
    s = launch_cols<T>(KDE_COLS(kde_cols_mid_kernel), c0, 1, plan->cols_variant, st, "kde_cols_mid_kernel");
    if (s != KDE_OK) return s;
    ColsParams<T> ci{};
    ci.in = B;
    ci.out = A;
    ci.S = I.Q;
    ci.Nin = (int)I.P[1];
    ci.Nout = (int)I.M[1];
    ci.Lw = -1;
    ci.lp = line_plan(I, 1);
    ci.tw = twiddles<T>(plan, 1);
    s = launch_cols<T>(KDE_COLS(kde_cols_inv_kernel), ci, I.M[0], plan->cols_variant, st, "kde_cols_inv_kernel");
    if (s != KDE_OK) return s;
  }
  C2RParams<T> cr{};
  cr.in = A;
  cr.out = (T*)density;
  cr.nrows = rows;
  cr.Mout = (int)I.M[dl];
  cr.Q = (int)I.Q;
  cr.lp = line_plan(I, dl);
  cr.tw = twiddles<T>(plan, dl);
  return launch_rows<T>(kde_rows_c2r_kernel<T>, "kde_rows_c2r_kernel", rows, cr, st);
}

// ---------------------------------------------------------------------------
// Count spectrum and batched pair sums (bandwidth selection by LSCV).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) kde_power1d_kernel(const typename Cplx<T>::type* __restrict__ X,
                                                          T* __restrict__ W, int Q, int P) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Q; k += gridDim.x * blockDim.x) {
    const T sc = (T)2.3283064365386963e-10;  // 2^-32
    const T re = X[k].x * sc, im = X[k].y * sc;
    W[k] = (T)half_weight(k, Q, P) * (re * re + im * im);
  }
}

// W = w(k) |2^-32 C|^2 on the half spectrum, in the kernel spectrum's order.
template <typename T>
kde_status power_spectrum_impl(kde_plan_s* plan, const int64_t* counts, void* Wout, void* ws,
                               cudaStream_t st) {
  using V = typename Cplx<T>::type;
  const kde_plan_info& I = plan->info;
  const int d = I.d, dl = d - 1;
  const long long* cnt = reinterpret_cast<const long long*>(counts);
  V* A = (V*)ws;
  int64_t rows = 1;
  for (int k = 0; k < d - 1; ++k) rows *= I.M[k];
  RowsParams<T> rp{};
  rp.nrows = rows;
  rp.Min = (int)I.M[dl];
  rp.in_stride = I.M[dl];
  rp.Q = (int)I.Q;
  rp.out = A;
  rp.lp = line_plan(I, dl);
  rp.tw = twiddles<T>(plan, dl);
  kde_status s = counts_rows<T>(plan, cnt, rows, rp, st);
  if (s != KDE_OK) return s;
  if (d == 1) {
    LaunchScope ls("kde_power1d_kernel", st);
    kde_power1d_kernel<T><<<(unsigned)((I.Q + 255) / 256), 256, 0, st>>>(A, (T*)Wout, (int)I.Q,
                                                                         (int)I.P[0]);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_power1d_kernel");
  }
  const V* src = A;
  int64_t S = I.Q;
  if (d == 3) {
    V* B = A + rows * I.Q;
    ColsParams<T> c1{};
    c1.in = A;
    c1.out = B;
    c1.S = I.Q;
    c1.Nin = (int)I.M[1];
    c1.Lw = -1;
    c1.lp = line_plan(I, 1);
    c1.tw = twiddles<T>(plan, 1);
    s = launch_cols<T>(KDE_COLS(kde_cols_fwd_kernel), c1, I.M[0], plan->cols_variant, st,
                       "kde_cols_fwd_kernel");
    if (s != KDE_OK) return s;
    src = B;
    S = I.P[1] * I.Q;
  }
  ColsParams<T> c0{};
  c0.in = src;
  c0.out_real = (T*)Wout;
  c0.S = S;
  c0.Nin = (int)I.M[0];
  c0.Lw = -1;
  c0.lp = line_plan(I, 0);
  c0.tw = twiddles<T>(plan, 0);
  c0.Qw = (int)I.Q;
  c0.Plw = (int)I.P[dl];
  return launch_cols<T>(KDE_COLS(kde_cols_power_kernel), c0, 1, plan->cols_variant, st,
                        "kde_cols_power_kernel");
}

// Scratch for one chunk of kBatch matrices: lag-grid rows (at most
// 2 (P_0 - M_0) + 1 per matrix, since every accepted matrix has
// M_0 + L_0 <= P_0) and the partial sums.
size_t lscv_workspace(const kde_plan_info& I) {
  const size_t cb = (I.precision == KDE_F32) ? 8 : 16;
  const int64_t rows_max = (I.d == 1) ? 1 : 2 * (I.P[0] - I.M[0]) + 1;
  int64_t S = I.Q;
  if (I.d == 3) S = I.P[1] * I.Q;
  // lag rows of the last axis for d = 2; d = 1 keeps one real spectrum row
  const size_t t1 = (size_t)kBatch * rows_max * I.Q * cb;
  const size_t parts = (size_t)kBatch * (size_t)(S + 1) * sizeof(double);
  return ((t1 + 255) & ~(size_t)255) + parts;
}

template <typename T>
kde_status lscv_impl(kde_plan_s* plan, int64_t n, int nH, const double* Hs, const void* Wsp,
                     double* S_out, double* lscv_out, void* ws, cudaStream_t st) {
  using V = typename Cplx<T>::type;
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  double prodP = 1.0;
  for (int k = 0; k < d; ++k) prodP *= (double)I.P[k];
  const size_t cb = sizeof(V);
  const int64_t rows_max = (d == 1) ? 1 : 2 * (I.P[0] - I.M[0]) + 1;
  const size_t t1_bytes = ((size_t)kBatch * rows_max * I.Q * cb + 255) & ~(size_t)255;
  V* T1 = (V*)ws;
  double* partial = (double*)((char*)ws + t1_bytes);
  int64_t S = I.Q;
  const int chunk_h = kBatch / 2;
  for (int h0 = 0; h0 < nH; h0 += chunk_h) {
    const int nh = std::min(chunk_h, nH - h0);
    BatchKGen<T> bk{};
    LscvReduce red{};
    bk.nb = 2 * nh;
    int64_t off = 0;
    int max_rows = 1;
    for (int i = 0; i < nh; ++i) {
      const double* H = Hs + (size_t)(h0 + i) * d * d;
      for (int h = 0; h < 2; ++h) {
        double A[9], Ainv[9], detA;
        int64_t L[KDE_MAX_D];
        for (int e = 0; e < d * d; ++e) A[e] = (h ? 2.0 : 1.0) * H[e];
        kde_status st2 = kde::matrix_support(plan, A, Ainv, &detA, L);
        if (st2 != KDE_OK) return st2;
        const int b = 2 * i + h;
        st2 = kgen_for<T>(I, A, detA, L, plan->layout_mode == KDE_LAYOUT_WAND, &bk.gen[b]);
        if (st2 != KDE_OK) return st2;
        bk.rows[b] = (d == 1) ? 1 : (int)(2 * L[0] + 1);
        bk.off[b] = off;
        off += (int64_t)bk.rows[b] * I.Q;
        max_rows = std::max(max_rows, bk.rows[b]);
        if (h == 0) red.K0[i] = std::pow(6.283185307179586476925287, -0.5 * d) / std::sqrt(detA);
      }
    }
    const int dl = d - 1;
    RowsParams<T> rp{};
    rp.Q = (int)I.Q;
    rp.lp = line_plan(I, dl);
    rp.tw = twiddles<T>(plan, dl);
    if (d == 1)
      rp.out_real = (T*)T1;
    else
      rp.out = T1;
    {
      const int P = rp.lp.N;
      const int64_t pairs = (max_rows + 1) / 2;
      const LineShape sh = line_shape<T>(pairs * bk.nb, P, 1);
      rp.tpl = sh.tpl;
      auto* fn = kde_rows_kgen_batch_kernel<T>;
      cudaError_t e = allow_smem(fn);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      LaunchScope ls("kde_rows_kgen_batch_kernel", st);
      dim3 grid((unsigned)((pairs + sh.lpb - 1) / sh.lpb), (unsigned)bk.nb);
      fn<<<grid, sh.tpl * sh.lpb, line_smem<T>(P, sh.lpb), st>>>(bk, rp);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_rows_kgen_batch_kernel");
    }
    int nparts;
    if (d == 1) {
      nparts = 1;
      LaunchScope ls("kde_dot1d_kernel", st);
      kde_dot1d_kernel<T><<<bk.nb, 256, 0, st>>>(bk.nb, (const T*)T1, (int)I.Q, (const T*)Wsp, partial);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "kde_dot1d_kernel");
    } else {
      ColsParams<T> cp{};
      cp.in = T1;
      cp.S = S;
      cp.lp = line_plan(I, 0);
      cp.tw = twiddles<T>(plan, 0);
      cp.W = (const T*)Wsp;
      cp.partial = partial;
      const int P = cp.lp.N;
      cudaError_t e;
      if (simd_cols<T>(plan->cols_variant, S, P)) {
        auto* fn = kde_cols_kgen_dot_kernel<T, true>;
        if ((e = allow_smem(fn)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        nparts = (int)((S + 2 * kSimdW - 1) / (2 * kSimdW));
        LaunchScope ls("kde_cols_kgen_dot_kernel", st);
        fn<<<dim3((unsigned)nparts, (unsigned)bk.nb), 256,
             (size_t)(1 + 2 * kSimdW) * P * sizeof(V), st>>>(bk, cp);
      } else {
        const LineShape sh = line_shape<T>((S + 1) / 2 * bk.nb, P, 2);
        cp.tpl = sh.tpl;
        const int Wc = 2 * sh.lpb;
        auto* fn = kde_cols_kgen_dot_kernel<T, false>;
        if ((e = allow_smem(fn)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        nparts = (int)((S + Wc - 1) / Wc);
        LaunchScope ls("kde_cols_kgen_dot_kernel", st);
        fn<<<dim3((unsigned)nparts, (unsigned)bk.nb), sh.tpl * sh.lpb, line_smem<T>(P, sh.lpb), st>>>(bk, cp);
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_cols_kgen_dot_kernel");
    }
    red.nb = bk.nb;
    red.nparts = nparts;
    red.scale = 1.0 / prodP;
    red.n = (double)n;
    {
      LaunchScope ls("kde_lscv_reduce_kernel", st);
      kde_lscv_reduce_kernel<<<nh, 32, 0, st>>>(red, partial, S_out ? S_out + 2 * h0 : nullptr,
                                                lscv_out + h0);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "kde_lscv_reduce_kernel");
    }
  }
  return KDE_OK;
}

// ---------------------------------------------------------------------------
// LSCV from the counts' autocorrelation (d = 2): R = F^{-1}|F(c)|^2 once per
// grid, then S(A) = sum over the support of K_A(delta o l) R(l) for every
// candidate -- no transform per candidate.
// ---------------------------------------------------------------------------
// Workspace: the autocorrelation's spectra, or (lag sums) the uploaded
// kernel parameters, K_H(0) and the FP64 partials of one chunk.
// At most this many work units per chunk: a unit holds kAcRows rows or more
// (the last of a matrix fewer), and L_0 < P_0 - M_0 + 1 for every matrix.
size_t ac_units_max(const kde_plan_info& I) {
  return (size_t)2 * kAcChunk * (size_t)((I.P[0] + kAcRows - 1) / kAcRows + 1);
}
// Uploaded per chunk: 2 nh AcGen, nh (K_H(0), n) pairs, then the work units.
size_t ac_upload_bytes(const kde_plan_info& I) {
  return ((size_t)2 * kAcChunk * sizeof(AcGen<double>) + (size_t)2 * kAcChunk * sizeof(double) +
          ac_units_max(I) * sizeof(int2) + 255) & ~(size_t)255;
}

size_t ac_workspace(const kde_plan_info& I) {
  const size_t cb = (I.precision == KDE_F32) ? 8 : 16;
  const size_t spec = ((size_t)(I.M[0] + I.P[0]) * I.Q * cb + 255) & ~(size_t)255;
  return std::max(spec, ac_upload_bytes(I) + ac_units_max(I) * sizeof(double));
}

template <typename T>
kde_status autocorr_impl(kde_plan_s* plan, const int64_t* counts, void* Rout, void* ws,
                         cudaStream_t st, int64_t nsets = 1, void* ws_B = nullptr) {
  using V = typename Cplx<T>::type;
  const kde_plan_info& I = plan->info;
  // nsets grids one after another: counts [nsets][M_0][M_1], R [nsets][P_0][P_1]
  V* A = (V*)ws;                                       // [nsets][M_0][Q] half spectra of the rows
  V* B = ws_B ? (V*)ws_B : A + nsets * I.M[0] * I.Q;   // [nsets][P_0][Q] after the axis-0 pass
  if constexpr (std::is_same<T, float>::value) {
    if (I.engine == KDE_ENGINE_TWO_PHASE && !plan->dft_tc)
      return fx_autocorr(plan, reinterpret_cast<const long long*>(counts), (float*)Rout, A, B,
                         nsets, st);
  }
  RowsParams<T> rp{};
  rp.nrows = nsets * I.M[0];
  rp.Min = (int)I.M[1];
  rp.in_stride = I.M[1];
  rp.Q = (int)I.Q;
  rp.out = A;
  rp.lp = line_plan(I, 1);
  rp.tw = twiddles<T>(plan, 1);
  kde_status s = counts_rows<T>(plan, reinterpret_cast<const long long*>(counts), nsets * I.M[0],
                                rp, st);
  if (s != KDE_OK) return s;
  ColsParams<T> cp{};
  cp.in = A;
  cp.out = B;
  cp.S = I.Q;
  cp.Nin = (int)I.M[0];
  cp.Nout = (int)I.P[0];
  cp.Lw = -1;
  cp.lp = line_plan(I, 0);
  cp.tw = twiddles<T>(plan, 0);
  // counts are in units of 2^-32; the inverse transforms are unnormalised
  cp.s_pre = (T)2.3283064365386963e-10;
  cp.s_post = (T)(1.0 / ((double)I.P[0] * (double)I.P[1]));
  s = launch_cols<T>(KDE_COLS(kde_cols_auto_kernel), cp, nsets, plan->cols_variant, st,
                     "kde_cols_auto_kernel");
  if (s != KDE_OK) return s;
  C2RParams<T> cr{};
  cr.in = B;
  cr.out = (T*)Rout;
  cr.nrows = nsets * I.P[0];
  cr.Mout = (int)I.P[1];
  cr.Q = (int)I.Q;
  cr.lp = line_plan(I, 1);
  cr.tw = twiddles<T>(plan, 1);
  return launch_rows<T>(kde_rows_c2r_kernel<T>, "kde_rows_c2r_kernel", nsets * I.P[0], cr, st);
}

// Host side of one chunk of lag-sum candidates: candidates c = c0 ..
// c0 + nh - 1 of set c / nH, bandwidth Hs[c], sample count ns[c / nH] (ns may
// be NULL: n is then given at launch).  Fills `up` with the device image
// AcGen[2 nh], (K0, n)[nh], work units; returns the unit count in *nunits.
template <typename T>
kde_status ac_build_chunk(kde_plan_s* plan, int64_t c0, int nh, int nH, const double* Hs,
                          const int64_t* ns, std::vector<unsigned char>& up, int* nunits) {
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  std::vector<AcGen<T>> gens(2 * nh, AcGen<T>{});
  std::vector<double> kn(2 * nh, 0.0);
  std::vector<int2> units;
  for (int i = 0; i < nh; ++i) {
    const int64_t c = c0 + i;
    const double* H = Hs + (size_t)c * d * d;
    for (int h = 0; h < 2; ++h) {
      double A[9], Ainv[9], detA;
      int64_t L[KDE_MAX_D];
      for (int e = 0; e < d * d; ++e) A[e] = (h ? 2.0 : 1.0) * H[e];
      kde_status st2 = kde::matrix_support(plan, A, Ainv, &detA, L);
      if (st2 != KDE_OK) return st2;
      KGen<T> kg;
      st2 = kgen_for<T>(I, A, detA, L, plan->layout_mode == KDE_LAYOUT_WAND, &kg);
      if (st2 != KDE_OK) return st2;
      double Dd[3], Bd[3];
      st2 = gauss_factor(I.d, A, I.delta, Dd, Bd);
      if (st2 != KDE_OK) return st2;
      const double log2e = 1.4426950408889634073599246810;  // 1 / ln 2
      AcGen<T>& g = gens[2 * i + h];
      g.L0 = kg.L[0];
      g.L1 = kg.L[1];
      g.wand = kg.wand;
      g.set = (int)(c / nH);
      g.D0 = (T)(Dd[0] * log2e);
      g.D1 = (T)(Dd[1] * log2e);
      g.b_hi = kg.Bh[0];
      g.b_lo = kg.Bl[0];
      g.C = kg.C;
      const int W = 2 * g.L1 + 1;
      g.rpu = std::max(kAcRows, (kAcTerms / W + kAcRows - 1) / kAcRows * kAcRows);
      g.u0 = (int)units.size();
      for (int r = 0; r <= g.L0; r += g.rpu) units.push_back(make_int2(2 * i + h, r));
      g.nu = (int)units.size() - g.u0;
      if (h == 0) {
        kn[2 * i] = std::pow(6.283185307179586476925287, -0.5 * d) / std::sqrt(detA);
        kn[2 * i + 1] = ns ? (double)ns[c / nH] : 0.0;
      }
    }
  }
  if (units.size() > ac_units_max(I)) return fail(KDE_ERR_UNSUPPORTED, "lag-sum work units overflow");
  const size_t gb = gens.size() * sizeof(AcGen<T>), kb = kn.size() * sizeof(double),
               ub = units.size() * sizeof(int2);
  up.resize(gb + kb + ub);
  std::memcpy(up.data(), gens.data(), gb);
  std::memcpy(up.data() + gb, kn.data(), kb);
  std::memcpy(up.data() + gb + kb, units.data(), ub);
  *nunits = (int)units.size();
  return KDE_OK;
}

// Device side of one chunk whose image (ac_build_chunk) is at `img`.
template <typename T>
kde_status ac_launch_chunk(const kde_plan_info& I, const void* img, int nh, int nunits,
                           const void* R, double* partial, double n_all, double* S_out,
                           double* lscv_out, cudaStream_t st) {
  const AcGen<T>* gens_dev = (const AcGen<T>*)img;
  const double* kn_dev = (const double*)((const char*)img + 2 * nh * sizeof(AcGen<T>));
  const int2* units_dev = (const int2*)((const char*)kn_dev + 2 * nh * sizeof(double));
  cudaError_t e;
  {
    LaunchScope ls("kde_lscv_ac_kernel", st);
    kde_lscv_ac_kernel<T><<<(unsigned)nunits, 256, 0, st>>>(
        gens_dev, units_dev, (const T*)R, (int)I.P[1], (int64_t)I.P[0] * I.P[1], partial);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kde_lscv_ac_kernel");
  }
  {
    LaunchScope ls("kde_lscv_reduce_kernel", st);
    kde_lscv_ac_reduce_kernel<T><<<nh, 32, 0, st>>>(gens_dev, kn_dev, n_all, partial, S_out, lscv_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kde_lscv_ac_reduce_kernel");
  }
  return KDE_OK;
}

// Candidates c = 0 .. nsets nH - 1 of set c / nH, bandwidth Hs[c], n[c / nH]:
// per chunk, the parameters are built on the host, copied into the
// workspace and launched.
template <typename T>
kde_status lscv_ac_impl(kde_plan_s* plan, int nsets, const int64_t* ns, int nH, const double* Hs,
                        const void* R, double* S_out, double* lscv_out, void* ws,
                        cudaStream_t st) {
  const kde_plan_info& I = plan->info;
  const int64_t total = (int64_t)nsets * nH;
  double* partial = (double*)((char*)ws + ac_upload_bytes(I));
  std::vector<unsigned char> up;
  for (int64_t h0 = 0; h0 < total; h0 += kAcChunk) {
    const int nh = (int)std::min<int64_t>(kAcChunk, total - h0);
    int nunits = 0;
    kde_status s = ac_build_chunk<T>(plan, h0, nh, nH, Hs, ns, up, &nunits);
    if (s != KDE_OK) return s;
    if ((s = upload_async(ws, up.data(), up.size(), st)) != KDE_OK) return s;
    s = ac_launch_chunk<T>(I, ws, nh, nunits, R, partial, 0.0, S_out ? S_out + 2 * h0 : nullptr,
                           lscv_out + h0, st);
    if (s != KDE_OK) return s;
  }
  return KDE_OK;
}

kde_status check_ws(const kde_plan_s* plan, void* ws, size_t bytes) {
  if (plan->info.workspace_bytes == 0) return KDE_OK;
  if (!ws) return fail(KDE_ERR_WORKSPACE, "workspace is NULL");
  if (bytes < plan->info.workspace_bytes) return fail(KDE_ERR_WORKSPACE, "workspace too small");
  if (((uintptr_t)ws & 15) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 16-byte aligned");
  return KDE_OK;
}

kde_status check_device(const kde_plan_s* plan) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device) return fail(KDE_ERR_INVALID_ARG, "plan was made on another device");
  return KDE_OK;
}

}  // namespace
}  // namespace kde

using namespace kde;

extern "C" kde_status kde_kernel_grid(kde_plan plan, int64_t n, void* Kspec, void* workspace,
                                      size_t workspace_bytes, kde_stream_t stream) {
  if (!plan || !Kspec) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(KDE_ERR_INVALID_ARG, "n must be >= 1 (the 1/n of Eq. 2)");
  kde_status s = check_ws(plan, workspace, workspace_bytes);
  if (s != KDE_OK) return s;
  if ((s = check_device(plan)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32) return kernel_grid_impl<float>(plan, n, Kspec, workspace, st);
  return kernel_grid_impl<double>(plan, n, Kspec, workspace, st);
}

extern "C" kde_status kde_fft_eval(kde_plan plan, const int64_t* counts, const void* Kspec,
                                   void* density, void* workspace, size_t workspace_bytes,
                                   kde_stream_t stream) {
  if (!plan || !counts || !Kspec || !density) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  kde_status s = check_ws(plan, workspace, workspace_bytes);
  if (s != KDE_OK) return s;
  if ((s = check_device(plan)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32)
    return fft_eval_impl<float>(plan, counts, Kspec, density, workspace, st);
  return fft_eval_impl<double>(plan, counts, Kspec, density, workspace, st);
}

// kde_fft_eval, then the counts set to zero: inside the second pass of the
// two-phase engine (the first pass is the only reader of the counts), else
// by one more operation after the evaluation.
extern "C" kde_status kde_fft_eval_consume(kde_plan plan, int64_t* counts, const void* Kspec,
                                           void* density, void* workspace, size_t workspace_bytes,
                                           kde_stream_t stream) {
  if (!plan || !counts || !Kspec || !density) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  kde_status s = check_ws(plan, workspace, workspace_bytes);
  if (s != KDE_OK) return s;
  if ((s = check_device(plan)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const kde_plan_info& I = plan->info;
  if (I.precision == KDE_F32 && I.engine == KDE_ENGINE_TWO_PHASE)
    return kde::fx_fft_eval(plan, reinterpret_cast<const long long*>(counts), (const float*)Kspec,
                            (float*)density, workspace, st,
                            reinterpret_cast<unsigned long long*>(counts));
  s = I.precision == KDE_F32 ? fft_eval_impl<float>(plan, counts, Kspec, density, workspace, st)
                             : fft_eval_impl<double>(plan, counts, Kspec, density, workspace, st);
  if (s != KDE_OK) return s;
  int64_t cells = 1;
  for (int k = 0; k < I.d; ++k) cells *= I.M[k];
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)cells * sizeof(int64_t), st);
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaMemsetAsync(counts)");
}

// ---------------------------------------------------------------------------
// Densities for many bandwidths on one grid (Eq. 10: C = F(c) computed once,
// K computed and applied per bandwidth).  KDE_F32 2-D plans with the
// two-phase engine; bandwidths in chunks of kMultiChunk per launch.
// ---------------------------------------------------------------------------
namespace kde {
namespace {

constexpr int kMultiChunk = 64;

struct MultiLayout {
  int Lmax0;
  size_t off_A, off_gens, off_L0, off_t1, off_K, off_S, total;
};

kde_status multi_layout(const kde_plan_s* plan, MultiLayout* m) {
  const kde_plan_info& I = plan->info;
  if (I.d != 2 || I.precision != KDE_F32 || I.engine != KDE_ENGINE_TWO_PHASE)
    return fail(KDE_ERR_UNSUPPORTED,
                "batched densities need a KDE_F32 2-D plan with the two-phase engine");
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  // every accepted bandwidth has M_0 + L_0 <= P_0
  m->Lmax0 = (int)(I.P[0] - I.M[0]);
  const size_t Q = (size_t)I.Q, M0 = (size_t)I.M[0], P0 = (size_t)I.P[0];
  m->off_A = 0;
  m->off_gens = up(M0 * Q * 8);
  m->off_L0 = m->off_gens + up(kMultiChunk * sizeof(KGen<float>));
  m->off_t1 = m->off_L0 + up(kMultiChunk * sizeof(int));
  m->off_K = m->off_t1 + up((size_t)kMultiChunk * (2 * m->Lmax0 + 1) * Q * 8);
  m->off_S = m->off_K + up((size_t)kMultiChunk * P0 * Q * 4);
  m->total = m->off_S + up((size_t)kMultiChunk * M0 * Q * 8);
  return KDE_OK;
}

}  // namespace
}  // namespace kde

extern "C" kde_status kde_fft_eval_multi_workspace_bytes(kde_plan plan, size_t* bytes) {
  if (!plan || !bytes) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  MultiLayout m;
  kde_status s = multi_layout(plan, &m);
  if (s != KDE_OK) return s;
  *bytes = m.total;
  return KDE_OK;
}

extern "C" kde_status kde_fft_eval_multi(kde_plan plan, int64_t n, int nH, const double* H,
                                         const int64_t* counts, void* density, void* workspace,
                                         size_t workspace_bytes, kde_stream_t stream) {
  if (!plan || (nH > 0 && (!H || !counts || !density)))
    return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (nH < 0 || n < 1) return fail(KDE_ERR_INVALID_ARG, "need nH >= 0 and n >= 1");
  MultiLayout m;
  kde_status s = multi_layout(plan, &m);
  if (s != KDE_OK) return s;
  if (nH == 0) return KDE_OK;
  if (!workspace || workspace_bytes < m.total)
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_fft_eval_multi_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if ((s = check_device(plan)) != KDE_OK) return s;
  const kde_plan_info& I = plan->info;
  // every bandwidth's factors and kernel-grid parameters, before any launch
  std::vector<KGen<float>> gens((size_t)nH);
  std::vector<int> L0((size_t)nH);
  double prodP = (double)I.P[0] * (double)I.P[1];
  for (int h = 0; h < nH; ++h) {
    double Ainv[9], det;
    int64_t L[KDE_MAX_D];
    if ((s = matrix_support(plan, H + 4 * h, Ainv, &det, L)) != KDE_OK) return s;
    if ((s = kgen_for<float>(I, H + 4 * h, det, L, plan->layout_mode == KDE_LAYOUT_WAND,
                             &gens[h])) != KDE_OK)
      return s;
    gens[h].C = (float)(1.0 / (6.283185307179586476925287 * std::sqrt(det)) /
                        ((double)n * 4294967296.0 * prodP));
    L0[h] = (int)L[0];
  }
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  float2* A = (float2*)(ws + m.off_A);
  if ((s = fx_count_spectra(plan, reinterpret_cast<const long long*>(counts), A, st)) != KDE_OK)
    return s;
  const size_t cells = (size_t)I.M[0] * I.M[1];
  for (int h0 = 0; h0 < nH; h0 += kMultiChunk) {
    const int nh = std::min(kMultiChunk, nH - h0);
    // the chunk's parameters: stream-ordered after the previous chunk's kernels
    if ((s = upload_async(ws + m.off_gens, gens.data() + h0, nh * sizeof(KGen<float>), st)) != KDE_OK ||
        (s = upload_async(ws + m.off_L0, L0.data() + h0, nh * sizeof(int), st)) != KDE_OK)
      return s;
    s = fx_eval_batch2(plan, A, nh, (const KGen<float>*)(ws + m.off_gens), (const int*)(ws + m.off_L0),
                       m.Lmax0, (float2*)(ws + m.off_t1), (float*)(ws + m.off_K),
                       (float2*)(ws + m.off_S), (float*)density + (size_t)h0 * cells, st);
    if (s != KDE_OK) return s;
  }
  return KDE_OK;
}

// ---------------------------------------------------------------------------
// kde_fft_eval_noalloc: kde_fft_eval with its scratch in a fixed device array
// instead of a caller-provided workspace, for callers that cannot allocate
// device memory at the point of the call (for example code running inside a
// framework that owns every allocation, or a real-time loop that must not
// enter the allocator).  Its size is fixed at build time and the array lives
// on every device that loads this library until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = KDE_NOALLOC_SCRATCH_BYTES;
static_assert(kNoAllocScratchBytes % 256 == 0, "the scratch array is a whole number of 256-byte blocks");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol's name is only a host-side handle, so the address is looked up
// once per device with that device current and cached.
kde_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(KDE_ERR_UNSUPPORTED, "device ordinal too large");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return KDE_OK;
}

}  // namespace

extern "C" size_t kde_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" kde_status kde_fft_eval_noalloc(kde_plan plan, const int64_t* counts, const void* Kspec,
                                           void* density, kde_stream_t stream) {
  if (!plan || !counts || !Kspec || !density) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (plan->info.workspace_bytes > kNoAllocScratchBytes)
    return fail(KDE_ERR_WORKSPACE,
                "kde_fft_eval_noalloc: the plan needs " + std::to_string(plan->info.workspace_bytes) +
                    " bytes of scratch, above the fixed " + std::to_string(kNoAllocScratchBytes) +
                    "; use kde_fft_eval with a workspace");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  void* scratch = nullptr;
  if ((s = noalloc_scratch(plan->device, &scratch)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32)
    return fft_eval_impl<float>(plan, counts, Kspec, density, scratch, st);
  return fft_eval_impl<double>(plan, counts, Kspec, density, scratch, st);
}

// ---------------------------------------------------------------------------
// Count spectrum and LSCV entry points.
// ---------------------------------------------------------------------------
extern "C" kde_status kde_power_spectrum(kde_plan plan, const int64_t* counts, void* W,
                                         void* workspace, size_t workspace_bytes,
                                         kde_stream_t stream) {
  if (!plan || !counts || !W) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  kde_status s = check_ws(plan, workspace, workspace_bytes);
  if (s != KDE_OK) return s;
  if ((s = check_device(plan)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32) return power_spectrum_impl<float>(plan, counts, W, workspace, st);
  return power_spectrum_impl<double>(plan, counts, W, workspace, st);
}

extern "C" kde_status kde_lscv_workspace_bytes(kde_plan plan, size_t* bytes) {
  if (!plan || !bytes) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (plan->info.d == 3) return fail(KDE_ERR_UNSUPPORTED, "LSCV batches support d = 1, 2");
  *bytes = lscv_workspace(plan->info);
  return KDE_OK;
}

extern "C" kde_status kde_lscv(kde_plan plan, int64_t n, int nH, const double* H, const void* W,
                               double* pair_sums, double* lscv, void* workspace,
                               size_t workspace_bytes, kde_stream_t stream) {
  if (!plan || !H || !W || !lscv) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (plan->info.d == 3) return fail(KDE_ERR_UNSUPPORTED, "LSCV batches support d = 1, 2");
  if (n < 2) return fail(KDE_ERR_INVALID_ARG, "LSCV needs n >= 2");
  if (nH < 0) return fail(KDE_ERR_INVALID_ARG, "nH < 0");
  if (nH == 0) return KDE_OK;
  if (!workspace || workspace_bytes < lscv_workspace(plan->info))
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_lscv_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32)
    return lscv_impl<float>(plan, n, nH, H, W, pair_sums, lscv, workspace, st);
  return lscv_impl<double>(plan, n, nH, H, W, pair_sums, lscv, workspace, st);
}

extern "C" kde_status kde_lscv_autocorr_workspace_bytes(kde_plan plan, size_t* bytes) {
  if (!plan || !bytes) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (plan->info.d != 2) return fail(KDE_ERR_UNSUPPORTED, "autocorrelation LSCV supports d = 2");
  *bytes = ac_workspace(plan->info);
  return KDE_OK;
}

extern "C" kde_status kde_autocorrelation(kde_plan plan, const int64_t* counts, void* R,
                                          void* workspace, size_t workspace_bytes,
                                          kde_stream_t stream) {
  if (!plan || !counts || !R) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (plan->info.d != 2) return fail(KDE_ERR_UNSUPPORTED, "autocorrelation LSCV supports d = 2");
  if (!workspace || workspace_bytes < ac_workspace(plan->info))
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_lscv_autocorr_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32) return autocorr_impl<float>(plan, counts, R, workspace, st);
  return autocorr_impl<double>(plan, counts, R, workspace, st);
}

// Workspace of kde_prepare2_batch: device copy of the offsets, the
// standardised samples, and the autocorrelation's two intermediates for
// every grid.
struct PrepLayout {
  size_t off_offsets, off_Z, off_A, off_B, total;
};

static PrepLayout prep_layout(const kde_plan_info& I, int64_t nsets, int64_t n_total) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t cb = I.precision == KDE_F32 ? 8 : 16;  // complex element
  PrepLayout L{};
  L.off_offsets = 0;
  L.off_Z = up((size_t)(nsets + 1) * sizeof(int64_t));
  L.off_A = L.off_Z + up((size_t)n_total * 2 * sizeof(float));
  L.off_B = L.off_A + up((size_t)nsets * I.M[0] * I.Q * cb);
  L.total = L.off_B + up((size_t)nsets * I.P[0] * I.Q * cb);
  return L;
}

static kde_status prep_check(kde_plan plan, int nsets) {
  if (!plan) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  const kde_plan_info& I = plan->info;
  if (I.d != 2) return fail(KDE_ERR_UNSUPPORTED, "batched preparation supports d = 2");
  if (I.M[0] != I.M[1] || I.M[0] < 32 || I.M[0] % 32)
    return fail(KDE_ERR_UNSUPPORTED, "batched preparation needs an M x M grid, M a multiple of 32");
  if (nsets < 0 || nsets > 65535) return fail(KDE_ERR_INVALID_ARG, "need 0 <= nsets <= 65535");
  return KDE_OK;
}

extern "C" kde_status kde_prepare2_batch_workspace_bytes(kde_plan plan, int nsets, int64_t n_total,
                                                         size_t* bytes) {
  kde_status s = prep_check(plan, nsets);
  if (s != KDE_OK) return s;
  if (!bytes || n_total < 0) return fail(KDE_ERR_INVALID_ARG, "bad argument");
  *bytes = prep_layout(plan->info, nsets, n_total).total;
  return KDE_OK;
}

extern "C" kde_status kde_prepare2_batch(kde_plan plan, int nsets, const float* X,
                                         const int64_t* offsets, int64_t* counts, double* moments,
                                         float* feat, void* R, void* workspace,
                                         size_t workspace_bytes, kde_stream_t stream) {
  kde_status s = prep_check(plan, nsets);
  if (s != KDE_OK) return s;
  if (nsets == 0) return KDE_OK;
  if (!X || !offsets || !counts || !moments || !feat || !R)
    return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (offsets[0] != 0) return fail(KDE_ERR_INVALID_ARG, "offsets[0] must be 0");
  int64_t n_max = 0;
  for (int b = 0; b < nsets; ++b) {
    const int64_t n = offsets[b + 1] - offsets[b];
    if (n < 2) return fail(KDE_ERR_INVALID_ARG, "every dataset needs at least 2 samples");
    if (n >= (int64_t(1) << 31)) return fail(KDE_ERR_INVALID_ARG, "a dataset has 2^31 samples or more");
    n_max = std::max(n_max, n);
  }
  const int64_t n_total = offsets[nsets];
  const kde_plan_info& I = plan->info;
  const PrepLayout L = prep_layout(I, nsets, n_total);
  if (!workspace || workspace_bytes < L.total)
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_prepare2_batch_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if ((s = check_device(plan)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  int64_t* off_dev = (int64_t*)(ws + L.off_offsets);
  float* Z = (float*)(ws + L.off_Z);
  if ((s = upload_async(off_dev, offsets, (size_t)(nsets + 1) * sizeof(int64_t), st)) != KDE_OK)
    return s;
  if ((s = standardize2_sets(X, off_dev, nsets, Z, moments, st)) != KDE_OK) return s;
  if ((s = bin_sets_f32(Z, off_dev, nsets, n_max, 2, plan->lo, plan->hi, I.M, counts, st)) != KDE_OK)
    return s;
  if ((s = features2_sets(counts, (int)I.M[0], nsets, off_dev, moments, feat, st)) != KDE_OK) return s;
  if (I.precision == KDE_F32)
    return autocorr_impl<float>(plan, counts, R, ws + L.off_A, st, nsets, ws + L.off_B);
  return autocorr_impl<double>(plan, counts, R, ws + L.off_A, st, nsets, ws + L.off_B);
}

static kde_status lscv_ac_entry(kde_plan plan, int nsets, const int64_t* n, int nH,
                                const double* H, const void* R, double* pair_sums, double* lscv,
                                void* workspace, size_t workspace_bytes, kde_stream_t stream) {
  if (!plan || !n || !H || !R || !lscv) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (plan->info.d != 2) return fail(KDE_ERR_UNSUPPORTED, "autocorrelation LSCV supports d = 2");
  if (nsets < 0 || nH < 0) return fail(KDE_ERR_INVALID_ARG, "nsets < 0 or nH < 0");
  for (int s = 0; s < nsets; ++s)
    if (n[s] < 2) return fail(KDE_ERR_INVALID_ARG, "LSCV needs n >= 2");
  if (nsets == 0 || nH == 0) return KDE_OK;
  if (!workspace || workspace_bytes < ac_workspace(plan->info))
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_lscv_autocorr_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32)
    return lscv_ac_impl<float>(plan, nsets, n, nH, H, R, pair_sums, lscv, workspace, st);
  return lscv_ac_impl<double>(plan, nsets, n, nH, H, R, pair_sums, lscv, workspace, st);
}

extern "C" kde_status kde_lscv_autocorr(kde_plan plan, int64_t n, int nH, const double* H,
                                        const void* R, double* pair_sums, double* lscv,
                                        void* workspace, size_t workspace_bytes,
                                        kde_stream_t stream) {
  return lscv_ac_entry(plan, 1, &n, nH, H, R, pair_sums, lscv, workspace, workspace_bytes, stream);
}

extern "C" kde_status kde_lscv_autocorr_batch(kde_plan plan, int nsets, const int64_t* n, int nH,
                                              const double* H, const void* R, double* pair_sums,
                                              double* lscv, void* workspace,
                                              size_t workspace_bytes, kde_stream_t stream) {
  return lscv_ac_entry(plan, nsets, n, nH, H, R, pair_sums, lscv, workspace, workspace_bytes, stream);
}

// A candidate set prepared once: its lag-sum parameters and work units live
// on the device, so scoring it against another dataset's autocorrelation is
// two launches per chunk of 1024 candidates with no host work.
struct kde_lscv_cands_s {
  kde_plan_s* plan;
  int nH;
  struct Chunk {
    void* dev;
    int64_t c0;
    int nh, nunits;
  };
  std::vector<Chunk> chunks;
};

static void cands_free(kde_lscv_cands_s* c) {
  for (auto& ch : c->chunks) cudaFree(ch.dev);
  delete c;
}

template <typename T>
static kde_status cands_build(kde_lscv_cands_s* c, const double* H) {
  std::vector<unsigned char> up;
  for (int64_t h0 = 0; h0 < c->nH; h0 += kAcChunk) {
    const int nh = (int)std::min<int64_t>(kAcChunk, c->nH - h0);
    int nunits = 0;
    kde_status s = ac_build_chunk<T>(c->plan, h0, nh, c->nH, H, nullptr, up, &nunits);
    if (s != KDE_OK) return s;
    kde_lscv_cands_s::Chunk ch{nullptr, h0, nh, nunits};
    cudaError_t e = cudaMalloc(&ch.dev, up.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(candidate set)");
    c->chunks.push_back(ch);
    e = cudaMemcpy(ch.dev, up.data(), up.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(candidate set)");
  }
  return KDE_OK;
}

extern "C" kde_status kde_lscv_cands_create(kde_plan plan, int nH, const double* H,
                                            kde_lscv_cands* out) {
  if (!plan || !H || !out) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (plan->info.d != 2) return fail(KDE_ERR_UNSUPPORTED, "autocorrelation LSCV supports d = 2");
  if (nH < 1) return fail(KDE_ERR_INVALID_ARG, "nH must be >= 1");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  auto* c = new kde_lscv_cands_s{plan, nH, {}};
  s = plan->info.precision == KDE_F32 ? cands_build<float>(c, H) : cands_build<double>(c, H);
  if (s != KDE_OK) {
    cands_free(c);
    return s;
  }
  *out = c;
  return KDE_OK;
}

extern "C" kde_status kde_lscv_cands_destroy(kde_lscv_cands cands) {
  if (!cands) return KDE_OK;
  cands_free(cands);
  return KDE_OK;
}

extern "C" kde_status kde_lscv_autocorr_cands(kde_lscv_cands cands, int64_t n, const void* R,
                                              double* pair_sums, double* lscv, void* workspace,
                                              size_t workspace_bytes, kde_stream_t stream) {
  if (!cands || !R || !lscv) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (n < 2) return fail(KDE_ERR_INVALID_ARG, "LSCV needs n >= 2");
  kde_plan_s* plan = cands->plan;
  if (!workspace || workspace_bytes < ac_workspace(plan->info))
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_lscv_autocorr_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  double* partial = (double*)((char*)workspace + ac_upload_bytes(plan->info));
  for (const auto& ch : cands->chunks) {
    double* S = pair_sums ? pair_sums + 2 * ch.c0 : nullptr;
    s = plan->info.precision == KDE_F32
            ? ac_launch_chunk<float>(plan->info, ch.dev, ch.nh, ch.nunits, R, partial, (double)n, S,
                                     lscv + ch.c0, st)
            : ac_launch_chunk<double>(plan->info, ch.dev, ch.nh, ch.nunits, R, partial, (double)n, S,
                                      lscv + ch.c0, st);
    if (s != KDE_OK) return s;
  }
  return KDE_OK;
}

// Scratch of kde_lscv_autocorr_cands_batch: the datasets' n, then one FP64
// partial per work unit of the largest chunk and dataset.
static size_t cands_batch_bytes(const kde_lscv_cands_s* c, int nsets) {
  int units = 0;
  for (const auto& ch : c->chunks) units = std::max(units, ch.nunits);
  const size_t nb = ((size_t)nsets * sizeof(double) + 255) & ~(size_t)255;
  return nb + (size_t)nsets * units * sizeof(double);
}

extern "C" kde_status kde_lscv_autocorr_cands_batch_workspace_bytes(kde_lscv_cands cands, int nsets,
                                                                    size_t* bytes) {
  if (!cands || !bytes) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (nsets < 0 || nsets > 65535) return fail(KDE_ERR_INVALID_ARG, "need 0 <= nsets <= 65535");
  *bytes = cands_batch_bytes(cands, nsets);
  return KDE_OK;
}

extern "C" kde_status kde_lscv_autocorr_cands_batch(kde_lscv_cands cands, int nsets,
                                                    const int64_t* n, const void* R,
                                                    double* pair_sums, double* lscv,
                                                    void* workspace, size_t workspace_bytes,
                                                    kde_stream_t stream) {
  if (!cands) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (nsets < 0 || nsets > 65535) return fail(KDE_ERR_INVALID_ARG, "need 0 <= nsets <= 65535");
  if (nsets == 0) return KDE_OK;
  if (!n || !R || !lscv) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  std::vector<double> nd((size_t)nsets);
  for (int b = 0; b < nsets; ++b) {
    if (n[b] < 2) return fail(KDE_ERR_INVALID_ARG, "LSCV needs n >= 2");
    nd[b] = (double)n[b];
  }
  if (!workspace || workspace_bytes < cands_batch_bytes(cands, nsets))
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_lscv_autocorr_cands_batch_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  kde_plan_s* plan = cands->plan;
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  const kde_plan_info& I = plan->info;
  cudaStream_t st = (cudaStream_t)stream;
  double* nset = (double*)workspace;
  double* partial = (double*)((char*)workspace + (((size_t)nsets * sizeof(double) + 255) & ~(size_t)255));
  if ((s = upload_async(nset, nd.data(), nd.size() * sizeof(double), st)) != KDE_OK) return s;
  cudaError_t e = cudaSuccess;
  const bool f32 = I.precision == KDE_F32;
  const size_t gsz = f32 ? sizeof(AcGen<float>) : sizeof(AcGen<double>);
  for (const auto& ch : cands->chunks) {
    const char* img = (const char*)ch.dev;
    const double* kn_dev = (const double*)(img + 2 * ch.nh * gsz);
    const int2* units_dev = (const int2*)((const char*)kn_dev + 2 * ch.nh * sizeof(double));
    const dim3 g1((unsigned)ch.nunits, (unsigned)nsets), g2((unsigned)((ch.nh + 7) / 8), (unsigned)nsets);
    double* S = pair_sums ? pair_sums + 2 * ch.c0 : nullptr;
    {
      LaunchScope ls("kde_lscv_ac_kernel", st);
      if (f32)
        kde_lscv_ac_kernel<float><<<g1, 256, 0, st>>>((const AcGen<float>*)img, units_dev,
                                                       (const float*)R, (int)I.P[1],
                                                       (int64_t)I.P[0] * I.P[1], partial);
      else
        kde_lscv_ac_kernel<double><<<g1, 256, 0, st>>>((const AcGen<double>*)img, units_dev,
                                                        (const double*)R, (int)I.P[1],
                                                        (int64_t)I.P[0] * I.P[1], partial);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_lscv_ac_kernel");
    }
    {
      LaunchScope ls("kde_lscv_ac_reduce_sets_kernel", st);
      if (f32)
        kde_lscv_ac_reduce_sets_kernel<float><<<g2, 256, 0, st>>>(
            (const AcGen<float>*)img, kn_dev, nset, partial, ch.nunits, ch.nh, cands->nH, S,
            lscv + ch.c0);
      else
        kde_lscv_ac_reduce_sets_kernel<double><<<g2, 256, 0, st>>>(
            (const AcGen<double>*)img, kn_dev, nset, partial, ch.nunits, ch.nh, cands->nH, S,
            lscv + ch.c0);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_lscv_ac_reduce_sets_kernel");
    }
  }
  return KDE_OK;
}

// Workspace of kde_lscv_theta_select: the uploaded n, reference thetas and
// offsets; the candidates' parameters, K_H(0) and pair sums.
struct ThetaLayout {
  size_t off_up, off_gens, off_K0, off_S, total;
};

static ThetaLayout theta_layout(int64_t nsets, int64_t J) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t cands = nsets * (J + 1);
  ThetaLayout L{};
  L.off_up = 0;
  L.off_gens = up((size_t)(nsets + 3 * nsets + 3 * J) * sizeof(double));
  L.off_K0 = L.off_gens + up((size_t)2 * cands * sizeof(AcGen<float>));
  L.off_S = L.off_K0 + up((size_t)cands * sizeof(double));
  L.total = L.off_S + up((size_t)2 * cands * sizeof(double));
  return L;
}

extern "C" kde_status kde_lscv_theta_select_workspace_bytes(kde_plan plan, int nsets, int J,
                                                            size_t* bytes) {
  if (!plan || !bytes) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (nsets < 0 || J < 1 || (int64_t)nsets * 2 * (J + 1) >= (int64_t(1) << 31))
    return fail(KDE_ERR_INVALID_ARG, "need nsets >= 0, J >= 1 and fewer than 2^31 matrices");
  *bytes = theta_layout(nsets, J).total;
  return KDE_OK;
}

extern "C" kde_status kde_lscv_theta_select(kde_plan plan, int nsets, const int64_t* n,
                                            const float* theta, const double* box, int J,
                                            const double* offsets, const double* ref, const void* R,
                                            double* lscv, double* out, void* workspace,
                                            size_t workspace_bytes, kde_stream_t stream) {
  if (!plan) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  const kde_plan_info& I = plan->info;
  if (I.d != 2 || I.precision != KDE_F32)
    return fail(KDE_ERR_UNSUPPORTED, "device-built candidates need a KDE_F32 2-D plan");
  if (nsets < 0 || J < 1 || (int64_t)nsets * 2 * (J + 1) >= (int64_t(1) << 31))
    return fail(KDE_ERR_INVALID_ARG, "need nsets >= 0, J >= 1 and fewer than 2^31 matrices");
  if (nsets == 0) return KDE_OK;
  if (!n || !theta || !box || !offsets || !ref || !R || !out)
    return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  const ThetaLayout L = theta_layout(nsets, J);
  if (!workspace || workspace_bytes < L.total)
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than kde_lscv_theta_select_workspace_bytes");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  std::vector<double> up((size_t)(nsets + 3 * nsets + 3 * J));
  for (int s = 0; s < nsets; ++s) {
    if (n[s] < 2) return fail(KDE_ERR_INVALID_ARG, "LSCV needs n >= 2");
    up[s] = (double)n[s];
  }
  for (int i = 0; i < 3 * nsets; ++i) {
    if (!std::isfinite(ref[i])) return fail(KDE_ERR_INVALID_ARG, "non-finite reference theta");
    up[nsets + i] = ref[i];
  }
  for (int i = 0; i < 3 * J; ++i) {
    if (!std::isfinite(offsets[i])) return fail(KDE_ERR_INVALID_ARG, "non-finite offset");
    up[4 * (size_t)nsets + i] = offsets[i];
  }
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(box[k])) return fail(KDE_ERR_INVALID_ARG, "non-finite box");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  double* upd = (double*)(ws + L.off_up);
  if ((s = upload_async(upd, up.data(), up.size() * sizeof(double), st)) != KDE_OK) return s;
  cudaError_t e = cudaSuccess;
  ThetaArgs t{};
  t.nsets = nsets;
  t.J = J;
  t.theta = theta;
  t.n = upd;
  t.ref = upd + nsets;
  t.off = upd + 4 * (size_t)nsets;
  for (int k = 0; k < 3; ++k) {
    t.box_lo[k] = box[k];
    t.box_hi[k] = box[3 + k];
  }
  t.tau = plan->tau;
  for (int k = 0; k < 2; ++k) {
    t.delta[k] = I.delta[k];
    t.M[k] = (int)I.M[k];
    t.P[k] = (int)I.P[k];
  }
  t.wand = plan->layout_mode == KDE_LAYOUT_WAND;
  t.per_axis = plan->range_mode != KDE_RANGE_CORRECTED;
  t.gens = (AcGen<float>*)(ws + L.off_gens);
  t.K0 = (double*)(ws + L.off_K0);
  double* S = (double*)(ws + L.off_S);
  const int64_t nmat = (int64_t)nsets * 2 * (J + 1);
  {
    LaunchScope ls("kde_theta_gen_kernel", st);
    kde_theta_gen_kernel<<<(unsigned)((nmat + 127) / 128), 128, 0, st>>>(t);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_theta_gen_kernel");
  }
  {
    LaunchScope ls("kde_lscv_theta_sums_kernel", st);
    kde_lscv_theta_sums_kernel<<<(unsigned)nmat, 256, 0, st>>>(t.gens, (const float*)R, (int)I.P[1],
                                                               (int64_t)I.P[0] * I.P[1], S);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_lscv_theta_sums_kernel");
  }
  {
    LaunchScope ls("kde_lscv_theta_pick_kernel", st);
    kde_lscv_theta_pick_kernel<<<nsets, 32, 0, st>>>(t, S, lscv, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_lscv_theta_pick_kernel");
  }
  return KDE_OK;
}

// ---------------------------------------------------------------------------
// Ragged batches: many independent 2-D problems (own samples, grid, H) in one
// set of launches.  Every pass is a persistent grid-stride kernel over the
// work items of all problems (a block maps its work index to a problem by
// binary search over per-pass prefix sums), so the batch costs seven launches
// whatever its size; problems of different sizes share each launch.
// ---------------------------------------------------------------------------
namespace kde {
namespace {

// Linear binning arithmetic for the batch kernel (the rounding rules of
// kde_bin: t = (x - lo) s rounded in the samples' type, i = floor(t),
// f = t - i, the last node folded to (M-2, 1), q = round-half-even(f 2^32)
// with q = 2^32 written as (i+1, 0); part w of the unit mass gives
// floor((w q + 2^31) / 2^32) to node i+1, axis 0 first).
template <typename T>
struct BinAxisLite {
  T lo, s, top;
  int M;
};

__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ bool lite_fixed(float f, int& i, unsigned& q) {
  if (f == 1.0f) {
    i += 1;
    q = 0;
  } else {
    q = __float2uint_rn(f * 4294967296.0f);  // f 2^32 < 2^32 exactly
  }
  return true;
}
__device__ __forceinline__ bool lite_fixed(double f, int& i, unsigned& q) {
  const unsigned long long Q = __double2ull_rn(f * 4294967296.0);
  if (Q == (1ull << 32)) {
    i += 1;
    q = 0;
  } else {
    q = (unsigned)Q;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ bool lite_position(T x, const BinAxisLite<T>& a, int& i, unsigned& q) {
  const T t = rn_mul(rn_sub(x, a.lo), a.s);
  if (!(t >= T(0) && t <= a.top)) return false;
  const T fl = floor(t);
  i = (int)fl;
  T f = rn_sub(t, fl);
  if (i == a.M - 1) {
    i = a.M - 2;
    f = T(1);
  }
  return lite_fixed(f, i, q);
}

__device__ __forceinline__ unsigned lite_mulhi(unsigned long long w, unsigned q) {
  const unsigned wl = (unsigned)w, wh = (unsigned)(w >> 32);
  return wh * q + __umulhi(wl, q) + ((wl * q) >> 31);
}

// corners (0,0), (0,1), (1,0), (1,1) (axis-0 offset first)
__device__ __forceinline__ void lite_corner_weights2(const unsigned* q, unsigned long long* w) {
  const unsigned long long one = 1ull << 32;
  const unsigned long long a1 = lite_mulhi(one, q[0]), a0 = one - a1;
  w[1] = lite_mulhi(a0, q[1]);
  w[0] = a0 - w[1];
  w[3] = lite_mulhi(a1, q[1]);
  w[2] = a1 - w[3];
}

enum BatchPass { BP_BIN = 0, BP_KROWS, BP_KCOLS, BP_ROWS, BP_MID, BP_C2R, BP_COUNT };

template <typename T>
struct BatchItem {
  using V = typename Cplx<T>::type;
  int64_t x_off, n;          // samples [x_off, x_off + n) of the concatenated X
  T lo[2], s[2], top[2];     // binning: lo, (M-1)/(hi-lo), M-1 in the samples' type
  int M[2], P[2], Q, L[2];
  int64_t counts_off;        // int64 elements
  int64_t kspec_off;         // real elements, [Q][P0] (column-major spectrum)
  int64_t A_off;             // complex elements, [M0][Q]
  int64_t T1_off;            // complex elements, [2 L0 + 1][Q]
  int64_t dens_off;          // real elements, [M0][M1]
  LinePlan lp[2];
  const V* tw[2];
  KGen<T> gen;
};

__device__ __forceinline__ int find_item(const int* __restrict__ start, int count, int w) {
  int lo = 0, hi = count - 1;  // largest i with start[i] <= w
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T>
struct BatchArgs {
  const BatchItem<T>* items;
  const int* wstart;   // [BP_COUNT][count + 1] work prefix per pass
  int count;
  int tpl_rows, tpl_cols;
  const T* X;
  long long* counts;
  T* kspec;
  typename Cplx<T>::type* A;
  typename Cplx<T>::type* T1;
  T* density;
};

// Binning of every problem's samples: the same arithmetic as the direct
// method.  Work item = (problem, chunk of kBinChunk samples); a block takes
// whole work items, so each knows its problem without a per-sample search.
constexpr int kBinChunk = 8192;

// Chunk vb of problem it's samples (all threads of the block).
template <typename T>
__device__ __forceinline__ void batch_bin_item(const BatchArgs<T>& a, int it, int64_t vb) {
  {
    const BatchItem<T>& B = a.items[it];
    const int64_t c0 = vb * kBinChunk;
    const int64_t c1 = min(B.n, c0 + kBinChunk);
    // two adjacent lanes per sample: lane parity p adds the corners at
    // offset p along the last axis, so a lane pair's two words share a
    // 32-byte sector three times in four and coalesce into one request
    const int par = threadIdx.x & 1;
    const int64_t jstep = blockDim.x >> 1;
    constexpr int U = 8;  // samples whose coordinates are loaded before any is added
    unsigned long long* c = reinterpret_cast<unsigned long long*>(a.counts + B.counts_off);
    for (int64_t j0 = c0 + (threadIdx.x >> 1); j0 < c1; j0 += U * jstep) {
      T xs[U][2];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = j0 + u * jstep;
        xs[u][0] = j < c1 ? a.X[(B.x_off + j) * 2] : T(0);
        xs[u][1] = j < c1 ? a.X[(B.x_off + j) * 2 + 1] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j0 + u * jstep >= c1) break;
        int i[2];
        unsigned q[2];
        bool in = true;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          BinAxisLite<T> ax{B.lo[k], B.s[k], B.top[k], B.M[k]};
          in &= lite_position<T>(xs[u][k], ax, i[k], q[k]);
        }
        if (!in) continue;
        unsigned long long wt[4];
        lite_corner_weights2(q, wt);
        const unsigned long long w0 = par ? wt[1] : wt[0], w1 = par ? wt[3] : wt[2];
        const int64_t base = (int64_t)i[0] * B.M[1] + i[1] + par;
        if (w0) atomicAdd(c + base, w0);
        if (w1) atomicAdd(c + base + B.M[1], w1);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) kde_batch_bin_kernel(BatchArgs<T> a) {
  const int* wst = a.wstart + BP_BIN * (a.count + 1);
  const int total = wst[a.count];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int it = find_item(wst, a.count, w);
    batch_bin_item<T>(a, it, w - wst[it]);
  }
}

// Per-block parameters of a pass over one problem (set by one thread).
template <typename T>
struct PassShared {
  RowsParams<T> rp;
  C2RParams<T> cr;
  ColsParams<T> cp;
  KGen<T> gen;
};

template <typename T>
__device__ __forceinline__ void batch_pass_params(const BatchArgs<T>& a, int PASS, int it,
                                                  PassShared<T>& sh) {
  {
    {
      const BatchItem<T>& B = a.items[it];
      RowsParams<T>& rp = sh.rp;
      C2RParams<T>& cr = sh.cr;
      ColsParams<T>& cp = sh.cp;
      KGen<T>& gen = sh.gen;
      if (PASS == BP_KROWS || PASS == BP_ROWS) {
        RowsParams<T> r{};
        r.Q = B.Q;
        r.lp = B.lp[1];
        r.tw = B.tw[1];
        r.tpl = a.tpl_rows;
        if (PASS == BP_KROWS) {
          r.nrows = 2 * B.L[0] + 1;
          r.out = a.T1 + B.T1_off;
          gen = B.gen;
        } else {
          r.nrows = B.M[0];
          r.Min = B.M[1];
          r.in_stride = B.M[1];
          r.out = a.A + B.A_off;
        }
        rp = r;
      } else if (PASS == BP_C2R) {
        C2RParams<T> c{};
        c.in = a.A + B.A_off;
        c.out = a.density + B.dens_off;
        c.nrows = B.M[0];
        c.Mout = B.M[1];
        c.Q = B.Q;
        c.tpl = a.tpl_rows;
        c.lp = B.lp[1];
        c.tw = B.tw[1];
        cr = c;
      } else {
        ColsParams<T> c{};
        c.S = B.Q;
        c.lp = B.lp[0];
        c.tw = B.tw[0];
        c.tpl = a.tpl_cols;
        if (PASS == BP_KCOLS) {
          c.in = a.T1 + B.T1_off;
          c.out_real = a.kspec + B.kspec_off;
          c.Nin = 2 * B.L[0] + 1;
          c.Lw = B.L[0];
        } else {
          c.in = a.A + B.A_off;
          c.out = a.A + B.A_off;
          c.K = a.kspec + B.kspec_off;
          c.Nin = B.M[0];
          c.Nout = B.M[0];
          c.Lw = -1;
        }
        cp = c;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void batch_pass_body(const BatchArgs<T>& a, int PASS, int it, int64_t vb,
                                                const PassShared<T>& sh) {
  if (PASS == BP_KROWS) rows_kgen_body<T>(sh.gen, sh.rp, vb);
  if (PASS == BP_ROWS) rows_counts_body<T>(a.counts + a.items[it].counts_off, sh.rp, vb);
  if (PASS == BP_C2R) rows_c2r_body<T>(sh.cr, vb);
  if (PASS == BP_KCOLS) cols_body_slab<T, COL_FWD_REAL>(sh.cp, 0, vb);
  if (PASS == BP_MID) cols_body_slab<T, COL_MID>(sh.cp, 0, vb);
}

template <typename T, int PASS>
__global__ void __launch_bounds__(256) kde_batch_pass_kernel(BatchArgs<T> a) {
  __shared__ PassShared<T> sh;
  __shared__ int item, base;
  const int* wst = a.wstart + PASS * (a.count + 1);
  const int total = wst[a.count];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    if (threadIdx.x == 0) {
      const int it = find_item(wst, a.count, w);
      item = it;
      base = wst[it];
      batch_pass_params<T>(a, PASS, it, sh);
    }
    __syncthreads();
    batch_pass_body<T>(a, PASS, item, w - base, sh);
    __syncthreads();  // the next item reloads twiddles and parameters
  }
}

// ---------------------------------------------------------------------------
// The whole ragged batch as one persistent launch.  Work items of every
// problem and stage (zero the counts, kernel rows, binning, kernel spectrum,
// count rows, middle axis, output rows) form one queue, in stage order or
// problem by problem (largest first); blocks claim items with an atomic
// counter.  An item waits for the stages of its own problem it reads from
// (per-problem completion counters); in either order those precede it in
// the queue, so a claimed item only waits on items already claimed by
// running blocks: the queue always progresses.  Every
// wait is bounded: after wait_polls polls the block records the timeout in
// the status word, raises the abort flag (waiters of this launch then give
// up at once) and leaves.  The last block out resets the queue for the next
// launch.  Completion: every thread fences its writes, the block barrier,
// then one thread adds to the counter; a waiter fences after it sees the
// count, and the stages read produced data through L2 (__ldcg).
// ---------------------------------------------------------------------------
enum PersistStage { PS_ZERO = 0, PS_KROWS, PS_BIN, PS_KCOLS, PS_ROWS, PS_MID, PS_C2R, PS_COUNT };
constexpr int kZeroChunk = 1 << 16;        // int64 counts zeroed per item
constexpr unsigned kCtlWords = 4;          // next, exited, abort, status; then done[count][PS_COUNT]
constexpr unsigned kDefaultWaitPolls = 1u << 22;   // about a second of polls

template <typename T>
struct PersistArgs {
  BatchArgs<T> a;
  const int* pstart;                // [PS_COUNT][count + 1] items per problem, prefix
  const int4* queue;                // per queue position: problem, stage, item within it
  int total;                        // queue length
  unsigned* ctl;
  unsigned wait_polls;
  int withhold;                     // stage whose completions are never signalled (-1: none)
};

__device__ __forceinline__ int stage_pass(int st) {
  switch (st) {
    case PS_KROWS: return BP_KROWS;
    case PS_KCOLS: return BP_KCOLS;
    case PS_ROWS: return BP_ROWS;
    case PS_MID: return BP_MID;
    case PS_C2R: return BP_C2R;
    default: return -1;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) kde_batch_persistent_kernel(PersistArgs<T> pa) {
  __shared__ PassShared<T> sh;
  __shared__ unsigned s_item;
  __shared__ int s_ok;
  const BatchArgs<T>& a = pa.a;
  unsigned* ctl = pa.ctl;
  unsigned* done = ctl + kCtlWords;
  const unsigned total = (unsigned)pa.total;
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctl[0], 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= total) break;
    const int4 q = pa.queue[item];
    const int it = q.x, st = q.y;
    const int64_t vb = q.z;
    if (threadIdx.x == 0) {
      int dep[2] = {-1, -1};
      if (st == PS_BIN) dep[0] = PS_ZERO;
      if (st == PS_KCOLS) dep[0] = PS_KROWS;
      if (st == PS_ROWS) dep[0] = PS_BIN;
      if (st == PS_MID) {
        dep[0] = PS_ROWS;
        dep[1] = PS_KCOLS;
      }
      if (st == PS_C2R) dep[0] = PS_MID;
      bool ok = true;
      for (int k = 0; k < 2 && ok; ++k) {
        if (dep[k] < 0) continue;
        const int* pd = pa.pstart + dep[k] * (a.count + 1);
        const unsigned need = (unsigned)(pd[it + 1] - pd[it]);
        volatile unsigned* cnt = done + (size_t)it * PS_COUNT + dep[k];
        volatile unsigned* abort_flag = ctl + 2;
        unsigned polls = 0;
        while (*cnt < need) {
          if (*abort_flag || ++polls > pa.wait_polls) {
            ok = false;
            break;
          }
          __nanosleep(256);
        }
      }
      if (!ok) {
        atomicExch(&ctl[3], 1u);   // status: a wait gave up (kept until checked)
        atomicExch(&ctl[2], 1u);   // abort this launch
      }
      __threadfence();
      s_ok = ok;
      if (ok && stage_pass(st) >= 0) batch_pass_params<T>(a, stage_pass(st), it, sh);
    }
    __syncthreads();
    if (!s_ok) break;
    if (st == PS_ZERO) {
      const BatchItem<T>& B = a.items[it];
      const int64_t cells = (int64_t)B.M[0] * B.M[1];
      long long* c = a.counts + B.counts_off;
      for (int64_t i = vb * kZeroChunk + threadIdx.x; i < min(cells, (vb + 1) * kZeroChunk);
           i += blockDim.x)
        c[i] = 0;
    } else if (st == PS_BIN) {
      batch_bin_item<T>(a, it, vb);
    } else {
      batch_pass_body<T>(a, stage_pass(st), it, vb, sh);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && st != pa.withhold) atomicAdd(done + (size_t)it * PS_COUNT + st, 1u);
  }
  // the last block out resets the queue and the counters for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl[1], 1u) == gridDim.x - 1) {
      for (int i = 0; i < a.count * PS_COUNT; ++i) done[i] = 0;
      ctl[0] = 0;
      ctl[2] = 0;
      __threadfence();
      ctl[1] = 0;
    }
  }
}

}  // namespace
}  // namespace kde

struct kde_batch_plan_s {
  int count;
  int precision;
  std::vector<kde_plan_s*> plans;   // per problem: info and twiddles
  void* items_dev;                  // BatchItem<T>[count]
  int* wstart_dev;                  // [BP_COUNT][count + 1]
  std::vector<int> wstart;          // host copy
  int64_t x_total, counts_elems, kspec_elems, A_elems, T1_elems, dens_elems;
  int Pmax;
  int tpl_rows, tpl_cols;           // launch shape (tunable)
  int mode;                         // KDE_BATCH_PERSISTENT or KDE_BATCH_STAGED (tunable)
  int* pstart_dev;                  // [PS_COUNT][count + 1] items per problem (persistent queue)
  std::vector<int> pstart;
  int4* queue_dev;                  // the persistent queue (problem, stage, item)
  int queue_len, queue_cap;
  int queue_order;                  // KDE_BATCH_QUEUE_STAGES or KDE_BATCH_QUEUE_PROBLEMS
  unsigned* ctl_dev;                // queue control words and completion counters
  unsigned wait_polls;
  int withhold;
  size_t workspace_bytes;
  std::vector<int64_t> n;           // samples per problem
  std::vector<kde_batch_item> items;  // the problems, for re-planning by the tuner
  kde_opts opts;
  int pad_policy;                   // KDE_BATCH_PAD_SMALLEST or KDE_BATCH_PAD_FEWEST_STAGES
  int radix_order;                  // 0: largest radix first, 1: smallest first
  // the kernel-grid passes need no samples: they run on this stream beside
  // the binning (fork and join events on the caller's stream)
  cudaStream_t side;
  cudaEvent_t fork, join;
};

namespace kde {
namespace {

constexpr int kBatchLines = 2;  // lines per block in the batch passes

template <typename T>
kde_status batch_upload(kde_batch_plan_s* bp, const kde_batch_item* items) {
  using V = typename Cplx<T>::type;
  std::vector<BatchItem<T>> h(bp->count);
  int64_t x = 0, cnt = 0, ks = 0, A = 0, T1 = 0, de = 0;
  for (int i = 0; i < bp->count; ++i) {
    const kde_plan_s* pl = bp->plans[i];
    const kde_plan_info& I = pl->info;
    BatchItem<T>& B = h[i];
    B.x_off = x;
    B.n = items[i].n;
    for (int k = 0; k < 2; ++k) {
      const double sk = (double)(I.M[k] - 1) / (pl->hi[k] - pl->lo[k]);
      B.lo[k] = (T)pl->lo[k];
      B.s[k] = (T)sk;
      B.top[k] = (T)(I.M[k] - 1);
      B.M[k] = (int)I.M[k];
      B.P[k] = (int)I.P[k];
      B.L[k] = (int)I.L[k];
      B.lp[k] = line_plan(I, k);
      B.tw[k] = twiddles<T>(pl, k);
    }
    B.Q = (int)I.Q;
    B.counts_off = cnt;
    B.kspec_off = ks;
    B.A_off = A;
    B.T1_off = T1;
    B.dens_off = de;
    kde_status sg = kgen_for<T>(I, pl->H, I.det_H, I.L, pl->layout_mode == KDE_LAYOUT_WAND, &B.gen);
    if (sg != KDE_OK) return sg;
    B.gen.C = (T)(std::pow(6.283185307179586476925287, -1.0) / std::sqrt(I.det_H) /
                  ((double)items[i].n * 4294967296.0 * (double)I.P[0] * (double)I.P[1]));
    x += items[i].n;
    cnt += I.M[0] * I.M[1];
    ks += I.P[0] * I.Q;
    A += I.M[0] * I.Q;
    T1 += (2 * I.L[0] + 1) * I.Q;
    de += I.M[0] * I.M[1];
  }
  bp->x_total = x;
  bp->counts_elems = cnt;
  bp->kspec_elems = ks;
  bp->A_elems = A;
  bp->T1_elems = T1;
  bp->dens_elems = de;
  cudaError_t e = cudaMalloc(&bp->items_dev, sizeof(BatchItem<T>) * bp->count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch items)");
  e = cudaMemcpy(bp->items_dev, h.data(), sizeof(BatchItem<T>) * bp->count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(batch items)");
  const size_t cb = sizeof(V), rb = sizeof(T);
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  bp->workspace_bytes = up(cnt * 8) + up(ks * rb) + up(A * cb) + up(T1 * cb);
  return KDE_OK;
}

int64_t items_n(const kde_batch_plan_s* bp, int i) { return bp->n[i]; }

// Work items per problem and pass for the current launch shape; uploaded.
kde_status batch_work(kde_batch_plan_s* bp) {
  const int c = bp->count;
  bp->wstart.assign((size_t)BP_COUNT * (c + 1), 0);
  const int lr = kBatchLines, lc = kBatchLines;
  for (int i = 0; i < c; ++i) {
    const kde_plan_info& I = bp->plans[i]->info;
    int w[BP_COUNT];
    w[BP_BIN] = (int)((bp->plans[i] ? items_n(bp, i) : 0) + kBinChunk - 1) / kBinChunk;
    w[BP_KROWS] = (int)((((2 * I.L[0] + 1) + 1) / 2 + lr - 1) / lr);
    w[BP_KCOLS] = (int)((I.Q + 2 * lc - 1) / (2 * lc));
    w[BP_ROWS] = (int)(((I.M[0] + 1) / 2 + lr - 1) / lr);
    w[BP_MID] = (int)((I.Q + lc - 1) / lc);
    w[BP_C2R] = w[BP_ROWS];
    for (int pss = 0; pss < BP_COUNT; ++pss)
      bp->wstart[(size_t)pss * (c + 1) + i + 1] = bp->wstart[(size_t)pss * (c + 1) + i] + w[pss];
  }
  // the persistent queue's stages: zeroing of the counts, then the passes
  bp->pstart.assign((size_t)PS_COUNT * (c + 1), 0);
  for (int i = 0; i < c; ++i) {
    const kde_plan_info& I = bp->plans[i]->info;
    int w[PS_COUNT];
    const int* ws = bp->wstart.data();
    auto per = [&](int pss) { return ws[(size_t)pss * (c + 1) + i + 1] - ws[(size_t)pss * (c + 1) + i]; };
    w[PS_ZERO] = (int)((I.M[0] * I.M[1] + kZeroChunk - 1) / kZeroChunk);
    w[PS_KROWS] = per(BP_KROWS);
    w[PS_BIN] = per(BP_BIN);
    w[PS_KCOLS] = per(BP_KCOLS);
    w[PS_ROWS] = per(BP_ROWS);
    w[PS_MID] = per(BP_MID);
    w[PS_C2R] = per(BP_C2R);
    for (int st = 0; st < PS_COUNT; ++st)
      bp->pstart[(size_t)st * (c + 1) + i + 1] = bp->pstart[(size_t)st * (c + 1) + i] + w[st];
  }
  // the queue: stage by stage, or problem by problem with the most work first
  std::vector<int4> q;
  auto items_of = [&](int i, int st) {
    return bp->pstart[(size_t)st * (c + 1) + i + 1] - bp->pstart[(size_t)st * (c + 1) + i];
  };
  if (bp->queue_order == KDE_BATCH_QUEUE_PROBLEMS) {
    std::vector<int> order(c);
    for (int i = 0; i < c; ++i) order[i] = i;
    std::vector<int64_t> work(c, 0);
    for (int i = 0; i < c; ++i) {
      const kde_plan_info& I = bp->plans[i]->info;
      work[i] = bp->n[i] + (int64_t)I.P[0] * I.P[1];
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    for (int i : order)
      for (int st = 0; st < PS_COUNT; ++st)
        for (int v = 0; v < items_of(i, st); ++v) q.push_back(make_int4(i, st, v, 0));
  } else {
    for (int st = 0; st < PS_COUNT; ++st)
      for (int i = 0; i < c; ++i)
        for (int v = 0; v < items_of(i, st); ++v) q.push_back(make_int4(i, st, v, 0));
  }
  cudaError_t e = cudaSuccess;
  if ((int)q.size() > bp->queue_cap) {
    if (bp->queue_dev) cudaFree(bp->queue_dev);
    bp->queue_dev = nullptr;
    bp->queue_cap = 0;
    e = cudaMalloc((void**)&bp->queue_dev, sizeof(int4) * q.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch queue)");
    bp->queue_cap = (int)q.size();
  }
  bp->queue_len = (int)q.size();
  e = cudaMemcpy(bp->wstart_dev, bp->wstart.data(), sizeof(int) * bp->wstart.size(),
                 cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(bp->pstart_dev, bp->pstart.data(), sizeof(int) * bp->pstart.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(bp->queue_dev, q.data(), sizeof(int4) * q.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaMemcpy(batch work)");
}

template <typename T>
kde_status batch_persistent(kde_batch_plan_s* bp, const BatchArgs<T>& a0, cudaStream_t st) {
  PersistArgs<T> pa{};
  pa.a = a0;
  pa.a.tpl_cols = pa.a.tpl_rows;   // one block shape for every stage
  pa.pstart = bp->pstart_dev;
  pa.queue = bp->queue_dev;
  pa.total = bp->queue_len;
  pa.ctl = bp->ctl_dev;
  pa.wait_polls = bp->wait_polls;
  pa.withhold = bp->withhold;
  auto* fn = kde_batch_persistent_kernel<T>;
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  const size_t smem = line_smem<T>(bp->Pmax, kBatchLines);
  const int threads = bp->tpl_rows * kBatchLines;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const int grid = std::max(1, std::min(pa.total, std::max(1, per_sm) * num_sms()));
  LaunchScope ls("kde_batch_persistent_kernel", st);
  fn<<<grid, threads, smem, st>>>(pa);
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_batch_persistent_kernel");
}

template <typename T>
kde_status batch_eval_impl(kde_batch_plan_s* bp, const void* X, void* density, void* ws,
                           cudaStream_t st) {
  using V = typename Cplx<T>::type;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char* w = (char*)ws;
  BatchArgs<T> a{};
  a.items = (const BatchItem<T>*)bp->items_dev;
  a.wstart = bp->wstart_dev;
  a.count = bp->count;
  a.tpl_rows = bp->tpl_rows;
  a.tpl_cols = bp->tpl_cols;
  a.X = (const T*)X;
  a.counts = (long long*)w;
  w += up(bp->counts_elems * 8);
  a.kspec = (T*)w;
  w += up(bp->kspec_elems * sizeof(T));
  a.A = (V*)w;
  w += up(bp->A_elems * sizeof(V));
  a.T1 = (V*)w;
  a.density = (T*)density;
  if (bp->mode == KDE_BATCH_PERSISTENT) return batch_persistent<T>(bp, a, st);
  // the kernel-grid passes (no samples needed) fork onto the plan's side
  // stream and join before the count rows
  cudaError_t e = cudaEventRecord(bp->fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bp->side, bp->fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "fork (batch kernel grid)");
  e = cudaMemsetAsync(a.counts, 0, bp->counts_elems * 8, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(batch counts)");
  const int sms = num_sms();
  const int c = bp->count;
  {
    const int total = bp->wstart[(size_t)BP_BIN * (c + 1) + c];
    LaunchScope ls("kde_batch_bin_kernel", st);
    if (total > 0) kde_batch_bin_kernel<T><<<std::min(total, sms * 8), 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kde_batch_bin_kernel");
  }
  auto run = [&](auto fn, int pass, int tpl, const char* name, cudaStream_t ss) -> kde_status {
    const int total = bp->wstart[(size_t)pass * (c + 1) + c];
    if (total == 0) return KDE_OK;
    cudaError_t e2 = allow_smem(fn);
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFuncSetAttribute");
    const size_t smem = line_smem<T>(bp->Pmax, kBatchLines);
    const int grid = std::min(total, sms * 8);
    LaunchScope ls(name, ss);
    fn<<<grid, tpl * kBatchLines, smem, ss>>>(a);
    e2 = cudaGetLastError();
    return e2 == cudaSuccess ? KDE_OK : cuda_fail(e2, name);
  };
  kde_status s;
  if ((s = run(kde_batch_pass_kernel<T, BP_KROWS>, BP_KROWS, bp->tpl_rows, "kde_batch_krows_kernel", bp->side)) != KDE_OK) return s;
  if ((s = run(kde_batch_pass_kernel<T, BP_KCOLS>, BP_KCOLS, bp->tpl_cols, "kde_batch_kcols_kernel", bp->side)) != KDE_OK) return s;
  e = cudaEventRecord(bp->join, bp->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, bp->join, 0);
  if (e != cudaSuccess) return cuda_fail(e, "join (batch kernel grid)");
  if ((s = run(kde_batch_pass_kernel<T, BP_ROWS>, BP_ROWS, bp->tpl_rows, "kde_batch_rows_kernel", st)) != KDE_OK) return s;
  if ((s = run(kde_batch_pass_kernel<T, BP_MID>, BP_MID, bp->tpl_cols, "kde_batch_mid_kernel", st)) != KDE_OK) return s;
  return run(kde_batch_pass_kernel<T, BP_C2R>, BP_C2R, bp->tpl_rows, "kde_batch_c2r_kernel", st);
}

}  // namespace
}  // namespace kde

namespace kde {
namespace {

// Padded length of one problem's axis under a batch padding policy: the
// smallest 7-smooth size >= need, or the one with the fewest radix stages
// up to 25% longer (ties: the shorter).
int64_t batch_pad(int64_t need, int policy) {
  auto smooth = [](int64_t x) {
    for (int q : {2, 3, 5, 7})
      while (x % q == 0) x /= q;
    return x == 1;
  };
  int64_t P = need;
  while (!smooth(P)) ++P;
  if (policy != KDE_BATCH_PAD_FEWEST_STAGES) return P;
  auto stages = [](int64_t x) {
    int n = 0;
    for (int r : {8, 7, 5, 4, 3, 2})
      while (x % r == 0) {
        x /= r;
        ++n;
      }
    return n;
  };
  int64_t best = P;
  for (int64_t q = P; q <= need + need / 4; ++q)
    if (smooth(q) && stages(q) < stages(best)) best = q;
  return best;
}

// (Re)creates every problem's plan under the batch's padding policy and
// radix order (the Stockham passes run the batch; the radix plan of an axis
// is applied in the chosen order).
kde_status batch_plans(kde_batch_plan_s* bp) {
  for (auto* p : bp->plans) kde_plan_destroy(p);
  bp->plans.clear();
  bp->Pmax = 0;
  for (size_t i = 0; i < bp->items.size(); ++i) {
    const kde_batch_item& it = bp->items[i];
    kde_opts o = bp->opts;
    o.engine = KDE_ENGINE_STOCKHAM;
    kde_plan_info info{};
    kde_status s = kde_plan_info_compute(2, it.M, it.lo, it.hi, it.H, &o, &info);
    if (s != KDE_OK) return s;
    for (int k = 0; k < 2; ++k)
      o.P_min[k] = std::max(o.P_min[k], batch_pad(it.M[k] + info.L[k], bp->pad_policy));
    kde_plan p = nullptr;
    if ((s = kde_plan_create(2, it.M, it.lo, it.hi, it.H, &o, &p)) != KDE_OK) return s;
    if (bp->radix_order == 1)
      for (int k = 0; k < 2; ++k) std::reverse(p->info.radix[k], p->info.radix[k] + p->info.nstages[k]);
    bp->plans.push_back(p);
    for (int k = 0; k < 2; ++k) bp->Pmax = std::max(bp->Pmax, (int)p->info.P[k]);
  }
  return KDE_OK;
}

// Re-plans, re-uploads the problem table and the work counts.
kde_status batch_rebuild(kde_batch_plan_s* bp) {
  kde_status s = batch_plans(bp);
  if (s != KDE_OK) return s;
  if (bp->items_dev) {
    cudaFree(bp->items_dev);
    bp->items_dev = nullptr;
  }
  s = (bp->precision == KDE_F32) ? batch_upload<float>(bp, bp->items.data())
                                 : batch_upload<double>(bp, bp->items.data());
  return s == KDE_OK ? batch_work(bp) : s;
}

}  // namespace
}  // namespace kde

extern "C" kde_status kde_batch_plan_create(int count, const kde_batch_item* items,
                                            const kde_opts* opts, kde_batch_plan* out) {
  if (!out || !items || count < 1) return fail(KDE_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  kde_batch_plan_s* bp = new (std::nothrow) kde_batch_plan_s();
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "out of host memory");
  bp->count = count;
  bp->precision = opts ? opts->precision : KDE_F32;
  bp->Pmax = 0;
  bp->tpl_rows = 64;
  bp->tpl_cols = 64;
  bp->mode = KDE_BATCH_PERSISTENT;
  bp->wait_polls = kDefaultWaitPolls;
  bp->withhold = -1;
  bp->pstart_dev = nullptr;
  bp->ctl_dev = nullptr;
  bp->queue_dev = nullptr;
  bp->queue_len = bp->queue_cap = 0;
  bp->queue_order = KDE_BATCH_QUEUE_PROBLEMS;
  bp->items_dev = nullptr;
  bp->wstart_dev = nullptr;
  bp->side = nullptr;
  bp->fork = bp->join = nullptr;
  kde_opts o{};
  o.tau = 3.7;
  if (opts) o = *opts;
  o.cols_variant = KDE_COLS_LINES;
  auto cleanup = [&](kde_status s) {
    for (auto* p : bp->plans) kde_plan_destroy(p);
    if (bp->items_dev) cudaFree(bp->items_dev);
    if (bp->wstart_dev) cudaFree(bp->wstart_dev);
    if (bp->pstart_dev) cudaFree(bp->pstart_dev);
    if (bp->ctl_dev) cudaFree(bp->ctl_dev);
    if (bp->queue_dev) cudaFree(bp->queue_dev);
    if (bp->side) cudaStreamDestroy(bp->side);
    if (bp->fork) cudaEventDestroy(bp->fork);
    if (bp->join) cudaEventDestroy(bp->join);
    delete bp;
    return s;
  };
  for (int i = 0; i < count; ++i) {
    if (items[i].n < 1 || items[i].n >= (int64_t(1) << 31))
      return cleanup(fail(KDE_ERR_INVALID_ARG, "every problem needs 1 <= n < 2^31"));
    bp->n.push_back(items[i].n);
    bp->items.push_back(items[i]);
  }
  bp->opts = o;
  bp->pad_policy = KDE_BATCH_PAD_SMALLEST;
  bp->radix_order = 0;
  kde_status s0 = batch_plans(bp);
  if (s0 != KDE_OK) return cleanup(s0);
  const size_t cb = (bp->precision == KDE_F32) ? 8 : 16;
  if (line_smem<float>(bp->Pmax, kBatchLines) / 8 * cb > kSmemMax)
    return cleanup(fail(KDE_ERR_UNSUPPORTED, "padded size too large for the batch passes"));
  cudaError_t e = cudaMalloc((void**)&bp->wstart_dev, sizeof(int) * BP_COUNT * (count + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&bp->pstart_dev, sizeof(int) * PS_COUNT * (count + 1));
  const size_t ctl_bytes = sizeof(unsigned) * (kCtlWords + (size_t)PS_COUNT * count);
  if (e == cudaSuccess) e = cudaMalloc((void**)&bp->ctl_dev, ctl_bytes);
  if (e == cudaSuccess) e = cudaMemset(bp->ctl_dev, 0, ctl_bytes);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc(batch work)"));
  kde_status s = (bp->precision == KDE_F32) ? batch_upload<float>(bp, items) : batch_upload<double>(bp, items);
  if (s == KDE_OK) s = batch_work(bp);
  if (s != KDE_OK) return cleanup(s);
  int lo_prio = 0, hi_prio = 0;
  cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
  e = cudaStreamCreateWithPriority(&bp->side, cudaStreamNonBlocking, hi_prio);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bp->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bp->join, cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "side stream (batch kernel grid)"));
  *out = bp;
  return KDE_OK;
}

extern "C" kde_status kde_batch_plan_query(kde_batch_plan bp, int64_t* x_rows, int64_t* density_elems,
                                           size_t* workspace_bytes) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  if (x_rows) *x_rows = bp->x_total;
  if (density_elems) *density_elems = bp->dens_elems;
  if (workspace_bytes) *workspace_bytes = bp->workspace_bytes;
  return KDE_OK;
}

extern "C" kde_status kde_batch_set_shape(kde_batch_plan bp, int tpl_rows, int tpl_cols) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  for (int t : {tpl_rows, tpl_cols})
    if (t != 32 && t != 64 && t != 128) return fail(KDE_ERR_INVALID_ARG, "threads per line: 32, 64 or 128");
  bp->tpl_rows = tpl_rows;
  bp->tpl_cols = tpl_cols;
  return KDE_OK;
}

extern "C" kde_status kde_batch_set_mode(kde_batch_plan bp, int mode) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  if (mode != KDE_BATCH_PERSISTENT && mode != KDE_BATCH_STAGED)
    return fail(KDE_ERR_INVALID_ARG, "mode: KDE_BATCH_PERSISTENT or KDE_BATCH_STAGED");
  bp->mode = mode;
  return KDE_OK;
}

extern "C" kde_status kde_batch_get_mode(kde_batch_plan bp, int* mode) {
  if (!bp || !mode) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  *mode = bp->mode;
  return KDE_OK;
}

extern "C" kde_status kde_batch_set_wait(kde_batch_plan bp, uint32_t polls, int withhold_stage) {
  if (!bp || polls == 0) return fail(KDE_ERR_INVALID_ARG, "need a plan and polls >= 1");
  if (withhold_stage < -1 || withhold_stage >= PS_COUNT)
    return fail(KDE_ERR_INVALID_ARG, "withhold_stage: -1 or a stage index 0..6");
  bp->wait_polls = polls;
  bp->withhold = withhold_stage;
  return KDE_OK;
}

extern "C" kde_status kde_batch_check(kde_batch_plan bp, kde_stream_t stream) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  unsigned flag = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(&flag, bp->ctl_dev + 3, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemset(bp->ctl_dev + 3, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "kde_batch_check");
  if (flag) return fail(KDE_ERR_TIMEOUT, "a wait of the persistent batch kernel gave up; the output is invalid");
  return KDE_OK;
}

extern "C" kde_status kde_batch_eval(kde_batch_plan bp, const void* X, void* density, void* workspace,
                                     size_t workspace_bytes, kde_stream_t stream) {
  if (!bp || !density || (!X && bp->x_total > 0)) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (!workspace || workspace_bytes < bp->workspace_bytes)
    return fail(KDE_ERR_WORKSPACE, "workspace smaller than the batch plan needs");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if (bp->precision == KDE_F32) return batch_eval_impl<float>(bp, X, density, workspace, st);
  return batch_eval_impl<double>(bp, X, density, workspace, st);
}

extern "C" kde_status kde_batch_plan_destroy(kde_batch_plan bp) {
  if (!bp) return KDE_OK;
  for (auto* p : bp->plans) kde_plan_destroy(p);
  cudaError_t e = cudaSuccess;
  if (bp->side) cudaStreamDestroy(bp->side);
  if (bp->fork) cudaEventDestroy(bp->fork);
  if (bp->join) cudaEventDestroy(bp->join);
  if (bp->items_dev) e = cudaFree(bp->items_dev);
  if (bp->wstart_dev) cudaFree(bp->wstart_dev);
  if (bp->pstart_dev) cudaFree(bp->pstart_dev);
  if (bp->ctl_dev) cudaFree(bp->ctl_dev);
  if (bp->queue_dev) cudaFree(bp->queue_dev);
  delete bp;
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaFree(batch)");
}

// Tuner for a batch plan: times kde_batch_eval with CUDA events on the
// stream (one warm-up and reps timed runs each) over the padding policy
// (smallest 7-smooth length, or the fewest radix stages within 25%), the
// radix order (largest or smallest radix first), the mode (persistent or
// staged) and the threads per line (32, 64, 128; rows and columns alike in
// the persistent mode, every pair in the staged one), skipping settings
// whose workspace exceeds the caller's, and keeps the fastest.  Re-plans
// the problems (set-up, not per evaluation); synchronises the stream.
extern "C" kde_status kde_batch_tune(kde_batch_plan bp, const void* X, void* density,
                                     void* workspace, size_t workspace_bytes, kde_stream_t stream,
                                     int reps, float* best_ms) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  if (reps < 1) reps = 3;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(KDE_ERR_CUDA, "cudaEventCreate");
  struct Cfg {
    int pad, order, mode, tr, tc, queue;
  };
  std::vector<Cfg> cfgs;
  for (int pad : {KDE_BATCH_PAD_SMALLEST, KDE_BATCH_PAD_FEWEST_STAGES})
    for (int order : {0, 1}) {
      for (int qo : {KDE_BATCH_QUEUE_PROBLEMS, KDE_BATCH_QUEUE_STAGES})
        for (int t : {32, 64, 128}) cfgs.push_back({pad, order, KDE_BATCH_PERSISTENT, t, t, qo});
      for (int tr : {32, 64, 128})
        for (int tc : {32, 64, 128})
          cfgs.push_back({pad, order, KDE_BATCH_STAGED, tr, tc, bp->queue_order});
    }
  float best = 1e30f;
  Cfg bc = {bp->pad_policy, bp->radix_order, bp->mode, bp->tpl_rows, bp->tpl_cols, bp->queue_order};
  // workspaces of at least 64 MB serve as the L2 flush between reps
  const size_t flush_bytes =
      workspace_bytes >= ((size_t)64 << 20) ? std::min(workspace_bytes, (size_t)256 << 20) : 0;
  // the timed runs go on a stream of the tuner's own, after the caller's
  // stream has reached this call
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return fail(KDE_ERR_CUDA, "cudaStreamCreate");
  }
  cudaEventRecord(e0, st);
  cudaStreamWaitEvent(cs, e0, 0);
  kde_status s = KDE_OK;
  int cur_pad = bp->pad_policy, cur_order = bp->radix_order, cur_q = bp->queue_order;
  for (const Cfg& c : cfgs) {
    if (c.pad != cur_pad || c.order != cur_order || c.queue != cur_q) {
      bp->pad_policy = c.pad;
      bp->radix_order = c.order;
      bp->queue_order = c.queue;
      if ((s = kde::batch_rebuild(bp)) != KDE_OK) break;
      cur_pad = c.pad;
      cur_order = c.order;
      cur_q = c.queue;
    }
    if (bp->workspace_bytes > workspace_bytes) continue;
    bp->mode = c.mode;
    bp->tpl_rows = c.tr;
    bp->tpl_cols = c.tc;
    if ((s = kde_batch_eval(bp, X, density, workspace, workspace_bytes, (kde_stream_t)cs)) != KDE_OK)
      break;
    // the evaluation as it is used: captured once as a CUDA graph (no host
    // gaps between the staged launches), replayed reps times; before each
    // replay a workspace of L2's order of size is overwritten (it is
    // scratch) so that the replay starts with the caches cold, as a new
    // batch would.  Plain launches if the capture fails.
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const kde_status sc = kde_batch_eval(bp, X, density, workspace, workspace_bytes, (kde_stream_t)cs);
      const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
      if (sc != KDE_OK || ec != cudaSuccess ||
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        graph = nullptr;
        exec = nullptr;
        cudaGetLastError();   // a failed capture leaves no error behind
      }
    } else {
      cudaGetLastError();
    }
    float ms = 0.f;
    for (int r = 0; r < reps && s == KDE_OK; ++r) {
      if (flush_bytes) {
        cudaError_t e = cudaMemsetAsync(workspace, 0, flush_bytes, cs);
        if (e != cudaSuccess) {
          s = cuda_fail(e, "cudaMemsetAsync(workspace)");
          break;
        }
      }
      cudaEventRecord(e0, cs);
      if (exec) {
        const cudaError_t e = cudaGraphLaunch(exec, cs);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaGraphLaunch(tuning run)");
      } else {
        s = kde_batch_eval(bp, X, density, workspace, workspace_bytes, (kde_stream_t)cs);
      }
      cudaEventRecord(e1, cs);
      if (s != KDE_OK) break;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        s = cuda_fail(e, "tuning run");
        break;
      }
      float one = 0.f;
      cudaEventElapsedTime(&one, e0, e1);
      ms += one;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (s != KDE_OK) break;
    ms /= reps;
    if (ms < best) {
      best = ms;
      bc = c;
    }
  }
  cudaStreamSynchronize(cs);
  cudaStreamDestroy(cs);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != KDE_OK) return s;
  if (bc.pad != cur_pad || bc.order != cur_order || bc.queue != cur_q) {
    bp->pad_policy = bc.pad;
    bp->radix_order = bc.order;
    bp->queue_order = bc.queue;
    if ((s = kde::batch_rebuild(bp)) != KDE_OK) return s;
  }
  bp->mode = bc.mode;
  bp->tpl_rows = bc.tr;
  bp->tpl_cols = bc.tc;
  if (best_ms) *best_ms = best;
  if ((s = kde_batch_check(bp, stream)) != KDE_OK) return s;
  return KDE_OK;
}

extern "C" kde_status kde_batch_set_queue_order(kde_batch_plan bp, int order) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  if (order != KDE_BATCH_QUEUE_STAGES && order != KDE_BATCH_QUEUE_PROBLEMS)
    return fail(KDE_ERR_INVALID_ARG, "order: KDE_BATCH_QUEUE_STAGES or KDE_BATCH_QUEUE_PROBLEMS");
  bp->queue_order = order;
  return kde::batch_work(bp);
}

extern "C" kde_status kde_batch_get_config(kde_batch_plan bp, int* pad_policy, int* radix_order,
                                           int64_t* P) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  if (pad_policy) *pad_policy = bp->pad_policy;
  if (radix_order) *radix_order = bp->radix_order | (bp->queue_order << 8);
  if (P)
    for (int i = 0; i < bp->count; ++i)
      for (int k = 0; k < 2; ++k) P[2 * i + k] = bp->plans[i]->info.P[k];
  return KDE_OK;
}

extern "C" kde_status kde_batch_get_shape(kde_batch_plan bp, int* tpl_rows, int* tpl_cols) {
  if (!bp) return fail(KDE_ERR_INVALID_ARG, "NULL plan");
  if (tpl_rows) *tpl_rows = bp->tpl_rows;
  if (tpl_cols) *tpl_cols = bp->tpl_cols;
  return KDE_OK;
}

KDE_DEBUG_READER(eval)
