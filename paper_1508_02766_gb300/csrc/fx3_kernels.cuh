// Three-phase variant of the two-phase passes, for long lines (P > 400):
// P = N1 N2 N3 with every factor about 10, so that a line is spread over
// P / min(N) threads (about 120 for P = 1080) holding ~10 values each instead
// of ~36 threads holding ~30 (long lines are few, so the passes need the
// extra threads to fill the GPU).  With N23 = N2 N3, n = n23 + N23 n1,
// n23 = n3 + N3 n2 and k = k1 + N1 (k2 + N2 k3):
//   phase A: thread n23 takes the N1-point DFT over n1 of x[n23 + N23 n1],
//            times e^{-2 pi i n23 k1 / P};
//   phase B: thread (k1, n3) the N2-point DFT over n2, times
//            e^{-2 pi i n3 k2 / N23};
//   phase C: thread (k1, k2) the N3-point DFT over n3, which gives
//            X[k1 + N1 (k2 + N2 k3)].
// The inverse runs C, B, A with conjugate twiddles.  One exchange buffer per
// line in shared memory, entry (k1, j) at k1 SK + j: phase A writes
// j = n23, phase B rewrites the slots it read (j = n3 + N3 n2 -> value for
// k2 = n2), phase C rewrites its slots (j = n3 + N3 k2 -> value for k3 = n3).
// Input positions n23 + N23 n1 and output positions k1 + N1 (k2 + N2 k3) are
// contiguous across neighbouring threads, so lines go to and from global
// memory directly.
#pragma once

#include "fx_kernels.cuh"

namespace kde {
namespace fx {

inline constexpr int kThreads3 = 512;

template <int N1, int N2, int N3>
constexpr int threads_per_line3() {
  constexpr int a = N2 * N3, b = N1 * N3, c = N1 * N2;
  return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

// ---- shared phase bodies on one line's exchange buffer --------------------

// Phase A forward: x (N1 values of thread n23) -> slots (k1, n23).
template <int N1, int N2, int N3>
__device__ __forceinline__ void p3_a_fwd(float2 (&x)[N1], int n23, const float2* __restrict__ tw,
                                         float2* line, int SK, int SJ) {
  dft<N1>(x);
  line[n23 * SJ] = x[0];
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) line[k1 * SK + n23 * SJ] = cmul(x[k1], __ldg(tw + n23 * k1));
}

// Phase B forward on thread (k1, n3): slots (k1, n3 + N3 n2) in place.
template <int N1, int N2, int N3>
__device__ __forceinline__ void p3_b_fwd(int k1, int n3, const float2* __restrict__ tw, float2* line,
                                         int SK, int SJ) {
  float2* base = line + k1 * SK + n3 * SJ;
  float2 y[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) y[n2] = base[N3 * n2 * SJ];
  dft<N2>(y);
  base[0] = y[0];
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) base[N3 * k2 * SJ] = cmul(y[k2], __ldg(tw + N1 * n3 * k2));
}

// Phase C forward on thread (k1, k2): z[k3] = X[k1 + N1 (k2 + N2 k3)].
template <int N1, int N2, int N3>
__device__ __forceinline__ void p3_c_fwd(float2 (&z)[N3], int k1, int k2, const float2* line, int SK,
                                         int SJ) {
  const float2* base = line + k1 * SK + N3 * k2 * SJ;
#pragma unroll
  for (int n3 = 0; n3 < N3; ++n3) z[n3] = base[n3 * SJ];
  dft<N3>(z);
}

// Phase C inverse on thread (k1, k2): z[k3] = X[k1 + N1 (k2 + N2 k3)] ->
// slots (k1, n3 + N3 k2).
template <int N1, int N2, int N3>
__device__ __forceinline__ void p3_c_inv(float2 (&z)[N3], int k1, int k2,
                                         const float2* __restrict__ tw, float2* line, int SK, int SJ) {
  idft<N3>(z);
  float2* base = line + k1 * SK + N3 * k2 * SJ;
  base[0] = z[0];
#pragma unroll
  for (int n3 = 1; n3 < N3; ++n3) base[n3 * SJ] = cmulc(z[n3], __ldg(tw + N1 * n3 * k2));
}

// Phase B inverse on thread (k1, n3): slots (k1, n3 + N3 k2) in place, the
// value for n2 times e^{+2 pi i (n3 + N3 n2) k1 / P}.
template <int N1, int N2, int N3>
__device__ __forceinline__ void p3_b_inv(int k1, int n3, const float2* __restrict__ tw, float2* line,
                                         int SK, int SJ) {
  float2* base = line + k1 * SK + n3 * SJ;
  float2 y[N2];
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) y[k2] = base[N3 * k2 * SJ];
  idft<N2>(y);
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    const int n23 = n3 + N3 * n2;
    base[N3 * n2 * SJ] = (n23 * k1 == 0) ? y[n2] : cmulc(y[n2], __ldg(tw + n23 * k1));
  }
}

// Phase A inverse on thread n23: x[n1] = value at position n23 + N23 n1.
template <int N1, int N2, int N3>
__device__ __forceinline__ void p3_a_inv(float2 (&x)[N1], int n23, const float2* line, int SK,
                                         int SJ) {
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) x[k1] = line[k1 * SK + n23 * SJ];
  idft<N1>(x);
}

// Slot of X[k] after phase C (rows): k1 = k mod N1, k2, k3 from k / N1.
template <int N1, int N2, int N3>
__device__ __forceinline__ int p3_slot(int k, int SK) {
  const int k1 = k % N1, r = k / N1;
  return k1 * SK + (r / N2) + N3 * (r % N2);
}

// ---- rows ------------------------------------------------------------------
template <int N1, int N2, int N3, int SRC>
__global__ void __launch_bounds__(kThreads3)
kde_fx3_rows_fwd_kernel(RowsArgs a, const long long* __restrict__ counts, KGen<float> g) {
  pdl_trigger();
  pdl_wait();
  constexpr int N23 = N2 * N3, P = N1 * N23;
  extern __shared__ float2 fx_sm[];
  rows_slab(a, g);
  const int SK = a.SK, LS = N1 * SK;
  const int t = threadIdx.x;
  if constexpr (SRC == SRC_KGEN) {
    rows_stage_kgen(a, g, fx_sm + a.B * LS);
    __syncthreads();
  }
  if (t < a.B * N23) {  // phase A
    const int b = t / N23, n23 = t - b * N23;
    const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
    if (r0 < a.nrows) {
      const bool two = r0 + 1 < a.nrows;
      float2 x[N1];
      if constexpr (SRC == SRC_COUNTS) {
        const long long* c0 = counts + r0 * a.in_stride;
        const long long* c1 = two ? c0 + a.in_stride : c0;
        long long v0[N1], v1[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
          const int pos = n23 + N23 * n1;
          v0[n1] = pos < a.Min ? __ldg(c0 + pos) : 0;
          v1[n1] = (pos < a.Min && two) ? __ldg(c1 + pos) : 0;
        }
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1)
          x[n1] = make_float2(count_value<float>(v0[n1]), count_value<float>(v1[n1]));
      } else {
        const float2* stage = fx_sm + a.B * LS + (size_t)b * P;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = stage[n23 + N23 * n1];
      }
      p3_a_fwd<N1, N2, N3>(x, n23, a.tw, fx_sm + b * LS, SK, 1);
    }
  }
  __syncthreads();
  if (t < a.B * N1 * N3) {  // phase B
    const int b = t / (N1 * N3), r = t - b * (N1 * N3);
    p3_b_fwd<N1, N2, N3>(r / N3, r % N3, a.tw, fx_sm + b * LS, SK, 1);
  }
  __syncthreads();
  if (t < a.B * N1 * N2) {  // phase C, results back to the slots
    const int b = t / (N1 * N2), r = t - b * (N1 * N2);
    const int k1 = r % N1, k2 = r / N1;
    float2 z[N3];
    p3_c_fwd<N1, N2, N3>(z, k1, k2, fx_sm + b * LS, SK, 1);
    float2* base = fx_sm + b * LS + k1 * SK + N3 * k2;
#pragma unroll
    for (int k3 = 0; k3 < N3; ++k3) base[k3] = z[k3];
  }
  __syncthreads();
  // X = F(x), Y = F(y) from Z = F(x + i y) on [0, Q)
  for (int b = 0; b < a.B; ++b) {
    const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
    if (r0 >= a.nrows) break;
    const bool two = r0 + 1 < a.nrows;
    const float2* z = fx_sm + b * LS;
    float2* o0 = a.out + r0 * a.Q;
    for (int k = t; k < a.Q; k += blockDim.x) {
      const int km = k == 0 ? 0 : P - k;
      const float2 zk = z[p3_slot<N1, N2, N3>(k, SK)];
      const float2 zm = z[p3_slot<N1, N2, N3>(km, SK)];
      o0[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      if (two) o0[a.Q + k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
  }
}

template <int N1, int N2, int N3>
__global__ void __launch_bounds__(kThreads3) kde_fx3_rows_c2r_kernel(RowsArgs a) {
  pdl_trigger();
  pdl_wait();
  constexpr int N23 = N2 * N3, P = N1 * N23;
  extern __shared__ float2 fx_sm[];
  KGen<float> g_unused;
  rows_slab(a, g_unused);
  const int SK = a.SK, LS = N1 * SK;
  const int t = threadIdx.x;
  if (t < a.B * N1 * N2) {  // phase C inverse from the half spectra
    const int b = t / (N1 * N2), r = t - b * (N1 * N2);
    const int k1 = r % N1, k2 = r / N1;
    const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
    if (r0 < a.nrows) {
      const bool two = r0 + 1 < a.nrows;
      const float2* x0 = a.in + r0 * a.Q;
      const float2* x1 = two ? x0 + a.Q : x0;
      float2 z[N3];
#pragma unroll
      for (int k3 = 0; k3 < N3; ++k3) {
        const int k = k1 + N1 * (k2 + N2 * k3);
        const bool lo = k < a.Q;
        const int kk = lo ? k : P - k;
        const float2 X = __ldg(x0 + kk);
        const float2 Y = two ? __ldg(x1 + kk) : make_float2(0.f, 0.f);
        z[k3] = lo ? make_float2(X.x - Y.y, X.y + Y.x) : make_float2(X.x + Y.y, Y.x - X.y);
      }
      p3_c_inv<N1, N2, N3>(z, k1, k2, a.tw, fx_sm + b * LS, SK, 1);
    }
  }
  __syncthreads();
  if (t < a.B * N1 * N3) {
    const int b = t / (N1 * N3), r = t - b * (N1 * N3);
    p3_b_inv<N1, N2, N3>(r / N3, r % N3, a.tw, fx_sm + b * LS, SK, 1);
  }
  __syncthreads();
  if (t < a.B * N23) {
    const int b = t / N23, n23 = t - b * N23;
    const int64_t r0 = 2 * ((int64_t)blockIdx.x * a.B + b);
    if (r0 < a.nrows) {
      const bool two = r0 + 1 < a.nrows;
      float2 x[N1];
      p3_a_inv<N1, N2, N3>(x, n23, fx_sm + b * LS, SK, 1);
      float* o0 = a.out_real + r0 * a.Mout;
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) {
        const int pos = n23 + N23 * n1;
        if (pos < a.Mout) {
          o0[pos] = x[n1].x;
          if (two) o0[a.Mout + pos] = x[n1].y;
        }
      }
    }
  }
}

// ---- columns: W = 2^lgB adjacent columns, column index fastest; entry
// (column c, k1, j) at c + j W + k1 SK ------------------------------------------
template <int N1, int N2, int N3, int MODE>
__global__ void __launch_bounds__(kThreads3) kde_fx3_cols_kernel(ColsArgs a) {
  pdl_trigger();
  pdl_wait();
  constexpr int N23 = N2 * N3, P = N1 * N23;
  extern __shared__ float2 fx_sm[];
  cols_slab(a);
  const int W = a.B, SK = a.SK;
  const int t = threadIdx.x;
  const int c = t & (W - 1), r = t >> a.lgB;
  const int64_t first = (int64_t)blockIdx.x * W * (MODE == COL_FWD_REAL ? 2 : 1);
  float2* line = fx_sm + c;
  // COL_MID: the kernel spectrum values of this thread's phase C, loaded
  // now so that their latency hides behind phases A and B
  float kpre[MODE == COL_MID ? N3 : 1];
  if constexpr (MODE == COL_MID) {
    const int64_t s = first + c;
    const bool v = s < a.S && r < N1 * N2;
    const float* pk = a.K + s + (int64_t)(r % N1 + N1 * (r / N1)) * a.S;
    const int64_t step = (int64_t)(N1 * N2) * a.S;
#pragma unroll
    for (int k3 = 0; k3 < N3; ++k3) {
      kpre[k3] = v ? __ldg(pk) : 0.f;
      pk += step;
    }
  }
  if constexpr (MODE == COL_INV) {
    if (r < N1 * N2) {  // phase C inverse from the input rows
      const int k1 = r % N1, k2 = r / N1;
      const int64_t s = first + c;
      const bool v = s < a.S;
      // rows k1 + N1 (k2 + N2 k3): one pointer stepped by N1 N2 rows
      const float2* in = a.in + s + (int64_t)(k1 + N1 * k2) * a.S;
      const int64_t step = (int64_t)(N1 * N2) * a.S;
      float2 z[N3];
#pragma unroll
      for (int k3 = 0; k3 < N3; ++k3) {
        z[k3] = v ? __ldg(in) : make_float2(0.f, 0.f);
        in += step;
      }
      p3_c_inv<N1, N2, N3>(z, k1, k2, a.tw, line, SK, W);
    }
  } else {
    if (r < N23) {  // phase A
      const int n23 = r;
      const float2* in = a.in;
      float2 x[N1];
      if constexpr (MODE == COL_FWD_REAL) {
        const int64_t s = first + 2 * c;
        const bool v0 = s < a.S, v1 = s + 1 < a.S;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
          const int j = col_source(n23 + N23 * n1, P, a.Lw, a.Nin);
          float2 p = make_float2(0.f, 0.f), q = make_float2(0.f, 0.f);
          if (j >= 0) {
            if (v0) p = __ldg(in + (int64_t)j * a.S + s);
            if (v1) q = __ldg(in + (int64_t)j * a.S + s + 1);
          }
          x[n1] = make_float2(p.x - q.y, p.y + q.x);
        }
      } else {
        const int64_t s = first + c;
        const bool v = s < a.S;
        if (a.Lw < 0) {  // plain rows: position pos reads row pos < Nin
          const float2* p = in + s + (int64_t)n23 * a.S;
          const int64_t step = (int64_t)N23 * a.S;
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) {
            x[n1] = (n23 + N23 * n1 < a.Nin && v) ? __ldg(p) : make_float2(0.f, 0.f);
            p += step;
          }
        } else {
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) {
            const int j = col_source(n23 + N23 * n1, P, a.Lw, a.Nin);
            x[n1] = (j >= 0 && v) ? __ldg(in + (int64_t)j * a.S + s) : make_float2(0.f, 0.f);
          }
        }
      }
      p3_a_fwd<N1, N2, N3>(x, n23, a.tw, line, SK, W);
    }
    __syncthreads();
    if (r < N1 * N3) p3_b_fwd<N1, N2, N3>(r / N3, r % N3, a.tw, line, SK, W);
    __syncthreads();
    if (r < N1 * N2) {  // phase C
      const int k1 = r % N1, k2 = r / N1;
      float2 z[N3];
      p3_c_fwd<N1, N2, N3>(z, k1, k2, line, SK, W);
      if constexpr (MODE == COL_FWD) {
        const int64_t s = first + c;
        if (s < a.S) {
          float2* out = a.out + s + (int64_t)(k1 + N1 * k2) * a.S;
          const int64_t step = (int64_t)(N1 * N2) * a.S;
#pragma unroll
          for (int k3 = 0; k3 < N3; ++k3) {
            *out = z[k3];
            out += step;
          }
        }
      } else if constexpr (MODE == COL_FWD_REAL) {
        const int64_t s = first + 2 * c;
        if (s < a.S) {
          const bool v1 = s + 1 < a.S;
          float* out = a.out_real + s;
#pragma unroll
          for (int k3 = 0; k3 < N3; ++k3) {
            const int64_t k = k1 + N1 * (k2 + N2 * k3);
            out[k * a.S] = z[k3].x;
            if (v1) out[k * a.S + 1] = z[k3].y;
          }
        }
      } else {  // COL_MID: times K, inverse phase C back to the slots
        if constexpr (MODE == COL_AUTO) {  // the power spectrum, for the autocorrelation
#pragma unroll
          for (int k3 = 0; k3 < N3; ++k3) {
            const float re = z[k3].x * a.s_pre, im = z[k3].y * a.s_pre;
            z[k3] = make_float2((re * re + im * im) * a.s_post, 0.f);
          }
        } else {
#pragma unroll
          for (int k3 = 0; k3 < N3; ++k3) {
            z[k3].x *= kpre[k3];
            z[k3].y *= kpre[k3];
          }
        }
        p3_c_inv<N1, N2, N3>(z, k1, k2, a.tw, line, SK, W);
      }
    }
  }
  if constexpr (MODE == COL_MID || MODE == COL_AUTO || MODE == COL_INV) {
    __syncthreads();
    if (r < N1 * N3) p3_b_inv<N1, N2, N3>(r / N3, r % N3, a.tw, line, SK, W);
    __syncthreads();
    if (r < N23) {
      const int64_t s = first + c;
      if (s < a.S) {
        float2 x[N1];
        p3_a_inv<N1, N2, N3>(x, r, line, SK, W);
        float2* out = a.out + s + (int64_t)r * a.S;
        const int64_t step = (int64_t)N23 * a.S;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
          if (r + N23 * n1 < a.Nout) *out = x[n1];
          out += step;
        }
      }
    }
  }
  if (a.clear) clear_words(a.clear, a.clear_n);
}

}  // namespace fx
}  // namespace kde
