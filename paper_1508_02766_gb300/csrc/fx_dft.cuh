// Register-resident DFTs of compile-time length N (FP32), for the two-phase
// FFT engine.  X_k = sum_n x_n e^{-2 pi i n k / N} in place, natural order in
// and out.  Composite lengths are split N = R M (R the largest of the base
// radices 8, 7, 5, 4, 3, 2 dividing N) by decimation in time: R interleaved
// sub-sequences of length M are transformed, multiplied by e^{-2 pi i r k / N}
// and combined by length-R DFTs; every index and twiddle is a compile-time
// constant, so the whole transform unrolls into registers.  The inverse
// (unnormalised) is conj(DFT(conj(x))).
#pragma once

#include <cuda_runtime.h>

#include "fft_engine.cuh"
#include "fx_math.h"

namespace kde {
namespace fx {

constexpr int base_radix(int N) {
  return N % 8 == 0 ? 8 : N % 7 == 0 ? 7 : N % 5 == 0 ? 5 : N % 4 == 0 ? 4 : N % 3 == 0 ? 3 : 2;
}

constexpr bool is_base(int N) { return N == 2 || N == 3 || N == 4 || N == 5 || N == 7 || N == 8; }

// x * e^{-2 pi i e / N} with the exponent known at compile time; quarter
// turns are swaps and sign changes.
template <int N, int E>
__device__ __forceinline__ float2 twiddle_mul(float2 x) {
  constexpr int e = E % N;
  if constexpr (e == 0) {
    return x;
  } else if constexpr ((4 * e) % N == 0) {
    constexpr int q = (4 * e) / N;  // e^{-i q pi / 2}
    if constexpr (q == 1) return make_float2(x.y, -x.x);
    else if constexpr (q == 2) return make_float2(-x.x, -x.y);
    else return make_float2(-x.y, x.x);
  } else {
    constexpr fxm::CS cs = fxm::cossin_2pi(e, N);
    constexpr float c = (float)cs.c, s = (float)(-cs.s);
    return make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
  }
}

template <int N, int R = base_radix(N), bool BASE = is_base(N)>
struct DFT;

template <int N, int R>
struct DFT<N, R, true> {
  __device__ __forceinline__ static void run(float2* x) { SmallDFT<float2, N, false>::run(x); }
};

template <int R>
struct DFT<1, R, false> {
  __device__ __forceinline__ static void run(float2*) {}
};

template <int N, int R>
struct DFT<N, R, false> {
  static constexpr int M = N / R;
  template <int r>
  __device__ __forceinline__ static void twiddle_row(float2 (&y)[R][M]) {
    if constexpr (r < R) {
      twiddle_cols<r, 1>(y);
      twiddle_row<r + 1>(y);
    }
  }
  template <int r, int k>
  __device__ __forceinline__ static void twiddle_cols(float2 (&y)[R][M]) {
    if constexpr (k < M) {
      y[r][k] = twiddle_mul<N, r * k>(y[r][k]);
      twiddle_cols<r, k + 1>(y);
    }
  }
  __device__ __forceinline__ static void run(float2* x) {
    float2 y[R][M];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int m = 0; m < M; ++m) y[r][m] = x[R * m + r];
#pragma unroll
    for (int r = 0; r < R; ++r) DFT<M>::run(y[r]);
    twiddle_row<1>(y);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      float2 t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = y[r][k];
      SmallDFT<float2, R, false>::run(t);
#pragma unroll
      for (int q = 0; q < R; ++q) x[k + M * q] = t[q];
    }
  }
};

template <int N>
__device__ __forceinline__ void dft(float2* x) {
  DFT<N>::run(x);
}

// Unnormalised inverse: conj(DFT(conj(x))).
template <int N>
__device__ __forceinline__ void idft(float2* x) {
#pragma unroll
  for (int i = 0; i < N; ++i) x[i].y = -x[i].y;
  DFT<N>::run(x);
#pragma unroll
  for (int i = 0; i < N; ++i) x[i].y = -x[i].y;
}

}  // namespace fx
}  // namespace kde
