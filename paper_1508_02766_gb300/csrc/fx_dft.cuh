// Register-resident DFTs of compile-time length N (FP32), for the two-phase
// FFT engine.  X_k = sum_n x_n e^{-+2 pi i n k / N} in place, natural order
// in and out (the inverse unnormalised).  Composite lengths are split
// N = R M (R the largest of the base radices 8, 7, 5, 4, 3, 2 dividing N) by
// decimation in time: R interleaved sub-sequences of length M are
// transformed, multiplied by e^{-+2 pi i r k / N} and combined by length-R
// DFTs; every index and twiddle is a compile-time constant, so the whole
// transform unrolls into registers.
//
// The arithmetic is packed: a complex value is one f32x2 register pair, so a
// complex sum is one packed add, a product with a real constant one packed
// multiply (or fused multiply-add), and a sum with a rotated value
// a -+ i b one packed fused multiply-add of the swapped pair (b.y, b.x) by
// (+-1, -+1) (a product with +-1 is exact, so each component is still one
// rounded addition).  Every component is rounded as the scalar FP32
// operation of the same form would be.
#pragma once

#include <cuda_runtime.h>

#include "fx_math.h"

namespace kde {
namespace fx {

constexpr int base_radix(int N) {
  return N % 8 == 0 ? 8 : N % 7 == 0 ? 7 : N % 5 == 0 ? 5 : N % 4 == 0 ? 4 : N % 3 == 0 ? 3 : 2;
}

constexpr bool is_base(int N) { return N == 2 || N == 3 || N == 4 || N == 5 || N == 7 || N == 8; }

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b: b times (-1, -1) (exact) plus a, one rounding per component
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 p_scale(float2 a, float c) { return __fmul2_rn(a, make_float2(c, c)); }
// acc + a c
__device__ __forceinline__ float2 p_fma(float2 a, float c, float2 acc) {
  return __ffma2_rn(a, make_float2(c, c), acc);
}
// rot(b) = -i b (forward) or +i b (inverse); a + rot(b) and a - rot(b)
template <bool INV>
__device__ __forceinline__ float2 p_add_rot(float2 a, float2 b) {
  return __ffma2_rn(make_float2(b.y, b.x), INV ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f), a);
}
template <bool INV>
__device__ __forceinline__ float2 p_sub_rot(float2 a, float2 b) {
  return __ffma2_rn(make_float2(b.y, b.x), INV ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f), a);
}

// x e^{-+2 pi i E / N} with the exponent known at compile time; quarter
// turns are exact component moves and sign changes.
template <int N, int E, bool INV>
__device__ __forceinline__ float2 twiddle_mul(float2 x) {
  constexpr int e = E % N;
  if constexpr (e == 0) {
    return x;
  } else if constexpr ((4 * e) % N == 0) {
    constexpr int q = (4 * e) / N;  // e^{-+ i q pi / 2}
    if constexpr (q == 2) return make_float2(-x.x, -x.y);
    else if constexpr ((q == 1) != INV) return make_float2(x.y, -x.x);   // -i x
    else return make_float2(-x.y, x.x);                                  // +i x
  } else {
    constexpr fxm::CS cs = fxm::cossin_2pi(e, N);
    constexpr float c = (float)cs.c, s = (float)cs.s;
    // forward x (c - i s) = (x.x c + x.y s, x.y c - x.x s); inverse with -s
    const float2 t = __fmul2_rn(x, make_float2(c, c));
    return __ffma2_rn(make_float2(x.y, x.x), INV ? make_float2(-s, s) : make_float2(s, -s), t);
  }
}

// Length-R DFTs of the base radices.
template <int R, bool INV>
struct BaseDFT;

template <bool INV>
struct BaseDFT<2, INV> {
  __device__ __forceinline__ static void run(float2* x) {
    const float2 a = x[0], b = x[1];
    x[0] = p_add(a, b);
    x[1] = p_sub(a, b);
  }
};

template <bool INV>
struct BaseDFT<4, INV> {
  __device__ __forceinline__ static void run(float2* x) {
    const float2 t0 = p_add(x[0], x[2]), t1 = p_sub(x[0], x[2]);
    const float2 t2 = p_add(x[1], x[3]), d = p_sub(x[1], x[3]);
    x[0] = p_add(t0, t2);
    x[2] = p_sub(t0, t2);
    x[1] = p_add_rot<INV>(t1, d);
    x[3] = p_sub_rot<INV>(t1, d);
  }
};

template <bool INV>
struct BaseDFT<8, INV> {
  __device__ __forceinline__ static void run(float2* x) {
    constexpr float h = 0.70710678118654752440f;
    float2 e[4] = {x[0], x[2], x[4], x[6]};
    float2 o[4] = {x[1], x[3], x[5], x[7]};
    BaseDFT<4, INV>::run(e);
    BaseDFT<4, INV>::run(o);
    // o_k times w_8^k, w_8 = e^{-+ i pi / 4}: (o_1 + rot o_1) / sqrt 2,
    // rot o_2, (rot o_3 - o_3) / sqrt 2
    const float2 w1 = p_scale(p_add_rot<INV>(o[1], o[1]), h);
    const float2 w3 = p_scale(p_sub_rot<INV>(o[3], o[3]), -h);
    x[0] = p_add(e[0], o[0]);
    x[4] = p_sub(e[0], o[0]);
    x[1] = p_add(e[1], w1);
    x[5] = p_sub(e[1], w1);
    x[2] = p_add_rot<INV>(e[2], o[2]);
    x[6] = p_sub_rot<INV>(e[2], o[2]);
    x[3] = p_add(e[3], w3);
    x[7] = p_sub(e[3], w3);
  }
};

// Odd R: pair legs n and R - n; A_k = x_0 + sum_n (x_n + x_{R-n}) cos(2 pi n k / R),
// B_k = sum_n (x_n - x_{R-n}) sin(2 pi n k / R); X_k = A_k + rot B_k,
// X_{R-k} = A_k - rot B_k.
template <int R, bool INV>
struct BaseDFT {
  static constexpr int H = (R - 1) / 2;
  __device__ __forceinline__ static void run(float2* x) {
    float2 sp[H], sm[H];
#pragma unroll
    for (int n = 1; n <= H; ++n) {
      sp[n - 1] = p_add(x[n], x[R - n]);
      sm[n - 1] = p_sub(x[n], x[R - n]);
    }
    float2 y[R];
    float2 s0 = x[0];
#pragma unroll
    for (int n = 0; n < H; ++n) s0 = p_add(s0, sp[n]);
    y[0] = s0;
    odd_terms<1>(x[0], sp, sm, y);
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = y[k];
  }
  template <int K>
  __device__ __forceinline__ static void odd_terms(float2 x0, const float2 (&sp)[H], const float2 (&sm)[H],
                                                   float2 (&y)[R]) {
    if constexpr (K <= H) {
      float2 A = x0, B;
      odd_sum<K, 1>(sp, sm, A, B);
      y[K] = p_add_rot<INV>(A, B);
      y[R - K] = p_sub_rot<INV>(A, B);
      odd_terms<K + 1>(x0, sp, sm, y);
    }
  }
  template <int K, int N>
  __device__ __forceinline__ static void odd_sum(const float2 (&sp)[H], const float2 (&sm)[H], float2& A,
                                                 float2& B) {
    if constexpr (N <= H) {
      constexpr fxm::CS cs = fxm::cossin_2pi((long long)N * K, R);
      constexpr float c = (float)cs.c, s = (float)cs.s;
      A = p_fma(sp[N - 1], c, A);
      B = N == 1 ? p_scale(sm[0], s) : p_fma(sm[N - 1], s, B);
      odd_sum<K, N + 1>(sp, sm, A, B);
    }
  }
};

template <int N, bool INV, int R = base_radix(N), bool BASE = is_base(N)>
struct DFT;

template <int N, bool INV, int R>
struct DFT<N, INV, R, true> {
  __device__ __forceinline__ static void run(float2* x) { BaseDFT<N, INV>::run(x); }
};

template <bool INV, int R>
struct DFT<1, INV, R, false> {
  __device__ __forceinline__ static void run(float2*) {}
};

template <int N, bool INV, int R>
struct DFT<N, INV, R, false> {
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
      y[r][k] = twiddle_mul<N, r * k, INV>(y[r][k]);
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
    for (int r = 0; r < R; ++r) DFT<M, INV>::run(y[r]);
    twiddle_row<1>(y);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      float2 t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = y[r][k];
      BaseDFT<R, INV>::run(t);
#pragma unroll
      for (int q = 0; q < R; ++q) x[k + M * q] = t[q];
    }
  }
};

template <int N>
__device__ __forceinline__ void dft(float2* x) {
  DFT<N, false>::run(x);
}

// Unnormalised inverse: X_k = sum_n x_n e^{+2 pi i n k / N}.
template <int N>
__device__ __forceinline__ void idft(float2* x) {
  DFT<N, true>::run(x);
}

}  // namespace fx
}  // namespace kde
