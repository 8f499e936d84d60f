// Mixed-radix FFT engine (radices 2, 3, 4, 5, 7, 8) for one line per group
// of threads.  (Larger radices nested in registers cut the passes over
// shared memory but raised every kernel to 128+ registers and lost more to
// occupancy than they saved; they are not used.)
//
// A group of tpl threads (tpl a multiple of 32) transforms one complex line
// of length N held in shared memory, with the self-sorting Stockham scheme:
// with Ns the product of the radices already applied, butterfly j of a
// radix-R stage reads x[j + r N/R], multiplies leg r by
// w_N^{r (j mod Ns) N/(Ns R)}, takes a length-R DFT and writes leg r to
// (j - j mod Ns) R + (j mod Ns) + r Ns.  Stages ping-pong between two buffers
// of the line, so the output is in natural order.  A group synchronises only
// itself: __syncwarp for one warp, a named barrier otherwise, so the lines
// of a block run independently.  tpl is chosen per launch from the number of
// lines: few long lines get many threads each, many lines get a warp each.
// Divisions by Ns use a precomputed reciprocal (exact for j, Ns < 2^13).
#pragma once

#include <cuda_runtime.h>

#include "../../include/kde_gb300.h"
#include "fx_dft.cuh"

namespace kde {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) {
  V v;
  v.x = a;
  v.y = b;
  return v;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
// Multiply by -i (forward) or +i (inverse).
template <typename V, bool INV> __device__ __forceinline__ V rot90(V a) {
  return INV ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}

// One stage of a line plan.  magic = floor(2^32 / Ns) + 1, so that
// j / Ns = umulhi(j, magic) for the j < 2^13 that occur.
struct Stage {
  int R, Ns, nb, twstep;
  unsigned magic;
};

struct LinePlan {
  int N;
  int nst;
  Stage st[KDE_MAX_STAGES];
};

// cos and sin of 2 pi m / R, m = 1 .. (R-1)/2, for the odd radices.
__device__ __forceinline__ double odd_cos(int R, int m) {
  if (R == 3) return -0.5;
  if (R == 5) return m == 1 ? 0.3090169943749474241022934 : -0.8090169943749474241022934;
  return m == 1 ? 0.6234898018587335305250049
                : (m == 2 ? -0.2225209339563144042889026 : -0.9009688679024191262361023);
}
__device__ __forceinline__ double odd_sin(int R, int m) {
  if (R == 3) return 0.8660254037844386467637232;
  if (R == 5) return m == 1 ? 0.9510565162951535721164393 : 0.5877852522924731291687060;
  return m == 1 ? 0.7818314824680298087084445
                : (m == 2 ? 0.9749279121818236070181317 : 0.4338837391175581204757683);
}

// Length-R DFT in registers, X_k = sum_n x_n e^{-+ 2 pi i n k / R}.
template <typename V, int R, bool INV> struct SmallDFT;

template <typename V, bool INV> struct SmallDFT<V, 2, INV> {
  __device__ __forceinline__ static void run(V* x) {
    V a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <typename V, bool INV> struct SmallDFT<V, 4, INV> {
  __device__ __forceinline__ static void run(V* x) {
    V t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
    V t2 = cadd(x[1], x[3]), t3 = rot90<V, INV>(csub(x[1], x[3]));
    x[0] = cadd(t0, t2);
    x[2] = csub(t0, t2);
    x[1] = cadd(t1, t3);
    x[3] = csub(t1, t3);
  }
};

template <typename V, bool INV> struct SmallDFT<V, 8, INV> {
  __device__ __forceinline__ static void run(V* x) {
    using R = decltype(V::x);
    const R h = (R)0.7071067811865475244008444;
    V e[4] = {x[0], x[2], x[4], x[6]};
    V o[4] = {x[1], x[3], x[5], x[7]};
    SmallDFT<V, 4, INV>::run(e);
    SmallDFT<V, 4, INV>::run(o);
    // o_k *= w_8^k with w_8 = e^{-+ i pi / 4}
    V o1 = rot90<V, INV>(o[1]);
    V w1 = mk<V>(h * (o[1].x + o1.x), h * (o[1].y + o1.y));   // (1 -+ i)/sqrt2 * o1
    V o2 = rot90<V, INV>(o[2]);
    V o3r = rot90<V, INV>(o[3]);
    V w3 = mk<V>(h * (o3r.x - o[3].x), h * (o3r.y - o[3].y));  // (-1 -+ i)/sqrt2 * o3
    x[0] = cadd(e[0], o[0]);
    x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], w1);
    x[5] = csub(e[1], w1);
    x[2] = cadd(e[2], o2);
    x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], w3);
    x[7] = csub(e[3], w3);
  }
};

// Odd R: pair legs n and R-n; A_k = x0 + sum (x_n + x_{R-n}) cos,
// B_k = sum (x_n - x_{R-n}) sin; X_k = A_k -+ i B_k, X_{R-k} = A_k +- i B_k.
template <typename V, int R, bool INV> struct SmallDFT {
  __device__ __forceinline__ static void run(V* x) {
    using F = decltype(V::x);
    constexpr int H = (R - 1) / 2;
    V sp[H], sm[H];
#pragma unroll
    for (int n = 1; n <= H; ++n) {
      sp[n - 1] = cadd(x[n], x[R - n]);
      sm[n - 1] = csub(x[n], x[R - n]);
    }
    V y[R];
    V s0 = x[0];
#pragma unroll
    for (int n = 0; n < H; ++n) s0 = cadd(s0, sp[n]);
    y[0] = s0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      V A = x[0], B = mk<V>(0, 0);
#pragma unroll
      for (int n = 1; n <= H; ++n) {
        int m = (n * k) % R;
        F c, s;
        if (m <= H) {
          c = (F)odd_cos(R, m);
          s = (F)odd_sin(R, m);
        } else {
          c = (F)odd_cos(R, R - m);
          s = -(F)odd_sin(R, R - m);
        }
        A.x += sp[n - 1].x * c;
        A.y += sp[n - 1].y * c;
        B.x += sm[n - 1].x * s;
        B.y += sm[n - 1].y * s;
      }
      V iB = rot90<V, INV>(B);  // -+ i B
      y[k] = cadd(A, iB);
      y[R - k] = csub(A, iB);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = y[k];
  }
};

// FP32: the same DFTs in packed f32x2 arithmetic (the two-phase engine's
// base radices); each component is rounded as in the scalar form.
template <int R, bool INV> struct SmallDFT<float2, R, INV> {
  __device__ __forceinline__ static void run(float2* x) { fx::BaseDFT<R, INV>::run(x); }
};
template <bool INV> struct SmallDFT<float2, 2, INV> {
  __device__ __forceinline__ static void run(float2* x) { fx::BaseDFT<2, INV>::run(x); }
};
template <bool INV> struct SmallDFT<float2, 4, INV> {
  __device__ __forceinline__ static void run(float2* x) { fx::BaseDFT<4, INV>::run(x); }
};
template <bool INV> struct SmallDFT<float2, 8, INV> {
  __device__ __forceinline__ static void run(float2* x) { fx::BaseDFT<8, INV>::run(x); }
};

// The threads of one line: index lt in [0, tpl) and the barrier they share.
struct LineGroup {
  int lt, tpl, bar;
  __device__ __forceinline__ void sync() const {
    if (tpl == 32)
      __syncwarp();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(tpl) : "memory");
  }
};

template <typename V, int R, bool INV>
__device__ __forceinline__ void line_stage(const V* __restrict__ in, V* __restrict__ out,
                                           const Stage& s, const V* __restrict__ tw,
                                           const LineGroup& g) {
  for (int j = g.lt; j < s.nb; j += g.tpl) {
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = in[j + r * s.nb];
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
    for (int r = 0; r < R; ++r) out[base + r * s.Ns] = x[r];
  }
}

// All stages of a line held in a (input) and b (scratch), both in shared
// memory and private to the group; returns the buffer holding the result.
// Callers g.sync() before (after filling a); the call ends with g.sync().
template <typename V, bool INV>
__device__ V* line_fft(V* a, V* b, const LinePlan& lp, const V* __restrict__ tw,
                       const LineGroup& g) {
  for (int s = 0; s < lp.nst; ++s) {
    const Stage& st = lp.st[s];
    switch (st.R) {
      case 2: line_stage<V, 2, INV>(a, b, st, tw, g); break;
      case 3: line_stage<V, 3, INV>(a, b, st, tw, g); break;
      case 4: line_stage<V, 4, INV>(a, b, st, tw, g); break;
      case 5: line_stage<V, 5, INV>(a, b, st, tw, g); break;
      case 7: line_stage<V, 7, INV>(a, b, st, tw, g); break;
      default: line_stage<V, 8, INV>(a, b, st, tw, g); break;
    }
    g.sync();
    V* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace kde
