// Kernel values on the lag lattice (Eq. 6) and the small index helpers
// shared by the Stockham and two-phase passes.
#pragma once

#include <cuda_runtime.h>

#include "../../include/kde_gb300.h"

namespace kde {

template <typename T>
struct KGen {
  int d;
  int L[KDE_MAX_D];
  int wand;
  // -q/2 = sum_k D_k u_k^2, u_k = m_k + sum_{j<k} B_kj m_j, m = l (|l| in
  // Wand's layout): the squares completed from the Cholesky factor of the
  // bandwidth; B = {B_10, B_20, B_21}, each the sum Bh + Bl of two T.
  T D[KDE_MAX_D];
  T Bh[3], Bl[3];
  T C;                        // (2 pi)^{-d/2} |H|^{-1/2} / (n 2^32 prod P)
};

__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float ex2(float x) { return exp2f(x); }
__device__ __forceinline__ double ex2(double x) { return exp2(x); }

// b m as the sum of the rounded product and its error (exact in FP32 up to
// b's own split into bh + bl).
template <typename T>
__device__ __forceinline__ T prod_lo(T bh, T bl, T m, T hi) {
  return fma(bh, m, -hi) + bl * m;
}

// k at lag l (Eq. 6 with the normalisations folded in).  The quadratic form
// is evaluated in completed squares: a nearly singular bandwidth would lose
// the small exponents near its long axis to cancellation in the expanded
// sum of A_ab l_a l_b.
template <typename T>
__device__ __forceinline__ T kernel_value(const KGen<T>& g, const int* l) {
  T m[KDE_MAX_D];
#pragma unroll
  for (int a = 0; a < KDE_MAX_D; ++a) m[a] = (a < g.d) ? (T)(g.wand ? abs(l[a]) : l[a]) : T(0);
  T e = g.D[0] * m[0] * m[0];
  if (g.d >= 2) {
    const T t = g.Bh[0] * m[0];
    const T u = (m[1] + t) + prod_lo(g.Bh[0], g.Bl[0], m[0], t);
    e = fma(g.D[1] * u, u, e);
  }
  if (g.d == 3) {
    const T t0 = g.Bh[1] * m[0], t1 = g.Bh[2] * m[1];
    const T u = ((m[2] + t0) + t1) + (prod_lo(g.Bh[1], g.Bl[1], m[0], t0) +
                                      prod_lo(g.Bh[2], g.Bl[2], m[1], t1));
    e = fma(g.D[2] * u, u, e);
  }
  return g.C * ex(e);
}

// Signed lag stored at wrapped position p of a length-P axis with support L,
// or a value > L if the position holds zero padding.
__device__ __forceinline__ int wrapped_lag(int p, int P, int L) {
  if (p <= L) return p;
  if (p >= P - L) return p - P;
  return L + 1;
}

// Input row feeding transform position pos: with Lw >= 0 the input rows hold
// the lags -Lw .. Lw placed at l mod P; otherwise row n sits at position n.
// Returns a value >= Nin for positions that hold zero padding.
__device__ __forceinline__ int source_row(int pos, int P, int Lw, int Nin) {
  if (Lw < 0) return pos;
  const int l = wrapped_lag(pos, P, Lw);
  return (l <= Lw) ? l + Lw : Nin;
}

// A count (int64, units of 2^-32) in the evaluation type.  Converting a
// 64-bit integer directly is slow on sm_103 (measured: about 2 us of a
// 1024-row pass); the value is rebuilt from its two 32-bit halves instead.
// FP64: hi 2^32 + lo is exact and the fma rounds once, the same result as a
// direct conversion.  FP32: the low half rounds once more (within one ulp).
template <typename T> __device__ __forceinline__ T count_value(long long v);
template <> __device__ __forceinline__ float count_value<float>(long long v) {
  return fmaf((float)(int)(v >> 32), 4294967296.0f, (float)(unsigned)(unsigned long long)v);
}
template <> __device__ __forceinline__ double count_value<double>(long long v) {
  return fma((double)(int)(v >> 32), 4294967296.0, (double)(unsigned)(unsigned long long)v);
}

}  // namespace kde
